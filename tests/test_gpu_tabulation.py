"""The mixed-precision GPU transport against the untabulated oracle.

The GPU's tables (FP32, interpolated in ln E; sampling tables) and its FP32
arithmetic are compared, whole showers against whole showers, with the
oracle's untabulated transport (every quantity from its definition; FP64),
whose reference statistics tests/golden/make_exact_showers.py stored by
running only the oracle.  Criteria of the shower parity: every layer within
3 combined standard errors, 0.5 % where that bound is active, per-material
totals likewise.  The GPU samples use the workloads' default seed, the
stored ones another: the two are independent.
"""
import json
import os

import pytest

from paper_2005_00949_gb300 import workloads as W

import shower_stats as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gvmod():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__
    __graft_entry__.build()
    from paper_2005_00949_gb300 import gv
    return gv


@pytest.mark.parametrize("n,E,golden", [
    (200_000, 1000.0, "exact_showers_e-1GeV_PbPS50.txt"),
    (65_536, 10_000.0, "exact_showers_e-10GeV_PbPS50.txt"),
], ids=["1GeV", "10GeV"])
def test_mixed_gpu_matches_untabulated_oracle(gvmod, n, E, golden):
    wl = W.pbps_electrons(n, E)
    ctx = gvmod.Context(wl, gvmod.gv_default_config(stack_capacity=1 << 23))
    r = ctx.transport(cells=False)
    ctx.close()
    assert r["status"] == 0
    got = S.compare(S.summarize(r["edep"], wl.n_layers), S.read(golden))
    assert got["active_layers"] >= 5, got
    assert got["active_materials"] == 2, got
    path = os.environ.get("GV_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"name": f"mixed_gpu_vs_untabulated_{E:g}MeV", "events": n, **got}) + "\n")


@pytest.mark.parametrize("make,golden", [
    (lambda: W.wsi_cells(2048, 100_000.0), "exact_showers_e-100GeV_WSi50.txt"),
    (lambda: W.with_msc(W.with_field(W.pblar_testem3(8192, 10_000.0), 4.0, 1)),
     "exact_showers_e-10GeV_PbLAr50_4T_msc.txt"),
], ids=["WSi_100GeV", "PbLAr_4T_msc"])
def test_mixed_gpu_matches_untabulated_oracle_other_layouts(gvmod, make, golden):
    """The W/Si cell calorimeter (0.5 MeV cuts) and the TestEm3 layout with
    its 4 T field and multiple scattering: per-layer and per-material
    criteria against the untabulated transport's stored showers."""
    wl = make()
    ctx = gvmod.Context(wl, gvmod.gv_default_config(stack_capacity=1 << 23))
    r = ctx.transport(cells=False)
    ctx.close()
    assert r["status"] == 0
    got = S.compare(S.summarize(r["edep"], wl.n_layers), S.read(golden))
    assert got["active_materials"] == 2, got
    path = os.environ.get("GV_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"name": f"mixed_gpu_vs_untabulated_{wl.name}", "events": wl.n_events, **got}) + "\n")
