"""Showers with multiple scattering (GV_P_MSC), in a magnetic field, with
rejection samplers and with the integral approach (GV_P_INTEGRAL), against
the oracle.

The scattering draws its uniforms from counter block 2 of each step on both
sides, so FP64 histories coincide with the oracle's event by event, and the
mixed-precision path is compared on per-layer means (and on cells where the
workload has them)."""
import numpy as np
import pytest

from paper_2005_00949_gb300 import workloads as W
from test_gpu_workloads import _conservation, _layer_stats, _report, _run
from test_gpu_transport import NTHR, _ctx, gvmod, layer_parity  # noqa: F401

pytestmark = pytest.mark.gpu


def test_fp64_msc_showers_follow_oracle_event_by_event(gvmod, oracle_mod):
    wl = W.with_msc(W.pbps_electrons(300, 1000.0))
    r = _run(gvmod, wl, precision=1, per_event_counts=1)
    ref = oracle_mod.Oracle(wl).transport(n_threads=NTHR)
    same = np.all(r["counts"][:, :11] == ref["counts"][:, :11], axis=1)
    assert same.mean() >= 0.9, same.mean()
    assert np.abs(r["edep"][same] - ref["edep"][same]).max() < 1e-9 * 1000.0
    # scattering changes the showers: the same events without it differ
    plain = oracle_mod.Oracle(W.pbps_electrons(300, 1000.0)).transport(n_threads=NTHR)
    assert not np.array_equal(plain["counts"], ref["counts"])


def test_mixed_msc_showers_and_conservation(gvmod, oracle_mod):
    wl = W.with_msc(W.pbps_electrons(20_000, 1000.0))
    r = _run(gvmod, wl, per_event_counts=1)
    ref = oracle_mod.Oracle(wl).transport(n_threads=NTHR)
    layer_parity(wl, r["edep"], ref["edep"])
    assert np.abs(_conservation(wl, r)).max() < 1e-5
    assert np.all(r["counts"][:, 7] == r["counts"][:, 8] + r["counts"][:, 9])


def test_msc_cells_wsi(gvmod, oracle_mod):
    """Lateral spread: the cell histogram of 100 GeV showers in W/Si."""
    wl = W.with_msc(W.wsi_cells(300, 100_000.0))
    r = _run(gvmod, wl, stack_capacity=1 << 23)
    ref = oracle_mod.Oracle(wl).transport(n_threads=NTHR)
    layer_parity(wl, r["edep"], ref["edep"])
    per_layer = r["edep"].reshape(300, 50, 2).sum((0, 2))
    assert np.allclose(r["cell"].sum((1, 2)), per_layer, rtol=1e-9)
    # radial profile: fraction of the deposit in rings of cells around the beam
    def rings(cell):
        tot = cell.sum()
        out = []
        for k in (2, 4, 8):
            out.append(cell[:, 16 - k:16 + k, 16 - k:16 + k].sum() / tot)
        return np.array(out)
    assert np.abs(rings(r["cell"]) - rings(ref["cell"])).max() < 0.005


def test_msc_testem3_and_bench_workload_measured(gvmod, oracle_mod):
    """The paper's TestEm3 layout with scattering (still without its field),
    and the benchmark workload with scattering on: parity and timing."""
    wl = W.with_msc(W.pblar_testem3(1000, 10_000.0))
    r = _run(gvmod, wl, per_event_counts=1)
    ref = oracle_mod.Oracle(wl).transport(n_threads=NTHR)
    layer_parity(wl, r["edep"], ref["edep"])
    mat = r["edep"].reshape(wl.n_events, 50, 2).sum(1).mean(0)
    cnt = r["counts"].mean(0)
    _report("testem3_PbLAr_10GeV_msc", events=wl.n_events, kernel_ms=r["kernel_ms"],
            edep_Pb_GeV=float(mat[0] / 1e3), edep_LAr_GeV=float(mat[1] / 1e3),
            gammas=float(cnt[4]), electrons=float(cnt[5] - 1), positrons=float(cnt[6]),
            charged_steps=float(cnt[2] + cnt[3]), neutral_steps=float(cnt[1]),
            layers=_layer_stats(wl, r["edep"], ref["edep"]))
    wl4 = W.with_msc(W.standard(W.PBPS_10GEV))
    r4 = _run(gvmod, wl4, stack_capacity=1 << 23)
    ref4 = oracle_mod.Oracle(wl4).transport(n_threads=NTHR)
    layer_parity(wl4, r4["edep"], ref4["edep"])
    c = r4["counters"]
    _report("e-10GeV_PbPS50_msc", events=wl4.n_events, kernel_ms=r4["kernel_ms"],
            events_per_s=wl4.n_events / (r4["kernel_ms"] / 1e3), steps_per_s=c["steps"] / (r4["kernel_ms"] / 1e3),
            steps=c["steps"], layers=_layer_stats(wl4, r4["edep"], ref4["edep"]))


# ---------------------------------------------------------------- magnetic field
def test_fp64_field_showers_follow_oracle_event_by_event(gvmod, oracle_mod):
    wl = W.with_field(W.pblar_testem3(300, 1000.0), 4.0, 1)
    r = _run(gvmod, wl, precision=1, per_event_counts=1)
    ref = oracle_mod.Oracle(wl).transport(n_threads=NTHR)
    same = np.all(r["counts"][:, :11] == ref["counts"][:, :11], axis=1)
    assert same.mean() >= 0.9, same.mean()
    assert np.abs(r["edep"][same] - ref["edep"][same]).max() < 1e-9 * 1000.0


def test_fp64_all_options_follow_oracle_event_by_event(gvmod, oracle_mod):
    """Every option at once in FP64 -- multiple scattering, a 4 T field,
    rejection samplers and the integral approach -- on the TestEm3 layout:
    the histories coincide with the oracle's event by event."""
    wl = W.with_integral(W.with_rejection(W.with_msc(W.with_field(W.pblar_testem3(200, 1000.0), 4.0, 1))))
    r = _run(gvmod, wl, precision=1, per_event_counts=1)
    ref = oracle_mod.Oracle(wl).transport(n_threads=NTHR)
    same = np.all(r["counts"][:, :11] == ref["counts"][:, :11], axis=1)
    assert same.mean() >= 0.9, same.mean()
    assert np.abs(r["edep"][same] - ref["edep"][same]).max() < 1e-9 * 1000.0
    assert np.abs(_conservation(wl, r)).max() < 1e-9


def test_mixed_all_options_cells_statistical(gvmod, oracle_mod):
    """Every option at once in mixed precision on the segmented W/Si
    calorimeter (cells scored at the helix midpoint): per-layer means and the
    lateral profile against the oracle."""
    wl = W.with_integral(W.with_rejection(W.with_msc(W.with_field(W.wsi_cells(400, 20_000.0), 4.0, 1))))
    r = _run(gvmod, wl, stack_capacity=1 << 23, per_event_counts=1)
    ref = oracle_mod.Oracle(wl).transport(n_threads=NTHR)
    layer_parity(wl, r["edep"], ref["edep"])
    assert np.abs(_conservation(wl, r)).max() < 1e-5
    per_layer = r["edep"].reshape(wl.n_events, wl.n_layers, -1).sum((0, 2))
    assert np.allclose(r["cell"].sum((1, 2)), per_layer, rtol=1e-9)

    def rings(cell):
        tot = cell.sum()
        return np.array([cell[:, 16 - k:16 + k, 16 - k:16 + k].sum() / tot for k in (2, 4, 8)])
    assert np.abs(rings(r["cell"]) - rings(ref["cell"])).max() < 0.005


def test_testem3_field_and_msc_paper_conditions(gvmod, oracle_mod):
    """The paper's TestEm3 conditions as far as this physics list goes: 50 x
    (2.3 mm Pb + 5.7 mm LAr), 10 GeV e-, 4 T transverse field, multiple
    scattering.  Parity with the oracle (mixed precision), conservation, and
    the per-material deposits and counts next to the paper's tables."""
    wl = W.with_msc(W.with_field(W.pblar_testem3(1000, 10_000.0), 4.0, 1))
    r = _run(gvmod, wl, per_event_counts=1)
    ref = oracle_mod.Oracle(wl).transport(n_threads=NTHR)
    layer_parity(wl, r["edep"], ref["edep"])
    assert np.abs(_conservation(wl, r)).max() < 1e-5
    mat = r["edep"].reshape(wl.n_events, 50, 2).sum(1).mean(0)
    cnt = r["counts"].mean(0)
    _report("testem3_PbLAr_10GeV_4T_msc", events=wl.n_events, kernel_ms=r["kernel_ms"],
            edep_Pb_GeV=float(mat[0] / 1e3), edep_LAr_GeV=float(mat[1] / 1e3),
            gammas=float(cnt[4]), electrons=float(cnt[5] - 1), positrons=float(cnt[6]),
            charged_steps=float(cnt[2] + cnt[3]), neutral_steps=float(cnt[1]),
            layers=_layer_stats(wl, r["edep"], ref["edep"]))


# ---------------------------------------------------------------- rejection samplers
def test_fp64_rejection_showers_follow_oracle_event_by_event(gvmod, oracle_mod):
    wl = W.with_rejection(W.pbps_electrons(300, 1000.0))
    r = _run(gvmod, wl, precision=1, per_event_counts=1)
    ref = oracle_mod.Oracle(wl).transport(n_threads=NTHR)
    same = np.all(r["counts"][:, :11] == ref["counts"][:, :11], axis=1)
    assert same.mean() >= 0.9, same.mean()
    assert np.abs(r["edep"][same] - ref["edep"][same]).max() < 1e-9 * 1000.0


def test_mixed_rejection_showers_and_measured(gvmod, oracle_mod):
    wl = W.with_rejection(W.standard(W.PBPS_10GEV))
    r = _run(gvmod, wl, stack_capacity=1 << 23)
    ref = oracle_mod.Oracle(wl).transport(n_threads=NTHR)
    layer_parity(wl, r["edep"], ref["edep"])
    c = r["counters"]
    _report("e-10GeV_PbPS50_rejection", events=wl.n_events, kernel_ms=r["kernel_ms"],
            events_per_s=wl.n_events / (r["kernel_ms"] / 1e3), steps=c["steps"],
            layers=_layer_stats(wl, r["edep"], ref["edep"]))


# ---------------------------------------------------------------- integral approach
def test_fp64_integral_showers_follow_oracle_event_by_event(gvmod, oracle_mod):
    wl = W.with_integral(W.pbps_mixed(300).subset(300))
    wl.primaries["E"] = np.minimum(wl.primaries["E"], 3000.0)
    r = _run(gvmod, wl, precision=1, per_event_counts=1)
    ref = oracle_mod.Oracle(wl).transport(n_threads=NTHR)
    same = np.all(r["counts"][:, :11] == ref["counts"][:, :11], axis=1)
    assert same.mean() >= 0.9, same.mean()
    assert np.abs(r["edep"][same] - ref["edep"][same]).max() < 1e-9 * 3000.0


def test_mixed_integral_showers_and_measured(gvmod, oracle_mod):
    wl = W.with_integral(W.standard(W.PBPS_10GEV))
    r = _run(gvmod, wl, stack_capacity=1 << 23, per_event_counts=1)
    ref = oracle_mod.Oracle(wl).transport(n_threads=NTHR)
    layer_parity(wl, r["edep"], ref["edep"])
    assert np.abs(_conservation(wl, r)).max() < 1e-5
    c = r["counters"]
    _report("e-10GeV_PbPS50_integral", events=wl.n_events, kernel_ms=r["kernel_ms"],
            events_per_s=wl.n_events / (r["kernel_ms"] / 1e3), steps=c["steps"], discrete=c["discrete"],
            layers=_layer_stats(wl, r["edep"], ref["edep"]))
