"""The C-ABI library builds, loads and exports every entry point include/gv.h
declares; argument validation answers without touching a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "gv.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2005_00949_gb300 import build, gv
    build.build()
    return gv.load()


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gv_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_entry_points():
    names = _declared()
    for must in ["gv_setup", "gv_build_tables", "gv_transport", "gv_sync", "gv_destroy",
                 "gv_strerror", "gv_default_config", "gv_unit_philox", "gv_unit_xs_lookup",
                 "gv_unit_eloss", "gv_unit_alias_sample", "gv_unit_interact", "gv_unit_distance"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_struct_layouts_match_header(lib, tmp_path):
    """ctypes mirrors and the primary dtype agree with the C compiler's layout."""
    import subprocess
    from paper_2005_00949_gb300 import gv, workloads as W
    structs = {"gv_material": gv.gv_material, "gv_layers": gv.gv_layers, "gv_cuts": gv.gv_cuts,
               "gv_config": gv.gv_config, "gv_result": gv.gv_result}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void){"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines.append('printf("gv_primary %zu\\n", sizeof(gv_primary));')
    for f in W.PRIMARY_DTYPE.names:
        cf = "E_MeV" if f == "E" else f
        lines.append(f'printf("gv_primary.{f} %zu\\n", offsetof(gv_primary, {cf}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-o", str(exe), str(src)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)]).decode().splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == C.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(cls, f).offset, (name, f)
    assert int(got["gv_primary"]) == W.PRIMARY_DTYPE.itemsize
    for f in W.PRIMARY_DTYPE.names:
        assert int(got[f"gv_primary.{f}"]) == W.PRIMARY_DTYPE.fields[f][1], f
    cfg = gv.gv_default_config()
    assert cfg.precision == gv.GV_MIXED and cfg.block_size % 32 == 0


def test_argument_validation_without_gpu(lib):
    from paper_2005_00949_gb300 import gv
    h = C.c_void_p()
    # no materials -> BAD_ARG before any CUDA call
    assert lib.gv_setup(C.byref(h), None, 0, None, None, None) == -1
    mats = (gv.gv_material * 1)()
    mats[0].n_elem = 1
    mats[0].Z[0], mats[0].A[0], mats[0].w[0], mats[0].rho, mats[0].I_eV = 82, 207.2, 1, 11.35, 823
    geo = gv.gv_layers()
    geo.n_layers, geo.n_sub = 10, 1
    geo.sub_thick_cm[0] = 0.5
    cuts = gv.gv_cuts(1.0, 1.0, 1e-3, 63)
    bad = gv.gv_cuts(1.0, 1.0, 1e-4, 63)  # track cut below the table grid
    assert lib.gv_setup(C.byref(h), mats, 1, C.byref(geo), C.byref(bad), None) == -1
    geo2 = gv.gv_layers()
    geo2.n_layers, geo2.n_sub = 2000, 1  # more sub-slabs than GV_MAX_SUBTOTAL
    geo2.sub_thick_cm[0] = 0.5
    assert lib.gv_setup(C.byref(h), mats, 1, C.byref(geo2), C.byref(cuts), None) == -1
    cfg = gv.gv_default_config(block_size=100)
    assert lib.gv_setup(C.byref(h), mats, 1, C.byref(geo), C.byref(cuts), C.byref(cfg)) == -1
    # every malformed material, geometry or cut is refused before any CUDA call
    def mat_case(**kw):
        m = (gv.gv_material * 1)()
        C.memmove(C.byref(m[0]), C.byref(mats[0]), C.sizeof(gv.gv_material))
        for k, v in kw.items():
            if k in ("Z", "A", "w"):
                getattr(m[0], k)[0] = v
            else:
                setattr(m[0], k, v)
        return m

    for kw in (dict(n_elem=0), dict(n_elem=1000), dict(rho=0.0), dict(rho=float("nan")), dict(I_eV=-1.0),
               dict(Z=0.0), dict(A=0.0), dict(w=0.0)):
        assert lib.gv_setup(C.byref(h), mat_case(**kw), 1, C.byref(geo), C.byref(cuts), None) == -1, kw
    assert lib.gv_setup(C.byref(h), mats, 0, C.byref(geo), C.byref(cuts), None) == -1
    assert lib.gv_setup(C.byref(h), mats, 5, C.byref(geo), C.byref(cuts), None) == -1  # > GV_MAX_MAT

    def geo_case(**kw):
        g = gv.gv_layers()
        C.memmove(C.byref(g), C.byref(geo), C.sizeof(gv.gv_layers))
        for k, v in kw.items():
            if k in ("sub_thick_cm", "sub_mat"):
                getattr(g, k)[0] = v
            else:
                setattr(g, k, v)
        return g

    for kw in (dict(n_layers=0), dict(n_sub=0), dict(n_sub=9), dict(sub_thick_cm=0.0), dict(sub_thick_cm=-1.0),
               dict(sub_mat=1), dict(sub_mat=-1), dict(nx_cells=-1), dict(nx_cells=4, ny_cells=4),
               dict(nx_cells=4, ny_cells=0, half_x_cm=5.0, half_y_cm=5.0), dict(field_T=1e5),
               dict(field_axis=3), dict(field_axis=-1)):
        g = geo_case(**kw)
        assert lib.gv_setup(C.byref(h), mats, 1, C.byref(g), C.byref(cuts), None) == -1, kw
    for bad_cuts in (gv.gv_cuts(1.0, 1.0, float("nan"), 63), gv.gv_cuts(1e-4, 1.0, 1e-3, 63),
                     gv.gv_cuts(1.0, 1e-4, 1e-3, 63)):
        assert lib.gv_setup(C.byref(h), mats, 1, C.byref(geo), C.byref(bad_cuts), None) == -1
    # every knob out of its range is refused before any CUDA call
    for bad_knob in (dict(precision=2), dict(mode=3), dict(block_size=32), dict(block_size=1024),
                     dict(blocks_per_sm=0), dict(steps_per_claim=0), dict(tail_steps_per_claim=5000),
                     dict(stack_capacity=100), dict(refill_batch=0), dict(refill_low_water=-1),
                     dict(generations_per_graph=3), dict(generations_per_graph=0), dict(max_generations=0),
                     dict(max_events_in_flight=-2), dict(claim_chunks=2), dict(along_steps=0),
                     dict(along_steps=65), dict(along_steps_photon=-1), dict(along_steps_photon=65),
                     dict(scoring=2), dict(l2_persist=-1), dict(local_stack=2),
                     dict(pdl=2), dict(device_loop=2), dict(pipeline=2), dict(pipeline=1, scoring=1)):
        cfg = gv.gv_default_config(**bad_knob)
        assert lib.gv_setup(C.byref(h), mats, 1, C.byref(geo), C.byref(cuts), C.byref(cfg)) == -1, bad_knob
    assert lib.gv_transport(None, None, 0, 1, 0, None, None) == -1
    assert lib.gv_unit_philox(None, None, None, 0, None) == 0
    assert lib.gv_unit_philox(None, None, None, -1, None) == -1
    assert lib.gv_strerror(-4) == b"track queue overflow"
    assert lib.gv_last_launches(None) == -1
