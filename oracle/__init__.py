"""ctypes wrapper of the FP64 CPU oracle (oracle/gv_oracle.c).

TEST INFRASTRUCTURE ONLY: tests/, the smoke check and the CPU-baseline leg of
bench.py may import this module; the product package never does.  The oracle
shares no code with the CUDA path; the only thing both sides share is the
seeded input module (paper_2005_00949_gb300.workloads), which carries data and
no transport arithmetic.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gv_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

GAMMA, ELECTRON, POSITRON = 0, 1, 2
M_COMPTON, M_PAIR, M_BREM, M_MOLLER, M_BHABHA, M_ANNIH = range(6)
NCOUNT = 12
COUNTER_NAMES = ["steps", "steps_gamma", "steps_eminus", "steps_eplus", "tracks_gamma",
                 "tracks_eminus", "tracks_eplus", "n_pair", "n_annih", "eplus_escaped",
                 "unscattered", "spare"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE FP64: no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "gv_oracle.h"))):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


class OrMaterial(C.Structure):
    _fields_ = [("n_elem", C.c_int), ("Z", C.c_double * 4), ("A", C.c_double * 4),
                ("w", C.c_double * 4), ("rho", C.c_double), ("I_eV", C.c_double)]


class OrSetup(C.Structure):
    _fields_ = [("n_mat", C.c_int), ("mat", OrMaterial * 4), ("n_layers", C.c_int),
                ("n_sub", C.c_int), ("sub_thick", C.c_double * 8), ("sub_mat", C.c_int * 8),
                ("half_x", C.c_double), ("half_y", C.c_double), ("nx", C.c_int), ("ny", C.c_int),
                ("gamma_cut", C.c_double), ("e_cut", C.c_double), ("track_cut", C.c_double),
                ("process_mask", C.c_uint), ("field_T", C.c_double), ("field_axis", C.c_int),
                ("reject_min", C.c_double * 6), ("exact", C.c_int)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            d, i, u, p = C.c_double, C.c_int, C.c_uint32, C.c_void_p
            lib.or_create.argtypes = [C.POINTER(OrSetup), C.POINTER(p)]
            lib.or_destroy.argtypes = [p]
            lib.or_material_X0.restype = d
            lib.or_material_X0.argtypes = [p, i]
            lib.or_material_nel.restype = d
            lib.or_material_nel.argtypes = [p, i]
            lib.or_klein_nishina_e.restype = d
            lib.or_klein_nishina_e.argtypes = [d]
            lib.or_xs.restype = d
            lib.or_xs.argtypes = [p, i, i, i, d]
            lib.or_dedx.restype = d
            lib.or_dedx.argtypes = [p, i, i, d]
            lib.or_dedx_parts.restype = d
            lib.or_dedx_parts.argtypes = [p, i, i, d, d, d, C.POINTER(d), C.POINTER(d)]
            lib.or_range_exact.restype = d
            lib.or_range_exact.argtypes = [p, i, i, d]
            lib.or_dcs.restype = d
            lib.or_dcs.argtypes = [i, d, d, d]
            lib.or_grid_size.restype = i
            lib.or_grid_energy.restype = d
            lib.or_grid_energy.argtypes = [i]
            lib.or_table_node.restype = d
            lib.or_table_node.argtypes = [p, i, i, i, i]
            lib.or_table_lookup.restype = d
            lib.or_table_lookup.argtypes = [p, i, i, i, d]
            lib.or_eloss.restype = d
            lib.or_eloss.argtypes = [p, i, i, d, d]
            lib.or_alias_info.argtypes = [p, i, C.POINTER(d), C.POINTER(i)]
            lib.or_alias_table.argtypes = [p, i, i, p, p, p]
            lib.or_alias_sample.restype = d
            lib.or_alias_sample.argtypes = [p, i, d, p, p]
            lib.or_philox4x32_10.argtypes = [p, p, p]
            lib.or_n_subtotal.argtypes = [p]
            lib.or_plane_z.restype = d
            lib.or_plane_z.argtypes = [p, i]
            lib.or_locate.argtypes = [p, d, d]
            lib.or_distance.restype = d
            lib.or_distance.argtypes = [p, p, p, i, C.POINTER(i), C.POINTER(i)]
            lib.or_interact.argtypes = [p, i, i, d, p, p, p, p]
            lib.or_has_rejection.argtypes = [i]
            lib.or_sigma_max.restype = d
            lib.or_sigma_max.argtypes = [p, i, i, d]
            lib.or_reject_sample.restype = d
            lib.or_reject_sample.argtypes = [p, i, d, p, C.POINTER(d), C.POINTER(i)]
            lib.or_exact_sample.restype = d
            lib.or_exact_sample.argtypes = [p, i, d, p, C.POINTER(d), C.POINTER(i)]
            lib.or_range_at.restype = d
            lib.or_range_at.argtypes = [p, i, i, d]
            lib.or_eloss_exact.restype = d
            lib.or_eloss_exact.argtypes = [p, i, i, d, d]
            lib.or_safety.restype = d
            lib.or_safety.argtypes = [p, p, i]
            lib.or_msc_theta0.restype = d
            lib.or_msc_theta0.argtypes = [p, i, d, d]
            lib.or_msc.argtypes = [p, i, d, d, d, p, p, p, p, p]
            lib.or_field_step_limit.restype = d
            lib.or_field_step_limit.argtypes = [p, i, d, p]
            lib.or_helix.argtypes = [p, i, d, d, p, p, p]
            lib.or_transport.argtypes = [p, p, C.c_long, C.c_long, C.c_uint64, p, p, p, p, i]
            lib.or_transport_events.argtypes = [p, p, C.c_long, C.c_long, C.c_long, C.c_uint64, p, p, p, p, i]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 of one counter (4 x u32) and key (2 x u32)."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib.or_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return o


def klein_nishina_e(k: float) -> float:
    return _load().or_klein_nishina_e(k)


class Oracle:
    """One oracle context: materials, geometry, cuts, FP64 tables.

    exact=True selects the untabulated transport: cross sections from their
    formulas at each track's own energy, range and continuous loss by
    quadrature and root finding, every final state by rejection from its
    DCS.  The default transport interpolates the stepping tables and samples
    the sampling tables, as the paper's method does (Sec. 3.5, Sec. 6.3)."""

    def __init__(self, wl, exact: bool = False):
        self.wl = wl
        self.exact = bool(exact)
        lib = _load()
        s = OrSetup()
        s.n_mat = len(wl.materials)
        for m, mat in enumerate(wl.materials):
            s.mat[m].n_elem = len(mat.Z)
            for j in range(len(mat.Z)):
                s.mat[m].Z[j] = mat.Z[j]
                s.mat[m].A[j] = mat.A[j]
                s.mat[m].w[j] = mat.w[j]
            s.mat[m].rho = mat.rho
            s.mat[m].I_eV = mat.I_eV
        s.n_layers = wl.n_layers
        s.n_sub = len(wl.sub_thick)
        for j, t in enumerate(wl.sub_thick):
            s.sub_thick[j] = t
            s.sub_mat[j] = wl.sub_mat[j]
        s.half_x, s.half_y, s.nx, s.ny = wl.half_x, wl.half_y, wl.nx, wl.ny
        s.gamma_cut, s.e_cut, s.track_cut = wl.gamma_cut, wl.e_cut, wl.track_cut
        s.process_mask = wl.process_mask
        s.field_T, s.field_axis = wl.field_T, wl.field_axis
        for m in range(6):
            s.reject_min[m] = wl.reject_min[m] if wl.reject_min is not None else math.inf
        s.exact = 1 if exact else 0
        self._setup = s
        h = C.c_void_p()
        rc = lib.or_create(C.byref(s), C.byref(h))
        if rc != 0:
            raise ValueError(f"or_create failed ({rc})")
        self.h = h
        self.lib = lib

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.or_destroy(self.h)
            self.h = None

    # -- physics
    def X0(self, mat: int) -> float:
        return self.lib.or_material_X0(self.h, mat)

    def n_el(self, mat: int) -> float:
        return self.lib.or_material_nel(self.h, mat)

    def xs(self, ptype: int, proc: int, mat: int, E: float) -> float:
        return self.lib.or_xs(self.h, ptype, proc, mat, E)

    def dedx(self, ptype: int, mat: int, E: float) -> float:
        return self.lib.or_dedx(self.h, ptype, mat, E)

    def dedx_parts(self, ptype, mat, E, cut_e, cut_g):
        a, b = C.c_double(), C.c_double()
        t = self.lib.or_dedx_parts(self.h, ptype, mat, E, cut_e, cut_g, C.byref(a), C.byref(b))
        return t, a.value, b.value

    def range_exact(self, ptype: int, mat: int, E: float) -> float:
        return self.lib.or_range_exact(self.h, ptype, mat, E)

    @staticmethod
    def dcs(model: int, E: float, v: float, cut: float = 0.0) -> float:
        return _load().or_dcs(model, E, v, cut)

    # -- tables
    @staticmethod
    def grid():
        lib = _load()
        return np.array([lib.or_grid_energy(i) for i in range(lib.or_grid_size())])

    def table_nodes(self, ptype: int, q: int, mat: int) -> np.ndarray:
        n = self.lib.or_grid_size()
        return np.array([self.lib.or_table_node(self.h, ptype, q, mat, i) for i in range(n)])

    def lookup(self, ptype: int, q: int, mat: int, E) -> np.ndarray:
        E = np.atleast_1d(np.asarray(E, dtype=np.float64))
        return np.array([self.lib.or_table_lookup(self.h, ptype, q, mat, float(e)) for e in E])

    def eloss(self, ptype: int, mat: int, E, s) -> np.ndarray:
        E = np.atleast_1d(np.asarray(E, dtype=np.float64))
        s = np.broadcast_to(np.asarray(s, dtype=np.float64), E.shape)
        return np.array([self.lib.or_eloss(self.h, ptype, mat, float(e), float(x))
                         for e, x in zip(E, s)])

    def alias_info(self, model: int):
        e, n = C.c_double(), C.c_int()
        self.lib.or_alias_info(self.h, model, C.byref(e), C.byref(n))
        return e.value, n.value

    def alias_table(self, model: int, ie: int):
        pdf = np.zeros(65)
        q = np.zeros(64, dtype=np.float32)
        a = np.zeros(64, dtype=np.int32)
        rc = self.lib.or_alias_table(self.h, model, ie, _ptr(pdf), _ptr(q), _ptr(a))
        if rc != 0:
            raise IndexError(ie)
        return pdf, q, a

    def alias_sample(self, model: int, E, u: np.ndarray):
        """Sample the physical variable for each energy E[i] with uniforms u[i, 0:3]."""
        E = np.atleast_1d(np.asarray(E, dtype=np.float64))
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(len(E), 3)
        out = np.empty(len(E))
        xi = np.empty(len(E))
        x = C.c_double()
        for i in range(len(E)):
            out[i] = self.lib.or_alias_sample(self.h, model, float(E[i]), _ptr(u[i]), C.byref(x))
            xi[i] = x.value
        return out, xi

    def interact(self, ptype: int, proc: int, E: float, d, u, rng=(0, 0, 0, 0, 0)) -> tuple:
        """rng: (id_lo, id_hi, step, key0, key1) of the interacting step (the
        rejection samplers' stream)."""
        dd = np.ascontiguousarray(d, dtype=np.float64)
        uu = np.ascontiguousarray(u, dtype=np.float64)
        rr = np.ascontiguousarray(rng, dtype=np.uint32)
        out = np.zeros(24)
        r = self.lib.or_interact(self.h, ptype, proc, E, _ptr(dd), _ptr(uu), _ptr(rr), _ptr(out))
        return r, out

    def sigma_max(self, ptype: int, mat: int, E) -> np.ndarray:
        E = np.atleast_1d(np.asarray(E, dtype=np.float64))
        return np.array([self.lib.or_sigma_max(self.h, ptype, mat, float(e)) for e in E])

    @staticmethod
    def has_rejection(model: int) -> bool:
        return bool(_load().or_has_rejection(model))

    def reject_sample(self, model: int, E: float, rng) -> tuple:
        """(physical variable, reduced variable, trials) by rejection."""
        rr = np.ascontiguousarray(rng, dtype=np.uint32)
        xi, tr = C.c_double(), C.c_int()
        v = self.lib.or_reject_sample(self.h, model, E, _ptr(rr), C.byref(xi), C.byref(tr))
        return v, xi.value, tr.value

    def exact_sample(self, model: int, E: float, rng) -> tuple:
        """(physical variable, proposal uniform, trials) from the exact sampler of
        any of the six models."""
        rr = np.ascontiguousarray(rng, dtype=np.uint32)
        xi, tr = C.c_double(), C.c_int()
        v = self.lib.or_exact_sample(self.h, model, E, _ptr(rr), C.byref(xi), C.byref(tr))
        return v, xi.value, tr.value

    def range_at(self, ptype: int, mat: int, E: float) -> float:
        """Untabulated range R(E) (node quadratures plus the partial interval)."""
        return self.lib.or_range_at(self.h, ptype, mat, E)

    def eloss_exact(self, ptype: int, mat: int, E: float, s: float) -> float:
        """Untabulated post-step energy: the root of int_{E'}^{E} dE/S = s."""
        return self.lib.or_eloss_exact(self.h, ptype, mat, E, s)

    # -- geometry
    def n_subtotal(self) -> int:
        return self.lib.or_n_subtotal(self.h)

    def plane_z(self, k: int) -> float:
        return self.lib.or_plane_z(self.h, k)

    def locate(self, z: float, w: float) -> int:
        return self.lib.or_locate(self.h, z, w)

    def distance(self, pos, d, sub: int):
        p = np.ascontiguousarray(pos, dtype=np.float64)
        q = np.ascontiguousarray(d, dtype=np.float64)
        nx, pl = C.c_int(), C.c_int()
        s = self.lib.or_distance(self.h, _ptr(p), _ptr(q), sub, C.byref(nx), C.byref(pl))
        return s, nx.value, pl.value

    def safety(self, pos, sub: int) -> float:
        p = np.ascontiguousarray(pos, dtype=np.float64)
        return self.lib.or_safety(self.h, _ptr(p), sub)

    # -- multiple scattering
    def msc_theta0(self, mat: int, T: float, s: float) -> float:
        return self.lib.or_msc_theta0(self.h, mat, T, s)

    def msc(self, sub: int, E_pre: float, E_post: float, s: float, d, pos, u):
        """(new direction, new position) after Gaussian scattering over a step."""
        dd = np.ascontiguousarray(d, dtype=np.float64)
        pp = np.ascontiguousarray(pos, dtype=np.float64)
        uu = np.ascontiguousarray(u, dtype=np.float64)
        od, op = np.zeros(3), np.zeros(3)
        self.lib.or_msc(self.h, sub, E_pre, E_post, s, _ptr(dd), _ptr(pp), _ptr(uu), _ptr(od), _ptr(op))
        return od, op

    # -- magnetic field
    def field_step_limit(self, ptype: int, E: float, d) -> float:
        dd = np.ascontiguousarray(d, dtype=np.float64)
        return self.lib.or_field_step_limit(self.h, ptype, E, _ptr(dd))

    def helix(self, ptype: int, E: float, s: float, d):
        """(displacement, new direction) along the helix after a path s."""
        dd = np.ascontiguousarray(d, dtype=np.float64)
        dp, nd = np.zeros(3), np.zeros(3)
        self.lib.or_helix(self.h, ptype, E, s, _ptr(dd), _ptr(dp), _ptr(nd))
        return dp, nd

    # -- transport
    def transport(self, primaries=None, n_events=None, seed=None, n_threads: int = 1,
                  cells: bool = True, first_event: int = 0):
        """Transport the workload's primaries (rows: events first_event ..
        first_event + n_events - 1, keyed by their global index)."""
        wl = self.wl
        p = wl.primaries if primaries is None else primaries
        p = np.ascontiguousarray(p)
        n_events = wl.n_events if n_events is None else n_events
        seed = wl.seed if seed is None else seed
        nsub = self.n_subtotal()
        edep = np.zeros((n_events, nsub))
        esc = np.zeros(n_events)
        cnt = np.zeros((n_events, NCOUNT), dtype=np.int64)
        ncell = wl.n_layers * wl.nx * wl.ny
        cell = np.zeros(max(ncell, 1)) if (cells and ncell > 0) else None
        rc = self.lib.or_transport_events(self.h, _ptr(p), len(p), first_event, n_events, C.c_uint64(seed),
                                          _ptr(edep), _ptr(cell) if cell is not None else None,
                                          _ptr(esc), _ptr(cnt), n_threads)
        if rc != 0:
            raise ValueError(f"or_transport failed ({rc})")
        res = {"edep": edep, "escape": esc, "counts": cnt}
        if cell is not None:
            res["cell"] = cell.reshape(wl.n_layers, wl.nx, wl.ny)
        return res
