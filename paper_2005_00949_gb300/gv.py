"""Thin ctypes binding of libgv.so (include/gv.h): argument marshalling only.

Every step of the transport runs in the library's CUDA kernels; PyTorch is
used only to own device memory and to name CUDA streams.  There is no CPU
fallback: if libgv.so is missing or the GPU is absent the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import workloads as W

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("GV_LIB", os.path.join(_HERE, "libgv.so"))
_lib = None
_lock = threading.Lock()

GV_OK = 0
GV_MIXED, GV_FP64 = 0, 1
GV_BATCHED, GV_ONE_EVENT_PER_LAUNCH = 0, 1
NCOUNT = 12
COUNTER_NAMES = ["steps", "steps_gamma", "steps_eminus", "steps_eplus", "tracks_gamma",
                 "tracks_eminus", "tracks_eplus", "n_pair", "n_annih", "eplus_escaped",
                 "unscattered", "generations", "geom_limited", "discrete", "lane_slots",
                 "live_peak"]


class GvError(RuntimeError):
    pass


class gv_material(C.Structure):
    _fields_ = [("n_elem", C.c_int), ("Z", C.c_double * 4), ("A", C.c_double * 4),
                ("w", C.c_double * 4), ("rho", C.c_double), ("I_eV", C.c_double)]


class gv_layers(C.Structure):
    _fields_ = [("n_layers", C.c_int), ("n_sub", C.c_int), ("sub_thick_cm", C.c_double * 8),
                ("sub_mat", C.c_int * 8), ("half_x_cm", C.c_double), ("half_y_cm", C.c_double),
                ("nx_cells", C.c_int), ("ny_cells", C.c_int), ("field_T", C.c_double),
                ("field_axis", C.c_int)]


class gv_cuts(C.Structure):
    _fields_ = [("gamma_cut_MeV", C.c_double), ("e_cut_MeV", C.c_double),
                ("track_cut_MeV", C.c_double), ("process_mask", C.c_uint),
                ("reject_min_MeV", C.c_double * 6)]


class gv_config(C.Structure):
    _fields_ = [("precision", C.c_int), ("mode", C.c_int), ("block_size", C.c_int),
                ("blocks_per_sm", C.c_int), ("steps_per_claim", C.c_int),
                ("tail_steps_per_claim", C.c_int), ("tail_threshold", C.c_longlong),
                ("stack_capacity", C.c_longlong), ("refill_low_water", C.c_longlong),
                ("refill_batch", C.c_longlong), ("generations_per_graph", C.c_int),
                ("max_generations", C.c_longlong), ("per_event_counts", C.c_int),
                ("process_sort", C.c_int), ("max_events_in_flight", C.c_longlong),
                ("claim_chunks", C.c_int), ("along_steps", C.c_int), ("scoring", C.c_int),
                ("l2_persist", C.c_int), ("pipeline", C.c_int), ("local_stack", C.c_int),
                ("pdl", C.c_int), ("device_loop", C.c_int), ("blocking", C.c_int),
                ("along_steps_photon", C.c_int)]


class gv_result(C.Structure):
    _fields_ = [("edep", C.c_void_p), ("cell_edep", C.c_void_p), ("escape_E", C.c_void_p),
                ("event_counts", C.c_void_p), ("counters", C.c_ulonglong * 16),
                ("status", C.c_int), ("kernel_ms", C.c_double)]


def load():
    """Load libgv.so (built by build.py); raise if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise GvError(f"{LIB_PATH} not built: run paper_2005_00949_gb300/build.py")
            lib = C.CDLL(LIB_PATH)
            vp, i, ll = C.c_void_p, C.c_int, C.c_longlong
            lib.gv_default_config.argtypes = [C.POINTER(gv_config)]
            lib.gv_setup.argtypes = [C.POINTER(vp), C.POINTER(gv_material), i, C.POINTER(gv_layers),
                                     C.POINTER(gv_cuts), C.POINTER(gv_config)]
            lib.gv_build_tables.argtypes = [vp]
            lib.gv_transport.argtypes = [vp, vp, ll, ll, C.c_ulonglong, vp, C.POINTER(gv_result)]
            lib.gv_transport_events.argtypes = [vp, vp, ll, ll, ll, C.c_ulonglong, vp, C.POINTER(gv_result)]
            lib.gv_sync.argtypes = [vp, vp]
            lib.gv_destroy.argtypes = [vp]
            lib.gv_destroy.restype = None
            lib.gv_strerror.argtypes = [i]
            lib.gv_strerror.restype = C.c_char_p
            lib.gv_last_launches.argtypes = [vp]
            lib.gv_last_launches.restype = ll
            lib.gv_transport_static.argtypes = [vp, vp, ll, ll, C.c_ulonglong, vp, vp, vp,
                                                C.POINTER(C.c_ulonglong)]
            lib.gv_unit_philox.argtypes = [vp, vp, vp, ll, vp]
            lib.gv_unit_xs_lookup.argtypes = [vp, i, i, vp, ll, vp, vp]
            lib.gv_unit_eloss.argtypes = [vp, i, i, vp, vp, ll, vp, vp]
            lib.gv_unit_alias_sample.argtypes = [vp, i, vp, vp, ll, vp, vp]
            lib.gv_unit_interact.argtypes = [vp, i, i, vp, vp, vp, ll, vp, vp, vp]
            lib.gv_unit_distance.argtypes = [vp, vp, vp, vp, ll, vp, vp, vp, vp]
            lib.gv_unit_msc.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, ll, vp, vp, vp]
            lib.gv_unit_field.argtypes = [vp, i, vp, vp, vp, ll, vp, vp]
            lib.gv_unit_sample.argtypes = [vp, i, i, vp, ll, C.c_ulonglong, vp, vp]
            _lib = lib
    return _lib


def _check(rc: int, what: str):
    if rc != GV_OK:
        raise GvError(f"{what}: {load().gv_strerror(rc).decode()} ({rc})")


def gv_default_config(**overrides) -> gv_config:
    cfg = gv_config()
    load().gv_default_config(C.byref(cfg))
    for k, v in overrides.items():
        setattr(cfg, k, v)
    return cfg


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _ptr(x):
    """Device or host address of a torch tensor / numpy array (or None)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


class Context:
    """gv_setup + gv_build_tables for one workload geometry / material set."""

    def __init__(self, wl: W.Workload, config: gv_config | None = None, **overrides):
        lib = load()
        self.wl = wl
        mats = (gv_material * len(wl.materials))()
        for m, mat in enumerate(wl.materials):
            mats[m].n_elem = len(mat.Z)
            for j in range(len(mat.Z)):
                mats[m].Z[j], mats[m].A[j], mats[m].w[j] = mat.Z[j], mat.A[j], mat.w[j]
            mats[m].rho, mats[m].I_eV = mat.rho, mat.I_eV
        geo = gv_layers()
        geo.n_layers, geo.n_sub = wl.n_layers, len(wl.sub_thick)
        for j, t in enumerate(wl.sub_thick):
            geo.sub_thick_cm[j] = t
            geo.sub_mat[j] = wl.sub_mat[j]
        geo.half_x_cm, geo.half_y_cm, geo.nx_cells, geo.ny_cells = wl.half_x, wl.half_y, wl.nx, wl.ny
        geo.field_T, geo.field_axis = wl.field_T, wl.field_axis
        cuts = gv_cuts(wl.gamma_cut, wl.e_cut, wl.track_cut, wl.process_mask)
        for m in range(6):
            cuts.reject_min_MeV[m] = wl.reject_min[m] if wl.reject_min is not None else 1e300
        cfg = config if config is not None else gv_default_config()
        for k, v in overrides.items():
            setattr(cfg, k, v)
        self.config = cfg
        h = C.c_void_p()
        _check(lib.gv_setup(C.byref(h), mats, len(wl.materials), C.byref(geo), C.byref(cuts),
                            C.byref(cfg)), "gv_setup")
        self.h = h
        self.lib = lib
        _check(lib.gv_build_tables(h), "gv_build_tables")
        self.last_result = None

    def close(self):
        if getattr(self, "h", None):
            self.lib.gv_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n_subtotal(self) -> int:
        return self.wl.n_layers * len(self.wl.sub_thick)

    def gv_transport(self, primaries, n_events: int, seed: int, edep, cell=None, escape=None,
                     event_counts=None, stream=None, sync: bool = True, first_event: int = 0) -> gv_result:
        """Call gv_transport_events with caller-owned buffers (torch tensors or
        numpy arrays, host or device).  `primaries` is a numpy PRIMARY_DTYPE
        array or a uint8 device tensor holding the same records.  sync=True
        also calls gv_sync (the result record is filled when it returns);
        sync=False returns once the transport is enqueued: call sync() later."""
        n = len(primaries) if isinstance(primaries, np.ndarray) else primaries.numel() // W.PRIMARY_DTYPE.itemsize
        res = gv_result()
        res.edep = _ptr(edep)
        res.cell_edep = _ptr(cell)
        res.escape_E = _ptr(escape)
        res.event_counts = _ptr(event_counts)
        # the buffers must outlive the transport in flight
        self._in_flight = (primaries, edep, cell, escape, event_counts)
        rc = self.lib.gv_transport_events(self.h, _ptr(primaries), n, first_event, n_events, C.c_ulonglong(seed),
                                          _stream_ptr(stream), C.byref(res))
        self.last_result = res
        _check(rc, "gv_transport")
        if sync:
            self.sync(stream)
        return res

    def sync(self, stream=None) -> gv_result:
        """gv_sync: complete the transport in flight; returns its result record."""
        _check(self.lib.gv_sync(self.h, _stream_ptr(stream)), "gv_sync")
        self._in_flight = None
        return self.last_result

    def transport(self, wl: W.Workload | None = None, seed: int | None = None, device: str = "cuda",
                  cells: bool = True, per_event: bool = False, stream=None, first_event: int = 0) -> dict:
        """Convenience: run a workload with device-resident buffers; returns numpy
        arrays.  first_event: global index of the workload's first event (a shard
        of a larger workload, whose primaries carry global event indices)."""
        import torch
        wl = wl or self.wl
        seed = wl.seed if seed is None else seed
        nsub = self.n_subtotal
        dev = torch.device(device)
        prim = torch.from_numpy(wl.primaries.view(np.uint8).copy()).to(dev)
        edep = torch.zeros((wl.n_events, nsub), dtype=torch.float64, device=dev)
        esc = torch.zeros(wl.n_events, dtype=torch.float64, device=dev)
        ncell = wl.n_layers * wl.nx * wl.ny
        cell = torch.zeros(ncell, dtype=torch.float64, device=dev) if (cells and ncell) else None
        evc = torch.zeros((wl.n_events, NCOUNT), dtype=torch.int64, device=dev) if per_event else None
        res = self.gv_transport(prim, wl.n_events, seed, edep, cell, esc, evc, stream, first_event=first_event)
        out = {"edep": edep.cpu().numpy(), "escape": esc.cpu().numpy(),
               "counters": dict(zip(COUNTER_NAMES, list(res.counters))), "status": res.status,
               "launches": self.lib.gv_last_launches(self.h), "kernel_ms": res.kernel_ms}
        if cell is not None:
            out["cell"] = cell.cpu().numpy().reshape(wl.n_layers, wl.nx, wl.ny)
        if evc is not None:
            out["counts"] = evc.cpu().numpy()
        return out

    # ---- element-wise entry points (device tensors in, device tensors out)
    def gv_unit_xs_lookup(self, ptype, mat, E, out, stream=None):
        _check(self.lib.gv_unit_xs_lookup(self.h, ptype, mat, _ptr(E), E.numel(), _ptr(out),
                                          _stream_ptr(stream)), "gv_unit_xs_lookup")

    def gv_unit_eloss(self, ptype, mat, E, s, out, stream=None):
        _check(self.lib.gv_unit_eloss(self.h, ptype, mat, _ptr(E), _ptr(s), E.numel(), _ptr(out),
                                      _stream_ptr(stream)), "gv_unit_eloss")

    def gv_unit_alias_sample(self, model, E, u, out, stream=None):
        _check(self.lib.gv_unit_alias_sample(self.h, model, _ptr(E), _ptr(u), E.numel(), _ptr(out),
                                             _stream_ptr(stream)), "gv_unit_alias_sample")

    def gv_unit_interact(self, ptype, proc, E, d, u, out, ret, stream=None):
        _check(self.lib.gv_unit_interact(self.h, ptype, proc, _ptr(E), _ptr(d), _ptr(u), E.numel(),
                                         _ptr(out), _ptr(ret), _stream_ptr(stream)),
               "gv_unit_interact")

    def gv_unit_distance(self, pos, d, sub, dist, nxt, plane, stream=None):
        _check(self.lib.gv_unit_distance(self.h, _ptr(pos), _ptr(d), _ptr(sub), sub.numel(),
                                         _ptr(dist), _ptr(nxt), _ptr(plane), _stream_ptr(stream)),
               "gv_unit_distance")


    def gv_unit_msc(self, sub, E_pre, E_post, s, d, pos, u, out_dir, out_pos, stream=None):
        _check(self.lib.gv_unit_msc(self.h, _ptr(sub), _ptr(E_pre), _ptr(E_post), _ptr(s), _ptr(d), _ptr(pos),
                                    _ptr(u), sub.numel(), _ptr(out_dir), _ptr(out_pos), _stream_ptr(stream)),
               "gv_unit_msc")


    def gv_unit_field(self, ptype, E, s, d, out, stream=None):
        _check(self.lib.gv_unit_field(self.h, ptype, _ptr(E), _ptr(s), _ptr(d), E.numel(), _ptr(out),
                                      _stream_ptr(stream)), "gv_unit_field")


    def gv_unit_sample(self, model, method, E, seed, out, stream=None):
        _check(self.lib.gv_unit_sample(self.h, model, method, _ptr(E), E.numel(), C.c_ulonglong(seed), _ptr(out),
                                       _stream_ptr(stream)), "gv_unit_sample")


def gv_unit_philox(ctr, key, out, stream=None):
    _check(load().gv_unit_philox(_ptr(ctr), _ptr(key), _ptr(out), ctr.numel() // 4,
                                 _stream_ptr(stream)), "gv_unit_philox")
