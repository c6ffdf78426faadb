"""Per-layer shower statistics and the statistical parity criteria.

A sample of showers is summarised by its size and the mean and variance
(ddof=1) of the per-event deposit of every layer and of every material
(summed over layers), so that a large reference sample can be stored as text
and compared with a fresh one later.  The criteria are those of the
statistical parity of whole showers: every layer within 3 combined standard
errors; within 0.5 % on the layers that hold at least 1 % of the deposit
wherever 0.5 % is at least 3 combined standard errors (the 0.5 % bound is
"active" there); every material total within 3 combined standard errors, and
within 0.5 % where that bound is active.
"""
from __future__ import annotations

import os

import numpy as np

from paper_2005_00949_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def summarize(edep: np.ndarray, n_layers: int) -> dict:
    """edep: [n_events, n_layers * n_sub] per-event deposits."""
    n = edep.shape[0]
    e = edep.reshape(n, n_layers, -1)
    lay = e.sum(2)
    mat = e.sum(1)
    return {"n": n, "layer_mean": lay.mean(0), "layer_var": lay.var(0, ddof=1),
            "mat_mean": mat.mean(0), "mat_var": mat.var(0, ddof=1)}


def compare(a: dict, b: dict, frac: float = 0.01, rel: float = 0.005, pull_max: float = 3.0) -> dict:
    """Apply the criteria to two summaries; raise AssertionError on failure.
    Returns the worst layer pull, the worst relative difference on the layers
    where 0.5 % is active, and how many layers and materials it was active on."""
    comb = np.sqrt(a["layer_var"] / a["n"] + b["layer_var"] / b["n"])
    d = np.abs(a["layer_mean"] - b["layer_mean"])
    live = comb > 0
    pull = np.zeros_like(d)
    pull[live] = d[live] / comb[live]
    ref = b["layer_mean"]
    assert pull.max() <= pull_max, ("layer pull", float(pull.max()), int(np.argmax(pull)))
    big = (ref >= frac * ref.sum()) & (3 * comb <= rel * ref)
    reld = np.zeros_like(d)
    reld[big] = d[big] / ref[big]
    assert (reld <= rel).all(), ("layer rel", float(reld.max()), int(np.argmax(reld)))
    cm = np.sqrt(a["mat_var"] / a["n"] + b["mat_var"] / b["n"])
    dm = np.abs(a["mat_mean"] - b["mat_mean"])
    assert (dm <= pull_max * cm + 1e-12).all(), ("material pull", (dm / np.maximum(cm, 1e-300)).tolist())
    mbig = 3 * cm <= rel * b["mat_mean"]
    assert (dm[mbig] <= rel * b["mat_mean"][mbig]).all(), ("material rel", (dm / b["mat_mean"]).tolist())
    return {"pull": float(pull.max()), "rel": float(reld.max()), "active_layers": int(big.sum()),
            "active_materials": int(mbig.sum()),
            "mat_rel": (dm / b["mat_mean"]).tolist()}


def write(path: str, s: dict, header: list[str]):
    with open(path, "w") as f:
        for h in header:
            f.write(f"# {h}\n")
        f.write(f"n {s['n']}\n")
        for i, (m, v) in enumerate(zip(s["layer_mean"], s["layer_var"])):
            f.write(f"layer {i} {float(m)!r} {float(v)!r}\n")
        for i, (m, v) in enumerate(zip(s["mat_mean"], s["mat_var"])):
            f.write(f"material {i} {float(m)!r} {float(v)!r}\n")


def read(name: str) -> dict:
    lm, lv, mm, mv, n = [], [], [], [], None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            c = line.split()
            if not c or c[0].startswith("#"):
                continue
            if c[0] == "n":
                n = int(c[1])
            elif c[0] == "layer":
                lm.append(float(c[2]))
                lv.append(float(c[3]))
            elif c[0] == "material":
                mm.append(float(c[2]))
                mv.append(float(c[3]))
    return {"n": n, "layer_mean": np.array(lm), "layer_var": np.array(lv),
            "mat_mean": np.array(mm), "mat_var": np.array(mv)}


def cell_pulls(a: np.ndarray, b: np.ndarray, frac: float = 0.005) -> np.ndarray:
    """Pulls between two cell histograms given as batch means [B, L, NX, NY]
    (each batch: a sum over its events divided by their number): every
    (layer, ix) and (layer, iy) projection, and every cell holding >= frac of
    its layer's deposit (on side b).  The standard error of a bin is the
    spread of its batch means over sqrt(B)."""
    def stats(x):
        return x.mean(0), x.std(0, ddof=1) / np.sqrt(x.shape[0])

    out = []
    for proj in ((3,), (2,), ()):
        ap = a.sum(proj) if proj else a
        bp = b.sum(proj) if proj else b
        am, as_ = stats(ap)
        bm, bs = stats(bp)
        comb = np.sqrt(as_ ** 2 + bs ** 2)
        sel = comb > 0
        if not proj:
            sel &= bm >= frac * bm.sum((1, 2), keepdims=True)
        out.append(((am - bm)[sel] / comb[sel]).ravel())
    return np.concatenate(out)


def asymmetric_cells_workload(n_events: int, energy: float, seed: int = 20261203) -> W.Workload:
    """The segmented W/Si calorimeter (50 layers, 32 x 32 cells of 1.25 cm)
    hit by e- whose entry points cover 4 cells in x (ix 11-14) and 2 in y
    (iy 17-18), tilted by 0.05 rad in x: a beam without the x/y symmetry, so
    that a swapped or shifted cell index shows in the histogram."""
    wl = W.wsi_cells(n_events, energy)
    rng = np.random.default_rng(seed)
    p = wl.primaries
    p["x"] = rng.uniform(-6.25, -1.25, n_events)
    p["y"] = rng.uniform(1.25, 3.75, n_events)
    p["u"] = 0.05
    p["v"] = 0.0
    p["w"] = np.sqrt(1.0 - 0.05 ** 2)
    return wl


def event_batch(wl: W.Workload, k: int, m: int) -> W.Workload:
    """Events k*m .. (k+1)*m - 1 of wl (global event indices kept)."""
    ev = wl.primaries["event"]
    p = wl.primaries[(ev >= k * m) & (ev < (k + 1) * m)].copy()
    e = dict(wl.__dict__)
    e.update(primaries=p, n_events=m, name=f"{wl.name}#{k}")
    return W.Workload(**e)
