"""Autotuner of the transport's launch shape and basket thresholds.

Coordinate descent over the knobs of gv_config on a sample of the target
workload, timing each candidate with gv_transport's own CUDA-event kernel
time (median of repeats).  Knobs:
  block_size, blocks_per_sm      -- launch shape of the persistent step kernel
  steps_per_claim                -- steps a thread takes on a claimed track
  tail_steps_per_claim, tail_threshold
                                 -- the same when the live population is small
  refill_low_water, refill_batch -- event-server refill thresholds (live-track
                                    budget below which primaries are injected)
  process_sort                   -- in-block re-basketing by selected process
  claim_chunks                   -- per-block or per-warp work claims
  along_steps, along_steps_photon
                                 -- steps a lane takes (charged track, photon)
                                    before its block baskets
  scoring                        -- direct or warp-merged tally atomics
Integer results do not depend on any of these (per-track random streams), so
the tuner only trades time.
"""
from __future__ import annotations

import json
import os
import time

from . import gv, workloads as W

SPACE = {
    "process_sort": [1, 0],
    "claim_chunks": [0, 1],
    "along_steps": [2, 3, 4, 6],
    "along_steps_photon": [3, 4, 5, 6],
    "scoring": [0, 1],
    "local_stack": [1, 0],
    "pdl": [1, 0],
    "block_size": [128, 256],
    "blocks_per_sm": [2, 3, 4],
    "steps_per_claim": [1, 2, 3, 4],
    "tail_steps_per_claim": [1, 2, 4, 8, 16],
    "tail_threshold": [1 << 15, 1 << 17, 1 << 19],
    "refill_low_water": [1 << 19, 1 << 21, 1 << 23],
    "refill_batch": [1 << 8, 1 << 11, 1 << 14],
}


def _measure(wl: W.Workload, cfg: gv.gv_config, repeats: int) -> float:
    ctx = gv.Context(wl, cfg)
    try:
        ctx.transport(wl)  # warm-up (graph capture, first-touch)
        ts = []
        for _ in range(repeats):
            r = ctx.transport(wl)
            ts.append(r["kernel_ms"])
        ts.sort()
        return ts[len(ts) // 2]
    finally:
        ctx.close()


def tune(wl: W.Workload, base: gv.gv_config | None = None, passes: int = 2, repeats: int = 3,
         space: dict | None = None, budget_s: float = 120.0, log=None) -> tuple[dict, float]:
    """Return (best knob values, best median kernel ms) for workload `wl`."""
    space = space or SPACE
    cfg = base or gv.gv_default_config(stack_capacity=1 << 23)
    best = {k: getattr(cfg, k) for k in space}
    t0 = time.time()

    def cfg_of(knobs):
        c = gv.gv_default_config()
        for f, _ in gv.gv_config._fields_:
            setattr(c, f, getattr(cfg, f))
        for k, v in knobs.items():
            setattr(c, k, v)
        return c

    best_ms = _measure(wl, cfg_of(best), repeats)
    for _ in range(passes):
        improved = False
        for k, values in space.items():
            for v in values:
                if v == best[k] or time.time() - t0 > budget_s:
                    continue
                trial = dict(best, **{k: v})
                try:
                    ms = _measure(wl, cfg_of(trial), repeats)
                except gv.GvError:
                    continue
                if log:
                    log(f"{k}={v}: {ms:.3f} ms (best {best_ms:.3f})")
                if ms < best_ms * 0.98:
                    best, best_ms, improved = trial, ms, True
        if not improved:
            break
    return best, best_ms


def apply(cfg: gv.gv_config, knobs: dict) -> gv.gv_config:
    for k, v in knobs.items():
        setattr(cfg, k, v)
    return cfg


TUNED_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned.json")


def load_or_tune(wl: W.Workload, path: str = TUNED_PATH, sample_events: int = 400, **kw) -> dict:
    """Tuned knobs for `wl`, cached in `path` (JSON keyed by workload name and GPU)."""
    import torch
    key = f"{wl.name}|{torch.cuda.get_device_name()}"
    db = {}
    if os.path.exists(path):
        with open(path) as f:
            db = json.load(f)
    if key in db:
        return db[key]["knobs"]
    knobs, ms = tune(wl.subset(min(sample_events, wl.n_events)), **kw)
    db[key] = {"knobs": knobs, "sample_kernel_ms": ms, "sample_events": sample_events}
    with open(path, "w") as f:
        json.dump(db, f, indent=1)
    return knobs


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(description="tune the transport launch shape for a workload")
    ap.add_argument("--workload", default=W.PBPS_10GEV, choices=sorted(W.STANDARD),
                    help="standard workload (workloads.STANDARD)")
    ap.add_argument("--sample-events", type=int, default=400)
    ap.add_argument("--budget-s", type=float, default=120.0)
    ap.add_argument("--path", default=TUNED_PATH)
    ap.add_argument("--force", action="store_true")
    a = ap.parse_args(argv)
    wl = W.standard(a.workload)
    if a.force and os.path.exists(a.path):
        with open(a.path) as f:
            db = json.load(f)
        import torch
        db.pop(f"{wl.name}|{torch.cuda.get_device_name()}", None)
        with open(a.path, "w") as f:
            json.dump(db, f, indent=1)
    knobs = load_or_tune(wl, a.path, a.sample_events, budget_s=a.budget_s, log=print)
    print(json.dumps({"workload": wl.name, "knobs": knobs}))


if __name__ == "__main__":
    main()
