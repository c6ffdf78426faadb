"""Benchmark: 10 GeV e- showers/s (and EM steps/s) on the 50-layer Pb/polystyrene
calorimeter, 2000 events per step, through the libgv C ABI.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

One step = one gv_transport call over the whole batch (every stage of the
stepping loop for every track of every event).  `value` times it with inputs
and tallies resident in HBM; `e2e` times the same call with host buffers
(host->device primaries and device->host tallies inside the timed region).
Between timed steps L2 is flushed by writing a 512 MiB buffer.  Under torchrun
each rank transports its own 2000-event shard (weak scaling, no collective on
the data path); rank 0 prints one JSON line.

--impl reference times the FP64 CPU oracle (the reference arm of this benchmark)
on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import datetime
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2005_00949_gb300 import workloads as W  # noqa: E402

METRIC = "EM steps/s and 10 GeV e- showers/s on 1 GB300; HBM roofline fraction"
WORKLOAD = ("e-10GeV_PbPS50_2000: 2000 x 10 GeV e- on 50 x (2 mm Pb + 5 mm polystyrene), "
            "40x40 cm, cuts 1 MeV")


def _config(world: int) -> dict:
    """The workload as both arms name it (identical for the GPU and the
    reference arm at one GPU)."""
    return {"workload": WORKLOAD, "events_per_gpu": 2000, "parallelism": f"events x{world}",
            "l2": "GPU arm: flushed between timed steps (512 MiB write); reference arm (host CPU): not applicable"}
N_EVENTS = 2000
E0 = 10_000.0
# algorithmic DRAM bytes of one track step of the mixed form in a
# step-synchronous wavefront: read + write a ~68 B track record (136 B),
# ~0.2 secondaries of 68 B (14 B), a basket index read and written (8 B)
SCOPE_BYTES_PER_STEP = 158.0
# the same count with this library's 64-byte track record and the measured
# secondaries per step
TRACK_BYTES = 64


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


KERNEL_SOURCES = ["gv_transport.cu", "gv_device.cuh", "gv_state.cuh", "gv_internal.h"]


def kernel_source_hash() -> str:
    """sha1 over the step kernel's sources: a DRAM-traffic figure taken with
    ncu holds only while it matches."""
    h = hashlib.sha1()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2005_00949_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def _traffic_per_launch():
    """dram__bytes_read.sum + dram__bytes_write.sum per step-kernel launch of
    this workload, from the ncu capture summarised in profiles/ (None if the
    kernel sources changed since)."""
    try:
        with open(os.path.join(ROOT, "profiles", "step_kernel_dram_traffic.json")) as f:
            t = json.load(f)
        if t.get("kernel_source_sha1") != kernel_source_hash():
            return None
        return float(t["dram_bytes_per_launch"])
    except (OSError, ValueError, KeyError):
        return None


def _workload(rank: int = 0, world: int = 1):
    """This rank's shard of the job: the job is world x 2000 showers (weak
    scaling), split by event range; the shard keeps global event indices
    (its random streams) and is transported with first_event = lo."""
    from paper_2005_00949_gb300 import sharding
    return sharding.shard_workload(W.pbps_electrons(N_EVENTS * world, E0), rank, world)


def _l2_profile():
    """L2 throughput (% of peak) and hit rate of the step kernel from the ncu
    capture summarised in profiles/ (None if the kernel sources changed since):
    the live track set stays in L2, so L2 rather than HBM carries its traffic."""
    try:
        with open(os.path.join(ROOT, "profiles", "step_kernel_l2.json")) as f:
            t = json.load(f)
        if t.get("kernel_source_sha1") != kernel_source_hash():
            return None
        return {k: t[k] for k in ("l2_throughput_pct", "l2_hit_rate_pct", "dram_throughput_pct", "workload")}
    except (OSError, ValueError, KeyError):
        return None


class Clocks:
    """nvidia-smi sampling (every 100 ms) around the timed region; the summary
    keeps the samples taken between mark_start() and mark_end()."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.p = None
        self.t0 = self.t1 = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    def __exit__(self, *a):
        self.rows = []
        if self.p is None:
            return
        time.sleep(0.25)
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 10:
                try:  # local wall-clock time of the sample
                    f[0] = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                except ValueError:
                    f[0] = None
                self.rows.append(f)

    def summary(self):
        rows = getattr(self, "rows", None) or []
        if rows and self.t0 is not None and self.t1 is not None:
            inside = [r for r in rows if r[0] is not None and self.t0 - 0.05 <= r[0] <= self.t1 + 0.05]
            if inside:
                rows = inside
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def cpu_baseline(wl, budget_events: int | None = None, repeats: int = 3):
    """The FP64 oracle, as it stands, on the host cores over a bounded sample
    (by default the whole workload, best of `repeats`)."""
    import oracle
    nthr = os.cpu_count() or 1
    n = budget_events or wl.n_events
    sub = wl.subset(min(n, wl.n_events))
    o = oracle.Oracle(sub)
    best, steps = None, 0
    for _ in range(repeats):
        t = time.perf_counter()
        r = o.transport(n_threads=nthr)
        dt = time.perf_counter() - t
        steps = int(r["counts"][:, 0].sum())
        best = dt if best is None else min(best, dt)
    return {"value": sub.n_events / best, "unit": "showers/s", "cores": nthr, "kind": "oracle",
            "sample": f"{sub.n_events} x 10 GeV e- ({steps} track steps) of the 2000-event workload, "
                      f"{nthr} threads, best of {repeats}: {best:.2f} s wall",
            "steps_per_s": steps / best}


def comparators(gv, wl, n_one_event):
    """The same workload through the other forms of the library on this GPU:
    FP64 everywhere (batched), and the plain one-event-per-launch schedule
    (FP64 and mixed) on the first `n_one_event` events."""
    out = {}
    forms = [("fp64_batched", dict(precision=gv.GV_FP64), wl),
             ("fp64_one_event_per_launch", dict(precision=gv.GV_FP64, mode=gv.GV_ONE_EVENT_PER_LAUNCH),
              wl.subset(n_one_event)),
             ("mixed_one_event_per_launch", dict(mode=gv.GV_ONE_EVENT_PER_LAUNCH), wl.subset(n_one_event))]
    for name, kw, w in forms:
        ctx = gv.Context(w, gv.gv_default_config(stack_capacity=1 << 22, **kw))
        if kw.get("mode") != gv.GV_ONE_EVENT_PER_LAUNCH:
            ctx.transport(w)  # warm-up (graph capture); the one-event forms are seconds long already
        r = ctx.transport(w)
        ms = r["kernel_ms"]
        out[name] = {"events": w.n_events, "ms": ms, "events_per_s": w.n_events / (ms / 1e3),
                     "steps_per_s": r["counters"]["steps"] / (ms / 1e3),
                     "timing": "CUDA events around the step-kernel graphs (library work stream)"}
        ctx.close()
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    wl, _, _ = _workload(0)
    nthr = os.cpu_count() or 1
    n_ev = N_EVENTS
    for _ in range(args.warmup):
        cpu_baseline(wl, nthr, repeats=1)
    times, vals = [], []
    for _ in range(args.steps):
        b = cpu_baseline(wl, n_ev, repeats=1)
        vals.append(b["value"])
        times.append(n_ev / b["value"])
    v = n_ev * len(times) / sum(times)
    line = {"metric": METRIC, "value": v, "unit": "showers/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * sum(times) / len(times) * (N_EVENTS / n_ev),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": _config(1),
            "reference": {"program": "the FP64 oracle (tabulated transport), host threads",
                          "sample_events_per_step": n_ev},
            "cpu_baseline": {"value": v, "unit": "showers/s", "cores": nthr, "kind": "oracle",
                             "sample": f"{n_ev} events per step of the 2000-event workload"},
            "e2e": {"value": v, "unit": "showers/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gv")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--events", type=int, default=N_EVENTS,
                    help="events per step (profiling of small cases only)")
    ap.add_argument("--capacity", type=int, default=1 << 23, help="track queue capacity per type")
    ap.add_argument("--no-comparators", action="store_true")
    ap.add_argument("--host-loop", action="store_true",
                    help="relaunch the generation graph from the host (device_loop=0): the same kernels, "
                         "in graphs that ncu can profile kernel by kernel")
    ap.add_argument("--comparator-events", type=int, default=N_EVENTS,
                    help="events of the one-event-per-launch comparators (default: the whole workload)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2005_00949_gb300 import gv

    wl, lo, hi = _workload(rank, world)
    if args.events != N_EVENTS:
        wl = wl.subset(args.events) if world == 1 else wl
    ctx = gv.Context(wl, gv.gv_default_config(stack_capacity=args.capacity,
                                              device_loop=0 if args.host_loop else 1))
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    prim_d = torch.from_numpy(wl.primaries.view(np.uint8).copy()).to(dev)
    nsub = ctx.n_subtotal
    edep = torch.zeros((wl.n_events, nsub), dtype=torch.float64, device=dev)
    esc = torch.zeros(wl.n_events, dtype=torch.float64, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def step():  # gv_transport_events + gv_sync
        return ctx.gv_transport(prim_d, wl.n_events, wl.seed, edep, None, esc, None, stream, first_event=lo)

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # ---- device-resident timing
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    steps_tot, kernel_ms, launches, sec = 0, 0.0, 0, 0
    barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        time.sleep(0.3)  # let the sampler start
        clk.mark_start()
        for i in range(args.steps):
            flush.fill_(i & 0xff)
            starts[i].record(stream)
            res = step()
            ends[i].record(stream)
            steps_tot += res.counters[0]
            sec += res.counters[4] + res.counters[5] + res.counters[6] - wl.n_events
            kernel_ms += res.kernel_ms
            launches += ctx.lib.gv_last_launches(ctx.h)
        torch.cuda.synchronize()
        clk.mark_end()
    barrier()
    ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    if dist is not None:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    ms_per_step = ms / args.steps
    events_all = wl.n_events * world
    value = events_all / (ms_per_step / 1000.0)
    steps_per_s = steps_tot * world / (ms / 1000.0)
    # ---- end to end through the C ABI with host buffers
    prim_h = torch.from_numpy(wl.primaries.view(np.uint8).copy()).pin_memory()
    edep_h = torch.zeros((wl.n_events, nsub), dtype=torch.float64).pin_memory()
    esc_h = torch.zeros(wl.n_events, dtype=torch.float64).pin_memory()
    e_ms = 0.0
    n_e2e = max(1, min(args.steps, 5))
    barrier()
    torch.cuda.synchronize()
    for i in range(n_e2e):
        flush.fill_(i & 0xff)
        torch.cuda.synchronize()
        t = time.perf_counter()
        ctx.gv_transport(prim_h, wl.n_events, wl.seed, edep_h, None, esc_h, None, stream, first_event=lo)
        torch.cuda.synchronize()
        e_ms += (time.perf_counter() - t) * 1000.0
    if dist is not None:
        t = torch.tensor([e_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e_ms = float(t.item())
    e2e = events_all / (e_ms / n_e2e / 1000.0)
    gathered = None
    if dist is not None:  # the one collective of the job: the tallies of every shard to rank 0
        from paper_2005_00949_gb300 import sharding
        gathered = sharding.gather_tallies(dist, {"edep": edep_h.numpy(), "escape": esc_h.numpy()}, lo, hi)
    if rank != 0:
        dist.destroy_process_group()
        return 0
    # ---- roofline of the step kernel
    peak, peak_kind = _peaks()
    sec_per_step = sec / max(steps_tot, 1)
    rec_bytes_per_step = 2 * TRACK_BYTES + TRACK_BYTES * sec_per_step
    alg_bytes = steps_tot * SCOPE_BYTES_PER_STEP  # this rank's steps, this rank's kernel time
    achieved = alg_bytes / (kernel_ms / 1000.0) / 1e9 if kernel_ms > 0 else None
    achieved_rec = steps_tot * rec_bytes_per_step / (kernel_ms / 1000.0) / 1e9 if kernel_ms > 0 else None
    traffic = _traffic_per_launch() if args.events == N_EVENTS else None
    l2 = _l2_profile()
    c = list(res.counters)
    working_launches = max(c[11], 1)  # generations of the last transport
    line = {
        "metric": METRIC, "value": value, "unit": "showers/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic",
        "config": _config(world),
        "precision": "mixed FP32 physics / FP64 positions and tallies",
        "steps_per_s": steps_per_s,
        "track_steps_per_step": steps_tot / args.steps / 1.0,
        "kernel_ms_per_step": kernel_ms / args.steps,
        "gpu_launches": int(launches),
        "e2e": {"value": e2e, "unit": "showers/s",
                "h2d_bytes_per_step": int(wl.primaries.nbytes),
                "d2h_bytes_per_step": int(edep_h.numel() * 8 + esc_h.numel() * 8)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "peak_source": f"{peak_kind} hbm_gbs",
                     "kernel": "gv::step_kernel<float>",
                     "alg_bytes_per_step": SCOPE_BYTES_PER_STEP,
                     "alg_bytes_per_launch": alg_bytes / args.steps / working_launches,
                     "alg_bytes_per_step_this_record": rec_bytes_per_step,
                     "frac_this_record": (achieved_rec / peak) if achieved_rec else None,
                     "traffic_unit": "DRAM bytes per working launch (ncu, full-size workload)",
                     "l2": l2},
        "clocks": clk.summary(),
    }
    line["diagnostics"] = {
        "generations": c[11], "live_peak": c[15],
        "geometry_limited_frac": c[12] / max(c[0], 1), "discrete_frac": c[13] / max(c[0], 1),
        "idle_lane_frac": 1.0 - c[0] / max(c[14], 1)}
    if not args.no_comparators:
        line["comparators"] = comparators(gv, wl, args.comparator_events)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl)
    print(json.dumps(line))
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
