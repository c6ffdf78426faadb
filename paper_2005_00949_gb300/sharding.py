"""Event sharding across GPUs (one process per GPU).

Events are independent and every random number is keyed by the event index
and the track's lineage, so an event's result does not depend on which rank
transports it or what else runs beside it.  A workload therefore splits into
contiguous event ranges, one per rank, with no exchange on the data path; each
rank transports its range with first_event = lo (tally rows for its own events
only), and the only collective is the final gather of per-event tallies (and a
sum of the cell histogram), done on the host.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import workloads as W


def shard_range(n_events: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous event range [lo, hi) of `rank` out of `world` (balanced)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(n_events, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def shard_workload(wl: W.Workload, rank: int, world: int) -> tuple[W.Workload, int, int]:
    """The primaries of this rank's events [lo, hi), as a workload of hi - lo
    events.  Event indices stay global (they key the random streams): pass
    first_event=lo to the transport, whose tally row i then holds event
    lo + i, so a rank allocates tallies for its own events only."""
    lo, hi = shard_range(wl.n_events, rank, world)
    ev = wl.primaries["event"]
    p = wl.primaries[(ev >= lo) & (ev < hi)].copy()
    return dataclasses.replace(wl, primaries=p, n_events=hi - lo, name=f"{wl.name}#{rank}/{world}"), lo, hi


def gather_event_rows(rows: list[np.ndarray]) -> np.ndarray:
    """Concatenate the per-rank event rows (ranks in order)."""
    return np.concatenate(rows, axis=0)


def gather_tallies(dist, local: dict, lo: int, hi: int) -> dict | None:
    """Gather per-event tallies (this rank's rows, events lo .. hi-1) and sum
    the cell histogram over ranks with a torch.distributed process group (any
    backend); returns the full tallies on rank 0 and None elsewhere."""
    assert len(local["edep"]) == hi - lo
    mine = {"edep": local["edep"], "escape": local["escape"]}
    if "counts" in local:
        mine["counts"] = local["counts"]
    if "cell" in local:
        mine["cell"] = local["cell"]
    world = dist.get_world_size()
    out = [None] * world
    dist.all_gather_object(out, mine)
    if dist.get_rank() != 0:
        return None
    full = {k: gather_event_rows([o[k] for o in out]) for k in mine if k != "cell"}
    if "cell" in mine:
        full["cell"] = np.sum([o["cell"] for o in out], axis=0)
    return full
