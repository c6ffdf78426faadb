"""Multi-rank event sharding on CPU (gloo, world size 2): each rank transports
its event range (tally rows for its own events only, random streams keyed by
the global event index) with the FP64 oracle, the tallies are gathered, and the
result equals the single-process transport exactly (per-event random streams)."""
import os
import socket

import numpy as np
import pytest

from paper_2005_00949_gb300 import sharding, workloads as W


def test_shard_ranges_partition_the_events():
    for n in [0, 1, 7, 100, 2001]:
        for world in [1, 2, 3, 8]:
            r = [sharding.shard_range(n, k, world) for k in range(world)]
            assert r[0][0] == 0 and r[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
            sizes = [hi - lo for lo, hi in r]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        sharding.shard_range(10, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl = W.wsi_cells(9, 2000.0)
        shard, lo, hi = sharding.shard_workload(wl, rank, world)
        res = oracle.Oracle(shard).transport(n_threads=2, first_event=lo)
        assert res["edep"].shape[0] == hi - lo  # rows of this rank's events only
        full = sharding.gather_tallies(dist, res, lo, hi)
        if rank == 0:
            q.put({k: v for k, v in full.items()})
    finally:
        dist.destroy_process_group()


def test_sharded_transport_equals_single_process(oracle_mod):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    full = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    wl = W.wsi_cells(9, 2000.0)
    ref = oracle_mod.Oracle(wl).transport(n_threads=2)
    assert np.array_equal(full["edep"], ref["edep"])
    assert np.array_equal(full["escape"], ref["escape"])
    assert np.array_equal(full["counts"], ref["counts"])
    assert np.allclose(full["cell"], ref["cell"], rtol=1e-12, atol=1e-12)


def _failing_rank_main(rank, world, port, q):
    """Rank 1 fails between steps (before the gather, nothing in flight);
    rank 0 must learn of it from its collective instead of waiting forever."""
    import datetime

    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=20))
    if rank == 1:
        os._exit(3)  # the rank dies without joining the gather
    local = {"edep": np.zeros((2, 2)), "escape": np.zeros(2)}
    try:
        sharding.gather_tallies(dist, local, 0, 2)
        q.put("gathered")
    except Exception as e:  # noqa: BLE001 -- any collective error is the detection
        q.put(f"detected: {type(e).__name__}")


def test_a_failed_rank_is_detected_by_the_gather():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_failing_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    msg = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
    assert msg.startswith("detected"), msg
    assert procs[1].exitcode == 3


def test_event_offset_rows_equal_the_full_transport(oracle_mod):
    """A range transported with first_event = lo gives, in rows 0 .. hi-lo-1,
    exactly rows lo .. hi-1 of the whole workload's transport."""
    wl = W.pbps_mixed(30).subset(30)
    wl.primaries["E"] = np.minimum(wl.primaries["E"], 2000.0)
    ref = oracle_mod.Oracle(wl).transport(n_threads=2)
    for rank, world in ((0, 3), (1, 3), (2, 3)):
        shard, lo, hi = sharding.shard_workload(wl, rank, world)
        r = oracle_mod.Oracle(shard).transport(n_threads=2, first_event=lo)
        assert np.array_equal(r["edep"], ref["edep"][lo:hi])
        assert np.array_equal(r["counts"], ref["counts"][lo:hi])
        assert np.array_equal(r["escape"], ref["escape"][lo:hi])
