"""gv_transport_static: the transport for callers that cannot let the library
allocate device memory during the call (frameworks that own a GPU's memory
through their own pools).  It must give the same showers as gv_transport --
identical integer histories, deposits equal up to the order of the FP64
atomic sums -- on consecutive calls that reuse its fixed scratch array, and
it must leave the device's free memory and torch's allocator unchanged.

This file is named so that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2005_00949_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__
    __graft_entry__.build()
    from paper_2005_00949_gb300 import gv
    return torch, gv


def _static_call(torch, gv, ctx, wl, seed, repeats=3):
    """gv_transport_static through the C ABI with device buffers, `repeats`
    times in a row (same inputs); returns the last call's results and the
    smallest drop of the device's free memory seen across one call -- other
    processes on a shared GPU can move it during any single call."""
    dev = torch.device("cuda")
    prim = torch.from_numpy(wl.primaries.view(np.uint8).copy()).to(dev)
    edep = torch.full((wl.n_events, ctx.n_subtotal), 7.0, dtype=torch.float64, device=dev)
    esc = torch.full((wl.n_events,), 7.0, dtype=torch.float64, device=dev)
    counters = (C.c_ulonglong * 16)()
    stream = torch.cuda.current_stream().cuda_stream
    used = []
    for _ in range(repeats):
        torch.cuda.synchronize()
        alloc0, res0 = torch.cuda.memory_allocated(), torch.cuda.memory_reserved()
        free0 = torch.cuda.mem_get_info()[0]
        rc = ctx.lib.gv_transport_static(ctx.h, prim.data_ptr(), len(wl.primaries), wl.n_events,
                                         C.c_ulonglong(seed), stream, edep.data_ptr(), esc.data_ptr(), counters)
        torch.cuda.synchronize()
        used.append(free0 - torch.cuda.mem_get_info()[0])
        # nothing went through torch's allocator either
        assert torch.cuda.memory_allocated() == alloc0 and torch.cuda.memory_reserved() == res0
        # gv_sync reports this call's status
        assert ctx.lib.gv_sync(ctx.h, stream) == rc
    return rc, edep.cpu().numpy(), esc.cpu().numpy(), list(counters), min(used)


def _reference(ctx, wl, seed):
    return ctx.transport(wl, seed=seed)


def test_static_transport_matches_allocating_transport_twice(env):
    torch, gv = env
    wl1 = W.pbps_electrons(300, 1000.0)
    # the reference runs the same compiled kernel (no in-block basketizer, one
    # claim per block), so deposits may differ only by the order of the sums
    ctx = gv.Context(wl1, gv.gv_default_config(stack_capacity=1 << 21, process_sort=0,
                                               claim_chunks=0))
    # second call: other primaries, fewer events, another seed -- what the first
    # call left in the scratch array must not leak into it
    wl2 = W.pbps_mixed(120).subset(120)
    wl2.primaries["E"] = np.minimum(wl2.primaries["E"], 3000.0)
    for wl, seed in [(wl1, 12345), (wl2, 777)]:
        # the allocating call first: whatever the driver sets up lazily on a
        # kernel's first launch is then in place before free memory is read
        ref = _reference(ctx, wl, seed)
        rc, edep, esc, cnt, used = _static_call(torch, gv, ctx, wl, seed)
        assert rc == 0, gv.load().gv_strerror(rc)
        names = gv.COUNTER_NAMES
        for i in range(11):  # steps, tracks, pairs, annihilations, escapes
            assert cnt[i] == ref["counters"][names[i]], (names[i], cnt[i], ref["counters"][names[i]])
        scale = np.maximum(ref["edep"].sum(1, keepdims=True), 1.0)
        assert (np.abs(edep - ref["edep"]) / scale).max() < 1e-9
        assert np.abs(esc - ref["escape"]).max() < 1e-9 * max(1.0, ref["escape"].max())
        assert used <= 0  # the call took no device memory


def test_static_transport_rejects_what_it_cannot_hold(env):
    torch, gv = env
    wl = W.pbps_electrons(4, 100.0)
    ctx = gv.Context(wl, gv.gv_default_config(stack_capacity=1 << 16))
    dev = torch.device("cuda")
    prim = torch.from_numpy(wl.primaries.view(np.uint8).copy()).to(dev)
    counters = (C.c_ulonglong * 16)()
    too_many = (1 << 16) + 1
    edep = torch.zeros((too_many, ctx.n_subtotal), dtype=torch.float64, device=dev)
    esc = torch.zeros(too_many, dtype=torch.float64, device=dev)
    s = torch.cuda.current_stream().cuda_stream
    assert ctx.lib.gv_transport_static(ctx.h, prim.data_ptr(), 4, too_many, 1, s, edep.data_ptr(),
                                       esc.data_ptr(), counters) == -1
    host_edep = np.zeros((4, ctx.n_subtotal))
    assert ctx.lib.gv_transport_static(ctx.h, prim.data_ptr(), 4, 4, 1, s, host_edep.ctypes.data,
                                       esc.data_ptr(), counters) == -1
    ctx64 = gv.Context(wl, gv.gv_default_config(precision=gv.GV_FP64, stack_capacity=1 << 16))
    assert ctx64.lib.gv_transport_static(ctx64.h, prim.data_ptr(), 4, 4, 1, s, edep.data_ptr(),
                                         esc.data_ptr(), counters) == -1


def test_static_transport_caps_events_in_flight_for_10GeV(env):
    """64 showers of 10 GeV e- in Pb/polystyrene: the events in flight follow
    the automatic cap (65,536 / (0.15 x 10,000 + 64) = 41 events), so the
    scratch queues hold them; energy is conserved over the batch."""
    torch, gv = env
    wl = W.pbps_electrons(64, 10_000.0)
    ctx = gv.Context(wl, gv.gv_default_config(stack_capacity=1 << 16))
    rc, edep, esc, cnt, used = _static_call(torch, gv, ctx, wl, wl.seed, repeats=1)
    assert rc == 0, gv.load().gv_strerror(rc)
    ME = 0.51099895
    tot = edep.sum() + esc.sum()
    want = 64 * 10_000.0 + 2 * ME * (cnt[8] - cnt[7])
    assert abs(tot - want) < 1e-6 * want
    assert cnt[15] <= 1 << 16  # peak live tracks within one queue's capacity


def test_static_transport_refuses_a_capturing_stream(env):
    """The call waits on the host between its launches, so a stream under
    capture is refused before anything is queued on it."""
    torch, gv = env
    wl = W.pbps_electrons(4, 100.0)
    ctx = gv.Context(wl, gv.gv_default_config(stack_capacity=1 << 16))
    dev = torch.device("cuda")
    prim = torch.from_numpy(wl.primaries.view(np.uint8).copy()).to(dev)
    edep = torch.zeros((4, ctx.n_subtotal), dtype=torch.float64, device=dev)
    esc = torch.zeros(4, dtype=torch.float64, device=dev)
    counters = (C.c_ulonglong * 16)()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s, capture_error_mode="relaxed"):
        rc = ctx.lib.gv_transport_static(ctx.h, prim.data_ptr(), 4, 4, 1, s.cuda_stream, edep.data_ptr(),
                                         esc.data_ptr(), counters)
        edep.add_(1.0)  # the capture records something
    assert rc == -1
    torch.cuda.synchronize()
    rc, _, _, _, _ = _static_call(torch, gv, ctx, wl, 1, repeats=1)
    assert rc == 0
