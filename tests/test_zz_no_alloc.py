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


def test_static_transport_takes_turns_with_other_transports(env):
    """The step kernels read the transport's state from one constant-memory
    record per GPU, which every transport takes in turn: a static call on
    one context and gv_transport on another, driven from two host threads
    on two streams at once, give the results each gives alone."""
    import threading
    torch, gv = env
    wl_a = W.pbps_electrons(200, 2000.0)
    wl_b = W.with_msc(W.pblar_testem3(100, 3000.0))
    ctx_a = gv.Context(wl_a, gv.gv_default_config(stack_capacity=1 << 20, process_sort=0, claim_chunks=0))
    ctx_b = gv.Context(wl_b, gv.gv_default_config(stack_capacity=1 << 20, per_event_counts=1))
    dev = torch.device("cuda")
    prim = torch.from_numpy(wl_a.primaries.view(np.uint8).copy()).to(dev)
    s_a = torch.cuda.Stream()

    def static_run():
        edep = torch.zeros((wl_a.n_events, ctx_a.n_subtotal), dtype=torch.float64, device=dev)
        esc = torch.zeros(wl_a.n_events, dtype=torch.float64, device=dev)
        counters = (C.c_ulonglong * 16)()
        torch.cuda.synchronize()
        rc = ctx_a.lib.gv_transport_static(ctx_a.h, prim.data_ptr(), len(wl_a.primaries), wl_a.n_events,
                                           C.c_ulonglong(wl_a.seed), s_a.cuda_stream, edep.data_ptr(),
                                           esc.data_ptr(), counters)
        s_a.synchronize()
        return rc, edep.cpu().numpy(), list(counters)

    alone_a = static_run()
    alone_b = ctx_b.transport(per_event=True)
    both = [None, None]

    def run_a():
        both[0] = static_run()

    def run_b():
        both[1] = ctx_b.transport(per_event=True)

    th = [threading.Thread(target=run_a), threading.Thread(target=run_b)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert alone_a[0] == 0 and both[0][0] == 0
    assert both[0][2][:11] == alone_a[2][:11]
    assert np.allclose(both[0][1], alone_a[1], rtol=1e-9, atol=1e-9)
    assert both[1]["status"] == 0
    assert np.array_equal(both[1]["counts"][:, :11], alone_b["counts"][:, :11])
    assert np.allclose(both[1]["edep"], alone_b["edep"], rtol=1e-9, atol=1e-9)
