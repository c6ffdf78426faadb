"""Cell-by-cell parity of the segmented calorimeter's deposit histogram.

The 50 x 32 x 32 cell histogram (W/Si layers, 1.25 cm cells, 100 GeV e-)
of the mixed GPU transport is compared with the FP64 oracle's, bin by bin.
The histogram is a sum over events, so each side transports the events in
32 batches (event ranges, first_event = the range's start) and the spread of
the batch means gives every bin's standard error.  The beam is deliberately
asymmetric -- entry points over 4 cells in x and 2 in y, tilted in x -- so
that swapping x and y, or moving a cell edge by one cell, changes the
projections by many standard errors.  Compared: every (layer, ix) and
(layer, iy) projection and every cell holding >= 0.5 % of its layer's
deposit; the largest pull is bounded for ~5000 comparisons at once (5.5
standard errors, Student t with ~60 degrees of freedom) and the mean squared
pull must be that of noise.
"""
import os

import numpy as np
import pytest

from paper_2005_00949_gb300 import workloads as W

import shower_stats as S

pytestmark = pytest.mark.gpu
NTHR = os.cpu_count() or 4
B = 32        # batches
M = 200       # events per batch


@pytest.fixture(scope="module")
def gvmod():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__
    __graft_entry__.build()
    from paper_2005_00949_gb300 import gv
    return gv


def _stats(x):
    """per-bin mean of the batch means and its standard error"""
    x = np.asarray(x)
    return x.mean(0), x.std(0, ddof=1) / np.sqrt(x.shape[0])


def test_cell_histogram_matches_oracle_bin_by_bin(gvmod, oracle_mod):
    wl = S.asymmetric_cells_workload(B * M, 100_000.0)
    ctx = gvmod.Context(wl, gvmod.gv_default_config(stack_capacity=1 << 23))
    o = oracle_mod.Oracle(wl)
    g_cells, o_cells = [], []
    for k in range(B):
        b = S.event_batch(wl, k, M)
        r = ctx.transport(b, first_event=k * M)
        assert r["status"] == 0
        g_cells.append(r["cell"] / M)
        # the oracle draws other random numbers (another seed): the two
        # samples are independent, as the standard errors assume
        ro = o.transport(primaries=b.primaries, n_events=M, n_threads=NTHR, first_event=k * M,
                         seed=wl.seed ^ 0x9E3779B9)
        o_cells.append(ro["cell"] / M)
        # the histogram sums to the per-layer tallies on both sides
        assert np.allclose(r["cell"].sum((1, 2)), r["edep"].reshape(M, 50, 2).sum((0, 2)), rtol=1e-9)
        assert np.allclose(ro["cell"].sum((1, 2)), ro["edep"].reshape(M, 50, 2).sum((0, 2)), rtol=1e-9)
    ctx.close()
    g = np.stack(g_cells)  # [B, 50, 32, 32]
    oc = np.stack(o_cells)
    p = S.cell_pulls(g, oc)
    assert len(p) > 3000
    assert np.abs(p).max() < 5.5, float(np.abs(p).max())
    assert 0.6 < np.mean(p * p) < 1.5, float(np.mean(p * p))
    # the beam's cells carry the deposit: around the shower maximum (layers
    # holding >= 2 % of it) the comparison resolves 1 % of their sum
    gm, gs = _stats(g[:, :, 11:15, 17:19].sum((2, 3)))
    om, os_ = _stats(oc[:, :, 11:15, 17:19].sum((2, 3)))
    big = om > 0.02 * om.sum()
    assert big.sum() >= 10
    res = np.sqrt(gs ** 2 + os_ ** 2)[big] / om[big]
    assert (res < 0.01).all(), res.max()
