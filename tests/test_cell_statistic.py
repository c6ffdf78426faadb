"""The cell-by-cell statistic of the segmented calorimeter, checked on the CPU.

The GPU test compares the GPU's 50 x 32 x 32 cell histogram with the
oracle's through shower_stats.cell_pulls.  Here the oracle is compared with
itself (two independent random streams), which the statistic must accept,
and with copies of itself carrying the mistakes the GPU test is meant to
catch -- x and y swapped, and every cell index shifted by one in x or in y
-- which it must reject by a wide margin.  Smaller showers (5 GeV) and
batches keep it to seconds.
"""
import os

import numpy as np

import shower_stats as S

NTHR = os.cpu_count() or 4
B, M = 32, 16


def _batches(oracle_mod, wl, seed):
    o = oracle_mod.Oracle(wl)
    out = []
    for k in range(B):
        b = S.event_batch(wl, k, M)
        r = o.transport(primaries=b.primaries, n_events=M, n_threads=NTHR, first_event=k * M, seed=seed)
        out.append(r["cell"] / M)
    return np.stack(out)


def test_cell_statistic_accepts_noise_and_rejects_index_mistakes(oracle_mod):
    wl = S.asymmetric_cells_workload(B * M, 5000.0)
    a = _batches(oracle_mod, wl, wl.seed)
    b = _batches(oracle_mod, wl, wl.seed ^ 0x9E3779B9)
    p = S.cell_pulls(a, b)
    assert len(p) > 1000
    assert np.abs(p).max() < 5.5, float(np.abs(p).max())
    assert 0.6 < np.mean(p * p) < 1.5, float(np.mean(p * p))
    for bad in (a.transpose(0, 1, 3, 2), np.roll(a, 1, axis=2), np.roll(a, -1, axis=3)):
        q = S.cell_pulls(bad, b)
        # rejected twice over: the largest pull at least twice the bound, the
        # mean squared pull at least twice its upper limit
        assert np.abs(q).max() > 11.0 and np.mean(q * q) > 3.0, (float(np.abs(q).max()), float(np.mean(q * q)))
