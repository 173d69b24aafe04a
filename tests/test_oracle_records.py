"""Pins of the oracle's measurement records (Appendix A): the PT walk
history (history_betas, the ladder slot of every system copy at every
measurement) and the block sums of maxit consecutive energy measurements.

The oracle records them inside its run loop; here the same chain is stepped
one measurement interval at a time and the records are rebuilt from what the
state shows after each step (the inverse of the permutation, the energies by
slot), so a record of the wrong quantity, slot, block or measurement fails.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("measure_every,maxit,n_meas", [(2, 3, 10), (1, 1, 7), (3, 4, 9)])
def test_records_equal_step_by_step_observation(measure_every, maxit, n_meas):
    k, kt = oracle.ladder_linear(0.2, 0.6, 6, 1.0)
    rec = oracle.new_state(4, 8, k, kt, 3, 5, n_a=2)
    rec.keep_history, rec.maxit = True, maxit
    ref = oracle.new_state(4, 8, k, kt, 3, 5, n_a=2)
    oracle.run(rec, measure_every * n_meas, pt_every=1, measure_every=measure_every)
    hist, A_seen, B_seen = [], [], []
    for _ in range(n_meas):
        oracle.run(ref, measure_every, pt_every=1, measure_every=measure_every)
        hist.append(np.argsort(ref.walker_at, axis=2))   # slot of each walker
        A_seen.append(ref.A.copy())
        B_seen.append(ref.B.copy())
    assert rec.n_meas == n_meas
    assert np.array_equal(rec.hist[:n_meas], np.stack(hist).astype(np.uint8))
    n_blocks = n_meas // maxit
    for b in range(n_blocks):
        assert np.array_equal(rec.blkA[b], sum(A_seen[b * maxit:(b + 1) * maxit]))
        assert np.array_equal(rec.blkB[b], sum(B_seen[b * maxit:(b + 1) * maxit]))
    # the complete blocks add up to the running measurement sums
    if n_meas % maxit == 0:
        assert np.array_equal(rec.blkA[:n_blocks].sum(axis=0), rec.sumA)
    # the walk moved (the records are not trivially the identity)
    assert np.any(rec.hist[:n_meas] != np.arange(6))
