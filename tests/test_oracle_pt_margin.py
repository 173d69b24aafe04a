"""Pin of the oracle's PT pass on decisions placed next to the acceptance
boundary (Sec. 2.1: exchange iff u < P, ln P = m dk + n dkt).

The inputs come from tests/pt_targets.py: bond counts chosen so that ln P
falls at, just inside and just outside the GPU kernel's float margin around
ln u, far away, or where a factor leaves the double range.  Here every pass
is replayed pair by pair with the exact logarithm of the oracle's own
rounded bases (mpmath, 40 digits): wherever the exact comparison is decided
by more than the powering's rounding bound, the oracle's permutation must be
the exact one.  A wrong sign, base, exponent or draw in the oracle's PT pass
changes permutations here.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from tests import pt_targets as P

mpmath = pytest.importorskip("mpmath")
mpmath.mp.dps = 40
LN_MAX = 709.78   # ln of the largest double
LN_MIN = -745.13  # ln of the smallest subnormal


def _factor_log(e: int, base: float):
    return abs(e) * mpmath.log(mpmath.mpf(base))


def _decide(m: int, n: int, s: int, bases, x: int):
    """Exact decision of u < P with the oracle's rounded bases, or None when
    rounding of the power chain (or of the range limits) could decide it."""
    ap, am, bp, bm = bases
    la = _factor_log(m, ap[s] if m >= 0 else am[s])
    lb = _factor_log(n, bp[s] if n >= 0 else bm[s])
    for v in (la, lb):
        if abs(abs(v) - LN_MAX) < 2 or abs(v - LN_MIN) < 2:
            return None
    if la > LN_MAX or lb > LN_MAX:
        other = lb if la > LN_MAX else la
        return not (other < LN_MIN)          # inf * 0 is NaN: reject
    if la < LN_MIN or lb < LN_MIN:
        return False                         # a factor is 0
    L = la + lb
    lnu = mpmath.log(mpmath.mpf(x)) - 32 * mpmath.log(2) if x else mpmath.mpf("-inf")
    tol = (2 * (abs(m) + abs(n)) + 4) * 2.0 ** -52
    if min(la, lb) < -700:
        tol += 1e-6                          # subnormal factor
    if abs(lnu - L) <= tol:
        return None
    return bool(lnu < L)


def _exact_pass(k, kt, seed, t, U, wa0):
    """Exact replay; returns (permutations, mask of chains decided exactly)."""
    bases = oracle.pt_bases(k, kt)
    n_samples, n_rep, n_slots = wa0.shape
    out = wa0.copy()
    ok = np.ones((n_samples, n_rep), dtype=bool)
    for a in range(n_samples):
        for r in range(n_rep):
            wa = list(wa0[a, r])
            A = -2 * U[a, r, :, 0]
            B = -2 * U[a, r, :, 1]
            xs = P.pt_draws(seed, np.full(n_slots - 1, a), np.full(n_slots - 1, r),
                            np.arange(n_slots - 1), t) if n_slots > 1 else []
            for s in range(n_slots - 1):
                X, Y = wa[s], wa[s + 1]
                d = _decide(int(A[Y] - A[X]), int(B[Y] - B[X]), s, bases, int(xs[s]))
                if d is None:
                    ok[a, r] = False
                    break
                if d:
                    wa[s], wa[s + 1] = Y, X
            out[a, r] = wa
    return out, ok


@pytest.mark.parametrize("name,k,kt,n_samples,n_rep,lim,search", [
    ("ladder8", None, None, 48, 4, 2 ** 29, True),
    ("tiny", [0.3, 0.3 + 3.7e-6], [0.5, 0.5 - 2.9e-6], 64, 8, 2 ** 29, False),
    ("wide", [0.3, 0.3 + 2.1e-9], [0.5, 0.5 - 1.7e-9], 64, 8, 2 ** 38, False),
    ("far", [0.3, 0.3 + 1e-7], [0.5, 0.5 - 1.3e-7], 64, 8, 2 ** 38, False),
])
def test_oracle_pt_matches_exact_comparison(name, k, kt, n_samples, n_rep, lim, search):
    if k is None:
        k, kt = oracle.ladder_linear(0.2, 0.5, 8, 1.0)
    k, kt = np.asarray(k, dtype=np.float64), np.asarray(kt, dtype=np.float64)
    rng = np.random.default_rng(11)
    seed, t = 0x1234_5678_9ABC, 5
    U, wa0, rel = P.make_case(k, kt, n_samples, n_rep, seed, t, rng, lim, search)
    # the generator reaches the band around the kernel's margin
    assert np.sum((np.abs(rel) > 0.9) & (np.abs(rel) < 1.2)) >= 10
    assert np.sum(np.abs(rel) < 0.5) >= 10
    got = P.oracle_pass(k, kt, seed, t, U, wa0)
    exact, ok = _exact_pass(k, kt, seed, t, U, wa0)
    assert ok.mean() > 0.8, f"{name}: too few chains decided exactly ({ok.mean():.2f})"
    bad = np.argwhere(ok & np.any(got != exact, axis=2))
    assert len(bad) == 0, f"{name}: oracle differs from the exact comparison at chains {bad[:5].tolist()}"
    # and the pass moved walkers (the inputs are not all one-sided)
    assert np.any(got != wa0)
    assert math.isfinite(float(rel.mean()))
