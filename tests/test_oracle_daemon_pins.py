"""Pins of the oracle's daemon rule (Sec. 2.1.1, Appendices B and C) against
things other than itself (no GPU): the truth table the paper prints, the
closed-form probabilities of the inverse-cumulative bytes, the full period of
the xoroshiro128 state step, the Metropolis probabilities of Eq. (3) at equal
couplings, and exact averages of a small prism from its transfer matrix.
"""
from __future__ import annotations

import math
import os
from fractions import Fraction

import mpmath
import numpy as np
import pytest

import oracle
from tests import exact

mpmath.mp.dps = 50
TWO64 = 1 << 64


# --------------------------------------------------------------------------
# Appendix B: the daemon's truth table
# --------------------------------------------------------------------------

def _truth_rows():
    path = os.path.join(os.path.dirname(__file__), "golden", "daemon_truth_table.txt")
    rows = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            b, ids, s, prob = [x.strip() for x in line.split("|")]
            rows.append((tuple(int(v) for v in b.split()), tuple(int(v) for v in ids.split()), int(s), prob))
    return rows


def test_daemon_truth_table_from_paper():
    rows = _truth_rows()
    assert len(rows) == 4
    for (b4, b8, b12), (id1, id2), s, _ in rows:
        assert id1 + 2 * id2 == s
        assert oracle.daemon_level(b4, b8, b12) == s


def test_daemon_level_distribution_closed_form():
    """Raw bits independent, each 1 with probability p: after the AND steps
    the level has the distribution of the paper's table, whatever the raw
    pattern (all 8 are reachable)."""
    rows = _truth_rows()
    for p in (Fraction(1, 3), Fraction(3, 10), Fraction(7, 100)):
        dist = [Fraction(0)] * 4
        for raw in range(8):
            b = [(raw >> i) & 1 for i in range(3)]
            pr = Fraction(1)
            for v in b:
                pr *= p if v else 1 - p
            # the level only sees the ANDed pattern
            b8 = b[0] & b[1]
            b12 = b8 & b[2]
            assert oracle.daemon_level(*b) == oracle.daemon_level(b[0], b8, b12)
            dist[oracle.daemon_level(*b)] += pr
        want = {"1-p": 1 - p, "p-p^2": p - p * p, "p^2-p^3": p * p - p ** 3, "p^3": p ** 3}
        for _, _, s, prob in rows:
            assert dist[s] == want[prob], (s, dist[s], want[prob])


def test_daemon_flip_is_metropolis_at_equal_coupling():
    """A site with u of its 6 bonds unsatisfied: the energy change of Eq. (3)
    (k_tau = k, evaluated on an explicit star of 6 neighbours) against the
    flip probability sum_d P(d) [flip(u, d)] of the daemon of the table."""
    for k in (0.05, 0.29, 0.5):
        p = math.exp(-4 * k)
        Pd = [1 - p, p - p * p, p * p - p ** 3, p ** 3]
        for u in range(7):
            S0 = 1
            nb = [-S0] * u + [S0] * (6 - u)          # J = +1 on every bond
            E_before = -sum(S0 * v for v in nb)
            E_after = -sum(-S0 * v for v in nb)
            want = min(1.0, math.exp(-k * (E_after - E_before)))
            got = sum(Pd[d] for d in range(4) if oracle.daemon_flip(u, d))
            assert abs(got - want) < 1e-15, (k, u, got, want)


# --------------------------------------------------------------------------
# Sec. 2.1.1: the cumulative table and n*
# --------------------------------------------------------------------------

def _bin_probs(cum):
    c = [0] + [int(v) for v in cum] + [TWO64]
    return [Fraction(c[n + 1] - c[n], TWO64) for n in range(256)]


@pytest.mark.parametrize("k", [0.0, 0.1, 0.29, 0.5, 1.3, 16.0])
def test_daemon_cumulative_is_product_of_bernoulli_bits(k):
    """Each of the 8 bits of n* is 1 with probability e^{-4k}, pairs are
    independent, and P(n) = p^pop(n) (1-p)^(8-pop(n)), all within the
    truncation of the 255 cut points (2^-64 each)."""
    cum = oracle.daemon_cumulative(k)
    assert np.all(np.diff(cum.astype(object)) >= 0)
    P = _bin_probs(cum)
    p = mpmath.exp(-4 * mpmath.mpf(k))
    tol = mpmath.mpf(2) ** -55
    for i in range(8):
        m = sum(P[n] for n in range(256) if (n >> i) & 1)
        assert abs(mpmath.mpf(m.numerator) / m.denominator - p) < tol
        for j in range(i + 1, 8):
            m2 = sum(P[n] for n in range(256) if (n >> i) & 1 and (n >> j) & 1)
            assert abs(mpmath.mpf(m2.numerator) / m2.denominator - p * p) < tol
    for n in range(256):
        c = bin(n).count("1")
        want = p ** c * (1 - p) ** (8 - c)
        assert abs(mpmath.mpf(P[n].numerator) / P[n].denominator - want) < mpmath.mpf(2) ** -63


def test_daemon_nstar_bins():
    """n*(R) is the bin of R: the last word below cumulative(n) lies in bin n
    and cumulative(n) itself in the next one; the extremes give 0 and 255."""
    cum = oracle.daemon_cumulative(0.29)
    c = [int(v) for v in cum]
    assert oracle.daemon_nstar(cum, 0) == 0
    assert oracle.daemon_nstar(cum, TWO64 - 1) == 255
    for n in range(255):
        lo = c[n - 1] if n > 0 else 0
        if c[n] > lo:
            assert oracle.daemon_nstar(cum, c[n] - 1) == n
        nxt = c[n + 1] if n + 1 < 255 else TWO64
        if nxt > c[n]:
            assert oracle.daemon_nstar(cum, c[n]) == n + 1


def test_daemon_words_bit_statistics():
    """Bits of the daemon words from many counters: frequency e^{-4k} at
    every bit position, independent across neighbouring bits and across
    the three words of one site (binomial 5-sigma bounds)."""
    k = 0.29
    p = math.exp(-4 * k)
    cum = oracle.daemon_cumulative(k)
    n = 3000
    W = np.zeros((3, n), dtype=np.uint64)
    for c in range(n):
        for which in range(3):
            W[which, c] = oracle.daemon_bword(12345, c % 7, c % 3, c % 5, c, c // 11, which, cum)
    bits = ((W[:, :, None] >> np.arange(32, dtype=np.uint64)) & np.uint64(1)).astype(np.float64)
    freq = bits.mean(axis=1)                                  # [3][32]
    sd1 = math.sqrt(p * (1 - p) / n)
    assert np.all(np.abs(freq - p) < 5 * sd1), freq
    sd2 = math.sqrt(p * p * (1 - p * p) / (n * 31))
    adj = (bits[:, :, :-1] * bits[:, :, 1:]).mean(axis=(1, 2))
    assert np.all(np.abs(adj - p * p) < 5 * sd2), adj
    sd3 = math.sqrt(p * p * (1 - p * p) / (n * 32))
    for a_, b_ in ((0, 1), (0, 2), (1, 2)):
        cross = (bits[a_] * bits[b_]).mean()
        assert abs(cross - p * p) < 5 * sd3, (a_, b_, cross)


# --------------------------------------------------------------------------
# xoroshiro128 state step: a full-period linear map
# --------------------------------------------------------------------------

def _is_prime(n: int) -> bool:
    if n < 2:
        return False
    for q in (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37):
        if n % q == 0:
            return n == q
    d, r = n - 1, 0
    while d % 2 == 0:
        d //= 2
        r += 1
    for a in (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37):   # deterministic below 3.3e24
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(r - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def _bits128(s0, s1):
    v = np.zeros(128, dtype=np.int64)
    for i in range(64):
        v[i] = (s0 >> i) & 1
        v[64 + i] = (s1 >> i) & 1
    return v


def _matpow(M, e):
    R = np.eye(128, dtype=np.int64)
    B = M.copy()
    while e:
        if e & 1:
            R = (R @ B) & 1
        B = (B @ B) & 1
        e >>= 1
    return R


def test_xoroshiro_state_step_has_full_period():
    """The step is GF(2)-linear and its matrix has multiplicative order
    2^128 - 1, the period of the published xoroshiro128 generators: M^(2^128)
    = M, and M^((2^128-1)/q) != I for every prime q of 2^128 - 1."""
    cols = []
    for i in range(128):
        s0, s1 = (1 << i, 0) if i < 64 else (0, 1 << (i - 64))
        cols.append(_bits128(*oracle.xoroshiro128pp_step(s0, s1)))
    M = np.stack(cols, axis=1)
    rng = np.random.default_rng(3)
    for _ in range(20):
        s0, s1 = (int.from_bytes(rng.bytes(8), "little") for _ in range(2))
        assert np.array_equal((M @ _bits128(s0, s1)) & 1, _bits128(*oracle.xoroshiro128pp_step(s0, s1)))
    order = (1 << 128) - 1
    factors = [3, 5, 17, 257, 641, 65537, 274177, 6700417, 67280421310721]
    assert math.prod(factors) == order and all(_is_prime(q) for q in factors)
    B = M.copy()
    for _ in range(128):
        B = (B @ B) & 1
    assert np.array_equal(B, M)
    eye = np.eye(128, dtype=np.int64)
    for q in factors:
        assert not np.array_equal(_matpow(M, order // q), eye), q


# --------------------------------------------------------------------------
# The daemon chain against exact averages
# --------------------------------------------------------------------------

def _spatially_free_sites(J, L=2):
    out = []
    for i in range(L * L):
        x, y = i % L, i // L
        jx, jy = (x + 1) % L + L * y, x + L * ((y + 1) % L)
        if J[i][0] != J[jx][0] and J[i][1] != J[jy][1]:
            out.append(i)
    return out


def test_daemon_rule_needs_equal_coupling():
    k, kt = oracle.ladder_linear(0.25, 0.45, 2, 1.0)
    with pytest.raises(ValueError):
        oracle.new_state(2, 64, k, kt, 1, 1, daemon=True)
    with pytest.raises(ValueError):
        oracle.new_state(2, 32, k, k, 1, 1, daemon=True)


@pytest.mark.parametrize("seed", [2])
def test_daemon_chain_matches_transfer_matrix_L2(seed):
    """L=2, L_tau=64, k_tau = k on a 2-slot ladder with PT: Monte Carlo <A>,
    <B> per slot of the daemon chain match the transfer-matrix values
    within 4 sigma (chunk means over 8 replicas)."""
    L, Lt = 2, 64
    k = np.array([0.3, 0.42])
    st = oracle.new_state(L, Lt, k, k.copy(), n_rep=8, seed=seed, daemon=True)
    J = st.J[0]
    assert _spatially_free_sites(J) == []
    oracle.run(st, 200)
    means_A, means_B = [], []
    for _ in range(30):
        sA0, sB0, m0 = st.sumA.copy(), st.sumB.copy(), st.n_meas
        oracle.run(st, 40, pt_every=1, measure_every=1)
        dm = st.n_meas - m0
        means_A.append((st.sumA - sA0).sum(axis=(0, 1)) / (dm * st.n_rep))
        means_B.append((st.sumB - sB0).sum(axis=(0, 1)) / (dm * st.n_rep))
    mA, mB = np.array(means_A), np.array(means_B)
    eA = mA.std(0, ddof=1) / math.sqrt(len(mA))
    eB = mB.std(0, ddof=1) / math.sqrt(len(mB))
    for s in range(2):
        xA, xB = exact.transfer_AB(J, L, Lt, k[s], k[s])
        assert abs(mA.mean(0)[s] - xA) < 4 * eA[s] + 1e-9, (s, mA.mean(0)[s], xA, eA[s])
        assert abs(mB.mean(0)[s] - xB) < 4 * eB[s] + 1e-9, (s, mB.mean(0)[s], xB, eB[s])


def test_transfer_matrix_matches_enumeration():
    rng = np.random.default_rng(5)
    for L, Lt in ((2, 3), (2, 4)):
        J = (1 - 2 * rng.integers(0, 2, size=(L * L, 2))).astype(np.int8)
        for k, kt in ((0.3, 0.3), (0.2, 0.8)):
            for ap in (False, True):
                a, b, _, _ = exact.enumerate_AB(J, L, Lt, k, kt, ap)
                ta, tb = exact.transfer_AB(J, L, Lt, k, kt, ap)
                assert abs(a - ta) < 1e-9 and abs(b - tb) < 1e-9, (L, Lt, k, kt, ap)


def test_daemon_chain_antiperiodic_matches_transfer_matrix_L2():
    """L=2, L_tau=64, antiperiodic along tau, k in {0.6, 0.8}: MC <A>, <B>
    match the antiperiodic transfer-matrix values within 4 sigma, and <B> at
    k = 0.8 excludes the periodic value (about 8 apart at this size)."""
    L, Lt = 2, 64
    k = np.array([0.6, 0.8])
    st = oracle.new_state(L, Lt, k, k.copy(), n_rep=8, seed=2, daemon=True, tau_ap=True)
    J = st.J[0]
    assert _spatially_free_sites(J) == []
    oracle.run(st, 300)
    means_A, means_B = [], []
    for _ in range(30):
        sA0, sB0, m0 = st.sumA.copy(), st.sumB.copy(), st.n_meas
        oracle.run(st, 40, pt_every=1, measure_every=1)
        dm = st.n_meas - m0
        means_A.append((st.sumA - sA0).sum(axis=(0, 1)) / (dm * st.n_rep))
        means_B.append((st.sumB - sB0).sum(axis=(0, 1)) / (dm * st.n_rep))
    mA, mB = np.array(means_A), np.array(means_B)
    eA = mA.std(0, ddof=1) / math.sqrt(len(mA))
    eB = mB.std(0, ddof=1) / math.sqrt(len(mB))
    for s in range(2):
        xA, xB = exact.transfer_AB(J, L, Lt, k[s], k[s], True)
        assert abs(mA.mean(0)[s] - xA) < 4 * eA[s] + 1e-9, (s, mA.mean(0)[s], xA, eA[s])
        assert abs(mB.mean(0)[s] - xB) < 4 * eB[s] + 1e-9, (s, mB.mean(0)[s], xB, eB[s])
    _, pB = exact.transfer_AB(J, L, Lt, k[1], k[1], False)
    assert abs(mB.mean(0)[1] - pB) > 20 * eB[1]


def test_one_system_sweep_is_the_chain_sweep():
    """The oracle's one-system sweep (used where the full chain is too slow)
    applies to a system exactly what the full run does to it (no PT)."""
    L, Lt = 4, 128
    k = np.array([0.25, 0.4, 0.55])
    for tau_ap in (False, True):
        st = oracle.new_state(L, Lt, k, k.copy(), n_rep=2, seed=8, n_a=2, tau_ap=tau_ap, daemon=True)
        S0 = st.S.copy()
        oracle.run(st, 2, pt_every=0)
        for a in range(2):
            for r in range(2):
                for w in range(3):
                    S = np.ascontiguousarray(S0[a, r, w])
                    for t in range(2):
                        oracle.daemon_sweep_system(L, Lt, 8, a, r, w, t, st.J[a], S, st.cum, tau_ap)
                    assert np.array_equal(S, st.S[a, r, w]), (tau_ap, a, r, w)
