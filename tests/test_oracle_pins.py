"""Pins of the CPU oracle against things other than itself (no GPU).

Each test fixes part of the oracle by something the paper or the mathematics
determines: a library routine (cuRAND's host Philox generator), closed forms,
exact enumeration of tiny lattices, symmetries of the Markov chain, and the
detailed-balance structure of the Metropolis table.
"""
from __future__ import annotations

import ctypes
import ctypes.util
import itertools
import math
import os

import mpmath
import numpy as np
import pytest

import oracle
from tests import exact

mpmath.mp.dps = 50


# --------------------------------------------------------------------------
# Philox4x32-10 (Sec. 2.1.1) against cuRAND's host generator
# --------------------------------------------------------------------------

def _curand():
    cands = [ctypes.util.find_library("curand")]
    for d in ("/usr/local/cuda/lib64", "/usr/local/cuda/targets/sbsa-linux/lib",
              "/usr/local/cuda/targets/x86_64-linux/lib"):
        cands += [os.path.join(d, "libcurand.so"), os.path.join(d, "libcurand.so.10")]
    for c in cands:
        if c and (os.path.exists(c) or not os.path.isabs(c)):
            try:
                return ctypes.CDLL(c)
            except OSError:
                pass
    pytest.skip("libcurand not found")


@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF0, 0xFFFFFFFFFFFFFFFF, 2 ** 32 + 7])
def test_philox_matches_curand_host_generator(seed):
    """cuRAND's host PHILOX4_32_10 generator emits, for output block i, the
    Philox4x32-10 of counter (0, 0, i, 0) under key (seed_lo, seed_hi)."""
    lib = _curand()
    gen = ctypes.c_void_p()
    CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        n = 4 * 512
        out = np.zeros(n, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for i in list(range(0, 512, 7)) + [511]:
        got = oracle.philox4x32_10([0, 0, i, 0], key)
        assert list(got) == list(out[4 * i:4 * i + 4]), (seed, i)


def test_philox_counter_words_all_matter():
    """Each counter word and key word changes the output (no dropped input)."""
    base = oracle.philox4x32_10([11, 22, 33, 44], [55, 66])
    for pos in range(4):
        c = [11, 22, 33, 44]
        c[pos] ^= 1
        assert list(oracle.philox4x32_10(c, [55, 66])) != list(base)
    for pos in range(2):
        kk = [55, 66]
        kk[pos] ^= 1
        assert list(oracle.philox4x32_10([11, 22, 33, 44], kk)) != list(base)


# --------------------------------------------------------------------------
# Ladder: exp(-2 k_tau) = tanh(k Gamma) (Sec. 1, generalised)
# --------------------------------------------------------------------------

def test_ladder_relation_and_equal_coupling_dual():
    k, kt = oracle.ladder_linear(0.25, 0.45, 8, 1.0)
    assert k[0] == 0.25 and k[-1] == 0.45
    assert np.all(np.diff(k) > 0)
    for ks, kts in zip(k, kt):
        lhs = mpmath.exp(-2 * mpmath.mpf(kts))
        rhs = mpmath.tanh(mpmath.mpf(ks) * 1.0)
        assert abs(lhs - rhs) / rhs < 1e-14
    # The paper's equal-coupling relation Gamma = -(1/2k) log tanh k (Sec. 1)
    # is the special case k_tau = k: with that Gamma the ladder returns k_tau = k.
    for kk in (0.29, 0.25, 0.32, 0.4):
        gamma = -math.log(math.tanh(kk)) / (2 * kk)
        _, kt2 = oracle.ladder_linear(kk, kk, 1, gamma)
        assert abs(kt2[0] - kk) < 1e-12


def test_paper_printed_value_footnote():
    """Sec. 2.1.1 footnote: for k = 0.32, e^{-4 k 8} = e^{-10.24} ~ 2^{-14.773}."""
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")
    vals = {}
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                key, v = line.split("=")
                vals[key.strip()] = float(v)
    k = vals["k_max"]
    assert abs(4 * k * 8 - vals["exponent"]) < 1e-12
    assert abs(math.log2(math.exp(-4 * k * 8)) - vals["log2_value"]) < 5e-4


# --------------------------------------------------------------------------
# Metropolis table (Sec. 2.1): detailed balance and the encoding rule
# --------------------------------------------------------------------------

@pytest.mark.parametrize("lo,hi,n,gamma", [(0.25, 0.45, 8, 1.0), (0.2, 0.5, 16, 1.0),
                                           (0.2, 0.5, 32, 0.8), (0.2, 0.5, 9, 1.2)])
def test_threshold_table_detailed_balance(lo, hi, n, gamma):
    k, kt = oracle.ladder_linear(lo, hi, n, gamma)
    T = oracle.thresholds(k, kt)
    two32 = mpmath.mpf(2) ** 32
    for s in range(n):
        for us in range(5):
            for ut in range(3):
                # exact log factor of the flip from the energy change
                d = -4 * mpmath.mpf(k[s]) * (2 - us) - 4 * mpmath.mpf(kt[s]) * (1 - ut)
                rev = T[s, 4 - us, 2 - ut]
                t = T[s, us, ut]
                if d >= 0:
                    assert t == 0xFFFFFFFF
                else:
                    # the reverse move is always accepted
                    assert rev == 0xFFFFFFFF
                    p = mpmath.exp(d)
                    assert t != 0xFFFFFFFF
                    assert abs(mpmath.mpf(int(t)) / two32 - p) <= mpmath.mpf(2) ** -32
                    assert mpmath.mpf(int(t)) <= p * two32
    # eight classes are always accepted for every slot of these ladders
    assert all(int((T[s] == 0xFFFFFFFF).sum()) >= 8 for s in range(n))


def test_threshold_table_equal_coupling_is_daemon_distribution():
    """With k_tau = k every flip costs 4k n, n = 3 - u_s - u_t; Sec. 2.1.1's
    daemon accepts such a move with P(s >= n) = e^{-4 k n}."""
    kk = 0.29
    T = oracle.thresholds(np.array([kk]), np.array([kk]))
    for us in range(5):
        for ut in range(3):
            nn = 3 - us - ut
            if nn <= 0:
                assert T[0, us, ut] == 0xFFFFFFFF
            else:
                assert abs(T[0, us, ut] / 2.0 ** 32 - math.exp(-4 * kk * nn)) < 2.0 ** -31


# --------------------------------------------------------------------------
# PT acceptance (Sec. 2.1)
# --------------------------------------------------------------------------

def test_pt_power_rule_against_exp():
    k, kt = oracle.ladder_linear(0.2, 0.5, 16, 1.0)
    ap, am, bp, bm = oracle.pt_bases(k, kt)
    rng = np.random.default_rng(5)
    for _ in range(200):
        s = int(rng.integers(0, 15))
        m = int(rng.integers(-300, 300))
        n = int(rng.integers(-300, 300))
        P = (oracle.pow_by_squaring(ap[s] if m >= 0 else am[s], abs(m))
             * oracle.pow_by_squaring(bp[s] if n >= 0 else bm[s], abs(n)))
        exact_v = mpmath.exp((mpmath.mpf(k[s]) - mpmath.mpf(k[s + 1])) * m
                             + (mpmath.mpf(kt[s]) - mpmath.mpf(kt[s + 1])) * n)
        # powering the stored bases: a rounding of half an ulp at any
        # multiply or squaring is amplified by the exponent still to come,
        # so the relative error stays below (|m| + |n| + 1) half-ulps
        pw_exact = (mpmath.mpf(ap[s] if m >= 0 else am[s]) ** abs(m)
                    * mpmath.mpf(bp[s] if n >= 0 else bm[s]) ** abs(n))
        assert abs(P - pw_exact) / pw_exact < (abs(m) + abs(n) + 1) * 2.0 ** -53
        # the stored bases are within one ulp, amplified by the exponent
        assert abs(P - exact_v) / exact_v < (2 * (abs(m) + abs(n)) + 1) * 2.0 ** -52
    for s in range(15):
        d = mpmath.mpf(k[s]) - mpmath.mpf(k[s + 1])
        assert abs(ap[s] - mpmath.exp(d)) / mpmath.exp(d) < 2.0 ** -52
        assert abs(am[s] - mpmath.exp(-d)) / mpmath.exp(-d) < 2.0 ** -52


def _stationary_perm_probs(k, kt, A, B):
    n = len(k)
    perms = list(itertools.permutations(range(n)))
    logw = []
    for p in perms:   # p[s] = walker at slot s
        logw.append(sum(mpmath.mpf(k[s]) * A[p[s]] + mpmath.mpf(kt[s]) * B[p[s]]
                        for s in range(n)))
    mx = max(logw)
    w = [mpmath.exp(x - mx) for x in logw]
    Z = sum(w)
    return perms, [float(x / Z) for x in w]


def test_pt_only_chain_samples_product_measure():
    """With configurations frozen, repeated PT passes sample the permutations
    with weight prod_s exp(k_s A_{w(s)} + k_tau,s B_{w(s)}); this fixes the
    sign of the exponent, the pair order and the energy indexing."""
    k = np.array([0.30, 0.34, 0.40])
    kt = np.array([0.55, 0.50, 0.42])
    A = np.array([10, 4, -3], dtype=np.int64)
    B = np.array([2, 9, 5], dtype=np.int64)
    perms, probs = _stationary_perm_probs(k, kt, A, B)
    n_rep, n_a, n_pass = 64, 40, 30
    counts = dict.fromkeys(perms, 0)
    for a in range(n_a):
        wa = np.tile(np.arange(3, dtype=np.int32), (n_rep, 1)).copy()
        Aa = np.tile(A, (n_rep, 1))
        Ba = np.tile(B, (n_rep, 1))
        for t in range(n_pass):
            oracle.pt_only(a, 99, k, kt, t, wa, Aa, Ba)
        for r in range(n_rep):
            counts[tuple(int(x) for x in wa[r])] += 1
    total = n_rep * n_a
    for p, pr in zip(perms, probs):
        sd = math.sqrt(total * pr * (1 - pr))
        assert abs(counts[p] - total * pr) < 5 * sd + 1, (p, counts[p], total * pr)
    # the law is far from uniform, and the counts reject the law a flipped
    # exponent sign would give
    _, flipped = _stationary_perm_probs(k, kt, -A, -B)
    assert any(abs(counts[p] - total * pr) > 5 * math.sqrt(total * pr * (1 - pr)) + 1
               for p, pr in zip(perms, flipped))


# --------------------------------------------------------------------------
# Energies (Eq. (3)) against a vectorised restatement on random states
# --------------------------------------------------------------------------

def test_energies_match_roll_formula():
    rng = np.random.default_rng(3)
    L, Lt = 6, 10
    J = (1 - 2 * rng.integers(0, 2, size=(2, L * L, 2))).astype(np.int8)
    S = (1 - 2 * rng.integers(0, 2, size=(2, 3, 4, L * L * Lt))).astype(np.int8)
    A, B = oracle.energies(L, Lt, J, S)
    for a in range(2):
        A2, B2 = exact.AB_of_configs(S[a].reshape(-1, L * L * Lt), J[a], L, Lt)
        assert np.array_equal(A[a].ravel(), A2)
        assert np.array_equal(B[a].ravel(), B2)


# --------------------------------------------------------------------------
# Statistical pins: Monte Carlo against exact results
# --------------------------------------------------------------------------

def _mc_means(st, n_chunks, chunk):
    """Per-slot chunk means of A and B (averaged over sample and replica)."""
    means_A, means_B = [], []
    for _ in range(n_chunks):
        sA0, sB0, m0 = st.sumA.copy(), st.sumB.copy(), st.n_meas
        oracle.run(st, chunk, pt_every=1, measure_every=1)
        dm = st.n_meas - m0
        means_A.append(((st.sumA - sA0).sum(axis=(0, 1)) / (dm * st.n_a * st.n_rep)))
        means_B.append(((st.sumB - sB0).sum(axis=(0, 1)) / (dm * st.n_a * st.n_rep)))
    mA, mB = np.array(means_A), np.array(means_B)
    return (mA.mean(0), mA.std(0, ddof=1) / math.sqrt(n_chunks),
            mB.mean(0), mB.std(0, ddof=1) / math.sqrt(n_chunks))


def _spatially_free_sites(J, L=2):
    """Sites whose four spatial bonds cancel whatever the spins (at L=2 both
    x-bonds of a site join the same pair, likewise the y-bonds)."""
    out = []
    for i in range(L * L):
        x, y = i % L, i // L
        jx, jy = (x + 1) % L + L * y, x + L * ((y + 1) % L)
        if J[i][0] != J[jx][0] and J[i][1] != J[jy][1]:
            out.append(i)
    return out


@pytest.mark.parametrize("seed", [2, 6])
def test_enumeration_L2_Ltau4_with_pt(seed):
    """L=2, L_tau=4 (16 spins, 65536 states): MC <A>, <B> per ladder slot
    match exact enumeration within 4 sigma.  At L=2 the bonds (x,+x) and
    (x+1,+x) join the same two sites and carry independent couplings.

    The seeds are ones whose couplings leave no spatially free site: such a
    site always has u_s = 2, and its imaginary-time ring of 4 spins under
    red/blue Metropolis (a flip of zero cost is always taken) keeps its
    domain walls forever, so time averages there depend on the start."""
    L, Lt = 2, 4
    k, kt = oracle.ladder_linear(0.25, 0.45, 4, 1.0)
    st = oracle.new_state(L, Lt, k, kt, n_rep=8, seed=seed)
    J = st.J[0]
    assert _spatially_free_sites(J) == []
    oracle.run(st, 200)                         # equilibrate
    mA, eA, mB, eB = _mc_means(st, 60, 400)
    for s in range(len(k)):
        xA, xB, _, _ = exact.enumerate_AB(J, L, Lt, k[s], kt[s])
        assert abs(mA[s] - xA) < 4 * eA[s] + 1e-9, (s, mA[s], xA, eA[s])
        assert abs(mB[s] - xB) < 4 * eB[s] + 1e-9, (s, mB[s], xB, eB[s])


def test_k_zero_trajectory_ignores_couplings():
    """k = 0: the Metropolis factor depends on u_t only, so the spin
    trajectory and the permutation are the same for any J (bit for bit),
    and B, which does not involve J, is the same too.  (The closed form of
    the periodic chain cannot pin the chain itself at k = 0: a ring of
    spins under red/blue Metropolis, where a zero-cost flip is always
    taken, is not ergodic.)"""
    L, Lt = 4, 8
    kts = np.array([0.2, 0.5, 0.9])
    st = oracle.new_state(L, Lt, np.zeros(3), kts, n_rep=4, seed=11)
    tw = _twin(st)
    oracle.alloc_obs(tw)
    tw.J = (-st.J).astype(np.int8)
    tw.J[0, 3, 1] = st.J[0, 3, 1]
    oracle.run(st, 30)
    oracle.run(tw, 30)
    assert np.array_equal(st.S, tw.S) and np.array_equal(st.walker_at, tw.walker_at)
    assert np.array_equal(st.B, tw.B)
    assert not np.array_equal(st.A, tw.A)


def test_k_tau_zero_layer_flip_maps_trajectory():
    """k_tau = 0: flipping every spin of one imaginary-time layer leaves all
    u_s unchanged and u_t unused, so the trajectory maps bit for bit."""
    L, Lt = 4, 6
    ks = np.array([0.2, 0.45, 0.8])
    st = oracle.new_state(L, Lt, ks, np.zeros(3), n_rep=4, seed=17)
    tw = _twin(st)
    oracle.alloc_obs(tw)
    flip = np.ones(L * L * Lt, dtype=np.int8)
    flip[2 * L * L:3 * L * L] = -1          # layer tau = 2
    tw.S = (st.S * flip).astype(np.int8)
    oracle.run(st, 30)
    oracle.run(tw, 30)
    assert np.array_equal(tw.S, st.S * flip)
    assert np.array_equal(tw.walker_at, st.walker_at)
    assert np.array_equal(tw.A, st.A)


def test_k_tau_zero_independent_layers():
    L, Lt = 4, 4
    ks = np.array([0.2, 0.45, 0.8])
    st = oracle.new_state(L, Lt, ks, np.zeros(3), n_rep=4, seed=13)
    J = st.J[0]
    oracle.run(st, 200)
    mA, eA, mB, eB = _mc_means(st, 60, 100)
    for s in range(3):
        xA = Lt * exact.layer_A(J, L, ks[s])
        assert abs(mA[s] - xA) < 4 * eA[s] + 1e-9, (s, mA[s], xA, eA[s])
        assert abs(mB[s]) < 4 * eB[s] + 1e-9


# --------------------------------------------------------------------------
# Symmetries: exact maps of whole trajectories
# --------------------------------------------------------------------------

def _twin(st):
    return oracle.OracleState(st.L, st.Ltau, st.k, st.ktau, st.n_rep, st.a_lo, st.n_a,
                              st.seed, st.J.copy(), st.S.copy(), st.walker_at.copy())


def test_global_spin_flip_maps_trajectory():
    k, kt = oracle.ladder_linear(0.25, 0.45, 8, 1.0)
    st = oracle.new_state(6, 8, k, kt, 4, seed=21, a_lo=3, n_a=2)
    tw = _twin(st)
    oracle.alloc_obs(tw)
    tw.S = (-tw.S).astype(np.int8)
    oracle.run(st, 25)
    oracle.run(tw, 25)
    assert np.array_equal(tw.S, -st.S)
    assert np.array_equal(tw.walker_at, st.walker_at)
    assert np.array_equal(tw.A, st.A) and np.array_equal(tw.B, st.B)


def test_gauge_transform_maps_trajectory():
    L, Lt = 6, 8
    k, kt = oracle.ladder_linear(0.2, 0.5, 6, 1.0)
    st = oracle.new_state(L, Lt, k, kt, 4, seed=5, a_lo=0, n_a=2)
    rng = np.random.default_rng(8)
    eps = (1 - 2 * rng.integers(0, 2, size=(2, L * L))).astype(np.int8)
    tw = _twin(st)
    oracle.alloc_obs(tw)
    for a in range(2):
        for i in range(L * L):
            x, y = i % L, i // L
            jx = (x + 1) % L + L * y
            jy = x + L * ((y + 1) % L)
            tw.J[a, i, 0] = eps[a, i] * st.J[a, i, 0] * eps[a, jx]
            tw.J[a, i, 1] = eps[a, i] * st.J[a, i, 1] * eps[a, jy]
    e_site = np.tile(eps, (1, Lt))                         # [a][N]
    tw.S = (st.S * e_site[:, None, None, :]).astype(np.int8)
    oracle.run(st, 25)
    oracle.run(tw, 25)
    assert np.array_equal(tw.S, st.S * e_site[:, None, None, :])
    assert np.array_equal(tw.walker_at, st.walker_at)
    assert np.array_equal(tw.A, st.A) and np.array_equal(tw.B, st.B)


def test_sample_subsets_are_independent():
    """Running samples 2..3 alone equals running them inside 0..3."""
    k, kt = oracle.ladder_linear(0.25, 0.45, 4, 1.0)
    full = oracle.new_state(4, 8, k, kt, 4, seed=9, a_lo=0, n_a=4)
    part = oracle.new_state(4, 8, k, kt, 4, seed=9, a_lo=2, n_a=2)
    oracle.run(full, 15)
    oracle.run(part, 15)
    assert np.array_equal(full.S[2:], part.S)
    assert np.array_equal(full.walker_at[2:], part.walker_at)


def test_run_is_resumable():
    k, kt = oracle.ladder_linear(0.25, 0.45, 4, 1.0)
    a = oracle.new_state(4, 8, k, kt, 4, seed=9)
    b = oracle.new_state(4, 8, k, kt, 4, seed=9)
    oracle.run(a, 12, measure_every=3)
    oracle.run(b, 5, measure_every=3)
    oracle.run(b, 7, measure_every=3)
    assert np.array_equal(a.S, b.S) and np.array_equal(a.walker_at, b.walker_at)
    assert np.array_equal(a.sumA, b.sumA) and np.array_equal(a.sumq2, b.sumq2)
    assert a.n_meas == b.n_meas == 4


def test_overlap_identity():
    """q = N - 2 * (number of sites where the two configurations differ);
    at measurement time the sums equal the overlaps of the state."""
    k, kt = oracle.ladder_linear(0.25, 0.45, 3, 1.0)
    st = oracle.new_state(4, 4, k, kt, 3, seed=2)
    oracle.run(st, 4, measure_every=4)
    S, wa = st.S[0], st.walker_at[0]
    p = 0
    for r1 in range(3):
        for r2 in range(r1 + 1, 3):
            for s in range(3):
                d = int((S[r1, wa[r1, s]] != S[r2, wa[r2, s]]).sum())
                assert st.sumq[0, s, p] == st.N - 2 * d
            p += 1


# --------------------------------------------------------------------------
# Antiperiodic boundary along tau (Sec. 1: S_{x,L_tau} = -S_{x,0})
# --------------------------------------------------------------------------

def test_exact_ring_closed_form_both_boundaries():
    """The enumeration helper against the transfer-matrix closed form of an
    Ising ring (k = 0 leaves independent rings): Z = (2 cosh K)^n +-
    (2 sinh K)^n, the minus sign for one bond of opposite sign."""
    J = np.ones((1, 2), dtype=np.int8)
    for ap in (False, True):
        for n in (4, 5, 6):
            for K in (0.3, 0.7, 1.1):
                _, xB, _, _ = exact.enumerate_AB(J, 1, n, 0.0, K, tau_ap=ap)
                assert abs(xB - exact.chain_B(1, n, K, tau_ap=ap)) < 1e-9 * n


def test_energies_antiperiodic_match_roll_formula():
    rng = np.random.default_rng(5)
    L, Lt = 4, 6
    J = (1 - 2 * rng.integers(0, 2, size=(2, L * L, 2))).astype(np.int8)
    S = (1 - 2 * rng.integers(0, 2, size=(2, 3, 4, L * L * Lt))).astype(np.int8)
    A, B = oracle.energies(L, Lt, J, S, tau_ap=True)
    Ap, Bp = oracle.energies(L, Lt, J, S, tau_ap=False)
    for a in range(2):
        A2, B2 = exact.AB_of_configs(S[a].reshape(-1, L * L * Lt), J[a], L, Lt, tau_ap=True)
        assert np.array_equal(A[a].ravel(), A2)
        assert np.array_equal(B[a].ravel(), B2)
    # only the wrap bond changes sign: B_ap = B_p - 2 sum_x S_{x,L_tau-1} S_{x,0}
    V = S.reshape(2, 3, 4, Lt, L * L).astype(np.int64)
    wrap = (V[:, :, :, Lt - 1] * V[:, :, :, 0]).sum(axis=-1)
    assert np.array_equal(B, Bp - 2 * wrap)
    assert np.array_equal(A, Ap)


@pytest.mark.parametrize("seed", [2])
def test_enumeration_L2_Ltau4_antiperiodic(seed):
    """L=2, L_tau=4 antiperiodic: MC <A>, <B> per slot match exact
    enumeration with the wrap bond of opposite sign (within 4 sigma)."""
    L, Lt = 2, 4
    k, kt = oracle.ladder_linear(0.25, 0.45, 4, 1.0)
    st = oracle.new_state(L, Lt, k, kt, n_rep=8, seed=seed, tau_ap=True)
    J = st.J[0]
    assert _spatially_free_sites(J) == []
    oracle.run(st, 200)
    mA, eA, mB, eB = _mc_means(st, 60, 400)
    for s in range(len(k)):
        xA, xB, _, _ = exact.enumerate_AB(J, L, Lt, k[s], kt[s], tau_ap=True)
        pA, pB, _, _ = exact.enumerate_AB(J, L, Lt, k[s], kt[s], tau_ap=False)
        assert abs(mA[s] - xA) < 4 * eA[s] + 1e-9, (s, mA[s], xA, eA[s])
        assert abs(mB[s] - xB) < 4 * eB[s] + 1e-9, (s, mB[s], xB, eB[s])
        assert abs(xB - pB) > 8 * eB[s]   # the boundary is visible in <B>


def test_k_tau_zero_antiperiodic_same_spins():
    """k_tau = 0: the table ignores u_t, so the antiperiodic run follows the
    periodic spin trajectory bit for bit; only B differs (the wrap bond)."""
    L, Lt = 4, 6
    ks = np.array([0.2, 0.45, 0.8])
    st = oracle.new_state(L, Lt, ks, np.zeros(3), n_rep=4, seed=19)
    ap = oracle.new_state(L, Lt, ks, np.zeros(3), n_rep=4, seed=19, tau_ap=True)
    oracle.run(st, 30)
    oracle.run(ap, 30)
    assert np.array_equal(st.S, ap.S) and np.array_equal(st.walker_at, ap.walker_at)
    assert np.array_equal(st.A, ap.A)
    assert not np.array_equal(st.B, ap.B)


@pytest.mark.parametrize("tau_ap", [False, True])
def test_long_tau_chain_matches_transfer_matrix(tau_ap):
    """L=2, L_tau=32 with separate couplings (k, k_tau) of a Gamma = 0.9
    ladder and PT: MC <A>, <B> per slot match the transfer-matrix values of
    the same boundary within 4 sigma, and at the first slot <B> excludes the
    other boundary's value (about 5 apart at this size)."""
    L, Lt = 2, 32
    k, kt = oracle.ladder_linear(0.3, 0.6, 2, 0.9)
    st = oracle.new_state(L, Lt, k, kt, n_rep=8, seed=2, tau_ap=tau_ap)
    J = st.J[0]
    assert _spatially_free_sites(J) == []
    oracle.run(st, 300)
    mA, eA, mB, eB = _mc_means(st, 30, 40)
    for s in range(2):
        xA, xB = exact.transfer_AB(J, L, Lt, k[s], kt[s], tau_ap)
        assert abs(mA[s] - xA) < 4 * eA[s] + 1e-9, (s, mA[s], xA, eA[s])
        assert abs(mB[s] - xB) < 4 * eB[s] + 1e-9, (s, mB[s], xB, eB[s])
    _, oB = exact.transfer_AB(J, L, Lt, k[0], kt[0], not tau_ap)
    assert abs(mB[0] - oB) > 8 * eB[0]
