"""Bond counts that place parallel-tempering decisions at chosen distances
from their acceptance boundary (test input generator, no GPU).

Sec. 2.1: the pair (s, s+1) of a chain exchanges iff u < P with
ln P = m dk + n dkt, m = A_Y - A_X, n = B_Y - B_X (A = 2N - 2 u_s,
B = N - 2 u_t), dk = k_s - k_{s+1}, dkt = k_tau,s - k_tau,s+1 and u the
pair's Philox word times 2^-32.  Given the draws, the generator picks the
integer count differences so that ln P lands where asked: at a chosen
multiple of the PT kernel's float-shortcut margin from ln u, at random, or
beyond the range where the factors stay finite.  Only the bond counts and
the start permutation are produced here; which pairs exchange is for the code
under test and the oracle to decide.
"""
from __future__ import annotations

import numpy as np

import oracle

LN2_32 = 32.0 * np.log(2.0)

# multiples of the margin placed around ln u (0: at the boundary itself)
NEAR = np.array([0.0, 0.3, -0.3, 0.9, -0.9, 0.99, -0.99, 1.01, -1.01, 1.1, -1.1, 1.5, -1.5, 3.0, -3.0])


def pt_draws(seed: int, a: np.ndarray, r: np.ndarray, s: np.ndarray, t: int) -> np.ndarray:
    """The PT word x of pair s of chain (a, r) after sweep t: word r & 3 of
    Philox(ctr (s, t, a, 4 << 28 | r >> 2), key (seed_lo, seed_hi))."""
    n = len(a)
    ctr = np.stack([s, np.full(n, t), a, (4 << 28) | (r >> 2)], axis=1).astype(np.uint64).astype(np.uint32)
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)
    out = oracle.philox4x32_10_many(ctr, key)
    return out[np.arange(n), r & 3]


def kernel_margin(m, n, dk: float, dkt: float) -> np.ndarray:
    """The PT kernel's float margin 1e-4 + (|m dk| + |n dkt|) 4.8e-7, with its
    float32 products."""
    la = np.abs(np.float32(m.astype(np.float32) * np.float32(dk))).astype(np.float64)
    lb = np.abs(np.float32(n.astype(np.float32) * np.float32(dkt))).astype(np.float64)
    return 1e-4 + (la + lb) * 4.8e-7


def _solve(T, dk: float, dkt: float, rng, search: np.ndarray):
    """Integers (i, j), m = 2i, n = 2j, with 2 i dk + 2 j dkt close to T
    (dk, dkt nonzero).  Where `search` is set, j is scanned over [-1000, 1000]
    for the smallest residual of i (incommensurate dk and dkt); elsewhere j
    is 0, a small random integer, or carries most of T."""
    n = len(T)
    mode = rng.integers(0, 3, n)
    j = np.where(mode == 1, rng.integers(-50, 51, n), 0).astype(np.int64)
    j = np.where(mode == 2, np.rint(T / (2.0 * dkt)), j).astype(np.int64)
    idx = np.flatnonzero(search)
    cand = np.arange(-1000, 1001, dtype=np.int64)
    for lo in range(0, len(idx), 256):
        sel = idx[lo:lo + 256]
        ir = (T[sel, None] - 2.0 * cand[None, :] * dkt) / (2.0 * dk)
        j[sel] = cand[np.argmin(np.abs(ir - np.rint(ir)), axis=1)]
    i = np.rint((T - 2.0 * j * dkt) / (2.0 * dk)).astype(np.int64)
    return i, j


def make_case(k, kt, n_samples: int, n_rep: int, seed: int, t: int, rng, lim: int, search: bool,
              frac_near: float = 0.6, frac_far: float = 0.05):
    """Bond counts U [a][r][walker][2] and start permutations [a][r][slot].

    Per pair, a fraction frac_near of the decisions is placed at NEAR
    multiples of the kernel margin from ln u, frac_far at |ln P| of about 800
    (factors that leave the double range, including inf * 0), the rest at
    ln P uniform in [-6, 1].  Counts stay in [0, lim).  Returns U, walker_at
    and, per targeted pair, (ln P - ln u) / margin for coverage checks."""
    k = np.asarray(k, dtype=np.float64)
    kt = np.asarray(kt, dtype=np.float64)
    n_slots = len(k)
    n_ch = n_samples * n_rep
    a = np.repeat(np.arange(n_samples, dtype=np.int64), n_rep)
    r = np.tile(np.arange(n_rep, dtype=np.int64), n_samples)
    perm = np.argsort(rng.random((n_ch, n_slots)), axis=1).astype(np.int32)
    us = np.zeros((n_ch, n_slots), dtype=np.int64)   # by slot of the originals
    ut = np.zeros_like(us)
    us[:, 0] = lim // 2
    ut[:, 0] = lim // 2
    rel = []
    for s in range(n_slots - 1):
        dk, dkt = float(k[s] - k[s + 1]), float(kt[s] - kt[s + 1])
        x = pt_draws(seed, a, r, np.full(n_ch, s, dtype=np.int64), t).astype(np.float64)
        lnu = np.log(np.maximum(x, 1.0)) - LN2_32
        cat = rng.random(n_ch)
        T = rng.uniform(-6.0, 1.0, n_ch)
        far = cat >= 1.0 - frac_far
        sgn = rng.integers(0, 3, n_ch)   # +800, -800, or +800 / -800 split over m and n
        T = np.where(far, np.where(sgn == 0, 800.0, -800.0), T)
        near = cat < frac_near
        T = np.where(near, lnu, T)
        scan = near & search
        i, j = _solve(T, dk, dkt, rng, scan)
        f = NEAR[rng.integers(0, len(NEAR), n_ch)]
        err = kernel_margin(2 * i, 2 * j, dk, dkt)
        T = np.where(near, lnu + f * err, T)
        i, j = _solve(T, dk, dkt, rng, scan)
        split = far & (sgn == 2)
        i = np.where(split, np.rint(800.0 / (2.0 * dk)).astype(np.int64), i)
        j = np.where(split, np.rint(-800.0 / (2.0 * dkt)).astype(np.int64), j)
        # steps too large for the count range (tiny dk with |ln P| ~ 800):
        # those decisions fall back to ln P uniform in [-6, 1]
        cap = lim // (2 * n_slots)
        big = (np.abs(i) > cap) | (np.abs(j) > cap)
        if big.any():
            i2, j2 = _solve(rng.uniform(-6.0, 1.0, n_ch), dk, dkt, rng, np.zeros(n_ch, bool))
            i, j = np.where(big, i2, i), np.where(big, j2, j)
        us[:, s + 1] = us[:, s] - i
        ut[:, s + 1] = ut[:, s] - j
        lnP = 2.0 * i * dk + 2.0 * j * dkt
        rel.append(((lnP - lnu) / kernel_margin(2 * i, 2 * j, dk, dkt))[near])
    if us.min() < 0 or us.max() >= lim or ut.min() < 0 or ut.max() >= lim:
        raise ValueError("bond counts outside the requested range")
    # slot order -> walker order: walker perm[c][s] holds the counts of slot s
    U = np.zeros((n_ch, n_slots, 2), dtype=np.int64)
    rows = np.arange(n_ch)[:, None]
    U[rows, perm, 0] = us
    U[rows, perm, 1] = ut
    return (U.reshape(n_samples, n_rep, n_slots, 2), perm.reshape(n_samples, n_rep, n_slots),
            np.concatenate(rel) if rel else np.zeros(0))


def oracle_pass(k, kt, seed: int, t: int, U: np.ndarray, walker_at: np.ndarray) -> np.ndarray:
    """The oracle's PT pass on the same counts (A = -2 u_s, B = -2 u_t up to
    constants that cancel in the differences)."""
    wa = walker_at.astype(np.int32).copy()
    for a in range(U.shape[0]):
        row = np.ascontiguousarray(wa[a])
        oracle.pt_only(a, seed, k, kt, t, row, -2 * U[a, :, :, 0], -2 * U[a, :, :, 1])
        wa[a] = row
    return wa
