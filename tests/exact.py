"""Exact results for tiny lattices, written from the definitions only.

These are the pins the oracle is checked against; nothing here calls the
oracle or the CUDA library.

* ``enumerate_AB``: brute-force Boltzmann averages of A = sum_spatial J S S
  and B = sum_tau S S over all 2^N configurations of an L x L x L_tau prism
  (periodic), weight exp(k A + k_tau B) -- Eq. (2)-(3) with a separate
  imaginary-time coupling.
* ``transfer_AB``: the same averages for a prism of any L_tau, periodic or
  antiperiodic, by the transfer matrix along tau (L <= 3), checked against
  ``enumerate_AB``.
* ``chain_B``: closed form for k = 0, where every spatial site carries an
  independent Ising ring of L_tau spins with coupling k_tau, periodic or
  antiperiodic (one bond of opposite sign).
"""
from __future__ import annotations

import numpy as np


def _all_configs(n: int) -> np.ndarray:
    idx = np.arange(1 << n, dtype=np.int64)
    bits = (idx[:, None] >> np.arange(n, dtype=np.int64)[None, :]) & 1
    return (1 - 2 * bits).astype(np.int8)       # bit 1 -> spin -1


def AB_of_configs(S: np.ndarray, J: np.ndarray, L: int, Ltau: int, tau_ap: bool = False):
    """A and B of a batch of configurations S[m][N] (site = x + L y + L^2 tau);
    J[L*L][2] with dir 0 = +x, dir 1 = +y.  tau_ap: S_{x,L_tau} = -S_{x,0}."""
    m = S.shape[0]
    V = S.reshape(m, Ltau, L, L).astype(np.int64)            # [m][tau][y][x]
    Jx = J[:, 0].reshape(L, L).astype(np.int64)              # [y][x]
    Jy = J[:, 1].reshape(L, L).astype(np.int64)
    A = (Jx[None, None] * V * np.roll(V, -1, axis=3)).sum(axis=(1, 2, 3))
    A += (Jy[None, None] * V * np.roll(V, -1, axis=2)).sum(axis=(1, 2, 3))
    up = np.roll(V, -1, axis=1)
    if tau_ap:
        up[:, Ltau - 1] = -up[:, Ltau - 1]
    B = (V * up).sum(axis=(1, 2, 3))
    return A, B


def enumerate_AB(J: np.ndarray, L: int, Ltau: int, k: float, ktau: float, tau_ap: bool = False):
    """Exact <A>, <B>, <A^2>, <B^2> at (k, k_tau) by enumeration (N <= 20)."""
    n = L * L * Ltau
    assert n <= 20
    S = _all_configs(n)
    A, B = AB_of_configs(S, J, L, Ltau, tau_ap)
    logw = k * A.astype(np.float64) + ktau * B.astype(np.float64)
    logw -= logw.max()
    w = np.exp(logw)
    Z = w.sum()
    return ((w * A).sum() / Z, (w * B).sum() / Z,
            (w * A * A).sum() / Z, (w * B * B).sum() / Z)


def layer_A(J: np.ndarray, L: int, k: float) -> float:
    """Exact <A_layer> of one 2D +-J layer (k_tau = 0), by enumeration."""
    n = L * L
    S = _all_configs(n)
    A, _ = AB_of_configs(S, J, L, 1)
    # with L_tau = 1 the tau-roll pairs a spin with itself; only A is used
    logw = k * A.astype(np.float64)
    logw -= logw.max()
    w = np.exp(logw)
    return float((w * A).sum() / w.sum())


def chain_B(L: int, Ltau: int, ktau: float, tau_ap: bool = False) -> float:
    """<B> for k = 0: L^2 independent rings of Ltau spins; the transfer
    matrix has eigenvalues 2 cosh K and 2 sinh K, and the bond of opposite
    sign of the antiperiodic ring flips the sign of the second:
    Z = (2 cosh K)^n +- (2 sinh K)^n, <B> = d ln Z / dK (per ring)."""
    n = Ltau
    c, s = np.cosh(ktau), np.sinh(ktau)
    sg = -1.0 if tau_ap else 1.0
    # divide numerator and denominator by (2 cosh K)^n
    t = np.tanh(ktau)
    num = n * (s / c + sg * t ** (n - 1))
    den = 1.0 + sg * t ** n
    return float(L * L * num / den)


def transfer_AB(J: np.ndarray, L: int, Ltau: int, k: float, ktau: float, tau_ap: bool = False):
    """Exact <A>, <B> of an L x L x L_tau prism by the transfer matrix along
    tau (L <= 3): with D = diag(exp(k A_layer)) and C[s, s'] = exp(k_tau
    s.s'), the slice-to-slice matrix is T = D^1/2 C D^1/2 and Z = Tr T^L_tau;
    antiperiodic (tau_ap): the bond L_tau-1 -> 0 has the opposite sign, its
    matrix T~ = D^1/2 C~ D^1/2 with C~[s, s'] = exp(-k_tau s.s'), and
    Z = Tr T^(L_tau - 1) T~.  Flipping every spin of one slice moves that
    twist and leaves A_layer unchanged, so every slice and every tau bond
    contributes alike:
    <A> = L_tau Tr(diag(A_layer) P) / Z with P the closed product, and
    <B> = L_tau Tr(D^1/2 (C o G) D^1/2 T^(L_tau - 2) T~) / Z (T~ = T when
    periodic), G[s, s'] = s.s'."""
    n = L * L
    assert n <= 9 and Ltau >= 2
    S = _all_configs(n).astype(np.float64)                      # [2^n][n]
    A_layer, _ = AB_of_configs(_all_configs(n), J, L, 1)
    A_layer = A_layer.astype(np.float64)
    G = S @ S.T
    d = np.exp(0.5 * k * (A_layer - A_layer.max()))

    def mat(sign):
        return d[:, None] * np.exp(sign * ktau * G) * d[None, :]

    T = mat(1.0)
    Tw = mat(-1.0) if tau_ap else T
    top = np.linalg.eigvalsh(T).max()
    Tn, Twn = T / top, Tw / top
    P = np.linalg.matrix_power(Tn, Ltau - 1) @ Twn
    Z = np.trace(P)
    mA = Ltau * np.trace(A_layer[:, None] * P) / Z
    TB = (d[:, None] * (np.exp(ktau * G) * G) * d[None, :]) / top
    mB = Ltau * np.trace(TB @ np.linalg.matrix_power(Tn, Ltau - 2) @ Twn) / Z
    return float(mA), float(mB)
