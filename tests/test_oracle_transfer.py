"""Pin of the oracle's transfer-matrix product (Sec. 2.2 Eq. (transfer-
matrix), Appendix D): the butterfly rounds and the parity-aware last factor
are checked against the transfer matrix built densely from its definition in
the computational basis (diagonal e^{-k H0/2}, the product over sites of
jP 1 + jM sigma^X) and projected onto the even and odd sectors with the basis
vectors (|n> +- |n-bar>)/sqrt 2."""
from __future__ import annotations

import numpy as np
import pytest

import oracle


def _dense_sector(L, k, kt, J, parity):
    ns = L * L
    dim = 1 << ns
    states = np.arange(dim, dtype=np.int64)
    spin = 1 - 2 * ((states[:, None] >> np.arange(ns)) & 1)          # S_j = -1 <=> bit j
    E = np.zeros(dim)
    for x2 in range(L):
        for x1 in range(L):
            i = x1 + L * x2
            ix, iy = (x1 + 1) % L + L * x2, x1 + L * ((x2 + 1) % L)
            E += J[i, 0] * spin[:, i] * spin[:, ix] + J[i, 1] * spin[:, i] * spin[:, iy]
    D = np.exp(0.5 * k * E)
    jP, jM = np.exp(kt) / (np.exp(kt) + np.exp(-kt)), np.exp(-kt) / (np.exp(kt) + np.exp(-kt))
    diff = states[:, None] ^ states[None, :]
    n_diff = np.array([bin(int(v)).count("1") for v in range(dim)])[diff]
    M = jP ** (ns - n_diff) * jM ** n_diff                          # prod_j (jP 1 + jM sigma^X_j)
    T = D[:, None] * M * D[None, :]
    half = dim // 2
    B = np.zeros((dim, half))
    for n in range(half):
        B[n, n] = 1 / np.sqrt(2)
        B[dim - 1 - n, n] = parity / np.sqrt(2)
    return B.T @ T @ B


@pytest.mark.parametrize("L,k,kt,parity", [(2, 0.3, 0.7, 1), (2, 0.45, 0.2, -1), (3, 0.29, 0.29, 1),
                                           (3, 0.5, 0.35, -1)])
def test_matvec_against_dense_transfer_matrix(L, k, kt, parity):
    J = oracle.init_couplings(L, 0, 1, 17 + L)[0]
    Ts = _dense_sector(L, k, kt, J, parity)
    rng = np.random.default_rng(3)
    for _ in range(3):
        v = rng.standard_normal(Ts.shape[0])
        assert np.allclose(oracle.transfer_matvec(L, k, kt, J, parity, v), Ts @ v, rtol=1e-12, atol=1e-12)
    # symmetric, and its leading eigenvalue is reached by power iteration with the product
    assert np.allclose(Ts, Ts.T, rtol=1e-12, atol=1e-14)
    lam = np.linalg.eigvalsh(Ts)[-1]
    v = np.ones(Ts.shape[0])
    for _ in range(400):
        v = oracle.transfer_matvec(L, k, kt, J, parity, v)
        v /= np.linalg.norm(v)
    assert v @ oracle.transfer_matvec(L, k, kt, J, parity, v) == pytest.approx(lam, rel=1e-9)
