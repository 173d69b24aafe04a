"""Pins of the oracle's imaginary-time observables (Appendix E.1): the sums
over tau_1 of Q~(tau_1, tau), its square and fourth power, and of the two
squared Fourier moduli of q~_x(tau_1, tau) = S_{x,tau_1} S_{x,tau_1+tau}.

Checked against what fixes them independently of the oracle's loops: the
closed forms at tau = 0, numpy's FFT (the circular autocorrelation along tau
gives sum_tau1 Q~; a 2-D FFT of q~ at the wave vectors (1, 0) and (0, 1)
gives the Fourier moduli), and exact symmetries (tau -> L_tau - tau, a global
spin flip, a shift of the configuration along tau)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle


def _random_config(L, Lt, n_rep, n_slots, seed):
    rng = np.random.default_rng(seed)
    # correlated along tau so that the lags matter: flip each spin with p = 0.2 per step
    S = np.empty((1, n_rep, n_slots, Lt, L, L), dtype=np.int8)
    S[..., 0, :, :] = np.where(rng.random((1, n_rep, n_slots, L, L)) < 0.5, 1, -1)
    for t in range(1, Lt):
        flip = rng.random((1, n_rep, n_slots, L, L)) < 0.2
        S[..., t, :, :] = np.where(flip, -S[..., t - 1, :, :], S[..., t - 1, :, :])
    wa = np.stack([rng.permutation(n_slots) for _ in range(n_rep)])[None].astype(np.int32)
    # site index x1 + L x2 + L^2 tau: [tau][x2][x1]
    return S.reshape(1, n_rep, n_slots, Lt * L * L), wa


@pytest.mark.parametrize("L,Lt", [(4, 8), (6, 12), (5, 7)])
def test_tau_observables_against_fft_and_closed_forms(L, Lt):
    S, wa = _random_config(L, Lt, 2, 3, seed=L * Lt)
    S1, S2, S4, SF = oracle.tau_observables(L, Lt, S, wa)
    conf = S.reshape(1, 2, 3, Lt, L, L).astype(np.float64)   # by walker: [a][r][w][tau][x2][x1]
    for r in range(2):
        for s in range(3):
            c = conf[0, r, wa[0, r, s]]
            # tau = 0: q~ = 1 everywhere
            assert S1[0, r, s, 0] == Lt * L * L and S2[0, r, s, 0] == Lt * L ** 4
            assert S4[0, r, s, 0] == Lt * L ** 8 and abs(SF[0, r, s, 0]) < 1e-20
            # sum over tau_1 of Q~: circular autocorrelation along tau, by FFT, summed over sites
            f = np.fft.fft(c, axis=0)
            auto = np.real(np.fft.ifft(np.conj(f) * f, axis=0)).sum(axis=(1, 2))
            assert np.array_equal(S1[0, r, s], np.rint(auto).astype(np.int64))
            # Fourier moduli of q~ by 2-D FFT, and Q~ powers, for every (tau_1, tau)
            for tau in range(Lt):
                q = c * np.roll(c, -tau, axis=0)                 # q~[tau_1][x2][x1]
                F2 = np.fft.fft2(q, axes=(1, 2))                 # [tau_1][k2][k1]
                mod = np.abs(F2[:, 0, 1]) ** 2 + np.abs(F2[:, 1, 0]) ** 2
                assert SF[0, r, s, tau] == pytest.approx(mod.sum(), rel=1e-12, abs=1e-9)
                Q = np.rint(F2[:, 0, 0].real).astype(np.int64)
                assert S2[0, r, s, tau] == (Q ** 2).sum() and S4[0, r, s, tau] == (Q ** 4).sum()
    # symmetries: tau -> L_tau - tau, a global flip, a shift along tau
    rev = np.concatenate([S1[..., :1], S1[..., :0:-1]], axis=-1)
    assert np.array_equal(S1, rev)
    assert np.allclose(SF, np.concatenate([SF[..., :1], SF[..., :0:-1]], axis=-1), rtol=1e-12, atol=1e-9)
    flipped = oracle.tau_observables(L, Lt, -S, wa)
    for x, y in zip((S1, S2, S4), flipped[:3]):
        assert np.array_equal(x, y)
    shifted = np.roll(S.reshape(1, 2, 3, Lt, L * L), 3, axis=3).reshape(S.shape)
    sh = oracle.tau_observables(L, Lt, np.ascontiguousarray(shifted), wa)
    for x, y in zip((S1, S2, S4), sh[:3]):
        assert np.array_equal(x, y)
    assert np.allclose(SF, sh[3], rtol=1e-12, atol=1e-9)
