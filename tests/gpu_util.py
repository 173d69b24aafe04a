"""Helpers shared by the GPU tests: run the library and the oracle on the same
seeded inputs and compare element by element."""
from __future__ import annotations

import numpy as np
import pytest

import oracle


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def make(qisg, L, Lt, lo, hi, n_slots, gamma, n_rep, n_samples, seed, **kw):
    ladder = qisg.ladder_linear(lo, hi, n_slots, gamma)
    cfg = qisg.Config(L, Lt, ladder, n_rep, n_samples, seed, **kw)
    return qisg.Instance(cfg), ladder


def oracle_state(ladder, L, Lt, n_rep, seed, a_lo=0, n_a=1, tau_ap=False):
    return oracle.new_state(L, Lt, ladder[:, 0], ladder[:, 1], n_rep, seed, a_lo=a_lo, n_a=n_a,
                            tau_ap=tau_ap)


def assert_same_state(inst, st, a_lo=0, what=""):
    n_a = st.n_a
    S = inst.spins(a_lo, n_a)
    wa = inst.permutation()[a_lo:a_lo + n_a]
    A, B = inst.energies()
    assert np.array_equal(wa, st.walker_at), f"{what}: permutation differs"
    if not np.array_equal(S, st.S):
        bad = np.argwhere(S != st.S)
        raise AssertionError(f"{what}: spins differ at {len(bad)} places, first {bad[:5].tolist()}")
    assert np.array_equal(A[a_lo:a_lo + n_a], st.A), f"{what}: A differs"
    assert np.array_equal(B[a_lo:a_lo + n_a], st.B), f"{what}: B differs"
