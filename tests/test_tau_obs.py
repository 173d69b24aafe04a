"""Imaginary-time observables on the GPU (Appendix E.1) against the oracle,
in every packing, on configurations after sweeps with PT (so the slots hold
permuted walkers), for a sub-range of samples and with the antiperiodic
boundary."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from tests.gpu_util import make, need_gpu, oracle_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qisg():
    need_gpu()
    from paper_2402_03920_gb300 import qisg as q
    q.load()
    return q


@pytest.mark.parametrize("layout,W,L,Lt,n_a,ap", [("SAMPLES", 32, 6, 16, 40, 0), ("SAMPLES", 64, 8, 8, 70, 1),
                                                   ("LANES", 32, 4, 10, 3, 0), ("SITES", 32, 4, 64, 2, 0),
                                                   ("SAMPLES", 32, 24, 32, 33, 0)])
def test_tau_observables_match_oracle(qisg, layout, W, L, Lt, n_a, ap):
    lay = getattr(qisg, f"QISG_LAYOUT_{layout}")
    if layout == "SITES":
        ladder = qisg.ladder_equal(0.25, 0.45, 5)
        inst = qisg.Instance(qisg.Config(L, Lt, ladder, 3, n_a, 41, layout=lay))
        st = oracle.new_state(L, Lt, ladder[:, 0], ladder[:, 1], 3, 41, n_a=n_a, daemon=True)
    else:
        inst, ladder = make(qisg, L, Lt, 0.2, 0.5, 5, 1.0, 3, n_a, 41, layout=lay, word_bits=W, tau_antiperiodic=ap)
        st = oracle_state(ladder, L, Lt, 3, 41, 0, n_a, tau_ap=bool(ap))
    with inst:
        inst.sweep(9)
        oracle.run(st, 9)
        got = inst.tau_observables()
        want = oracle.tau_observables(L, Lt, st.S, st.walker_at)
        for name, g, w in zip(("S1", "S2", "S4"), got[:3], want[:3]):
            assert np.array_equal(g, w), name
        assert np.array_equal(got[3], want[3]) or np.allclose(got[3], want[3], rtol=1e-12, atol=0), "SF"
        lo, n = min(1, n_a - 1), min(2, n_a - 1)
        sub = inst.tau_observables(lo, n)
        for g, w in zip(sub, got):
            assert np.array_equal(g, w[lo:lo + n])
