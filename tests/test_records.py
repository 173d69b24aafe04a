"""Measurement records on the GPU (Appendix A) against the oracle: the PT
walk history (history_betas) and the maxit block sums, in every packing,
through the captured sweep graph, across the wrap of their ring buffers and
after a state reset."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qisg():
    need_gpu()
    from paper_2402_03920_gb300 import qisg as q
    q.load()
    return q


@pytest.mark.parametrize("layout,W,n_samples,ap", [("LANES", 32, 3, 0), ("SAMPLES", 32, 40, 0),
                                                  ("SAMPLES", 64, 70, 1), ("SITES", 32, 2, 0)])
def test_walk_history_and_blocks_match_oracle(qisg, layout, W, n_samples, ap):
    lay = getattr(qisg, f"QISG_LAYOUT_{layout}")
    L, Lt, n_rep, seed, me, maxit = 4, 8, 3, 13, 2, 3
    if layout == "SITES":
        Lt = 64
        ladder = qisg.ladder_equal(0.25, 0.45, 5)
    else:
        ladder = qisg.ladder_linear(0.2, 0.5, 5, 1.0)
    hist_len, blocks_len = 7, 2
    cfg = qisg.Config(L, Lt, ladder, n_rep, n_samples, seed, word_bits=W, layout=lay, measure_every=me,
                      tau_antiperiodic=ap, history_len=hist_len, maxit=maxit, blocks_len=blocks_len)
    st = oracle.new_state(L, Lt, ladder[:, 0], ladder[:, 1], n_rep, seed, n_a=n_samples, tau_ap=bool(ap),
                          daemon=layout == "SITES")
    st.keep_history, st.maxit = True, maxit
    with qisg.Instance(cfg) as inst:
        for n in (4, 14, 12):                        # 2, 9, 15 measurements (the rings wrap)
            inst.sweep(n)
            oracle.run(st, n, pt_every=1, measure_every=me)
            m = st.n_meas
            lo = max(0, m - hist_len)
            assert np.array_equal(inst.walk_history(lo, m - lo), st.hist[lo:m]), (layout, m)
            nb = m // maxit
            blo = max(0, nb - blocks_len + (1 if m % maxit else 0))
            if nb > blo:
                A, B = inst.block_sums(blo, nb - blo)
                assert np.array_equal(A, st.blkA[blo:nb]) and np.array_equal(B, st.blkB[blo:nb]), (layout, m)
                e_s, e_t = inst.block_means(blo, nb - blo)
                N = L * L * Lt
                den = maxit * n_samples * n_rep
                assert np.allclose(e_s, st.blkA[blo:nb].sum(axis=(1, 2)) / (den * 2.0 * N), rtol=1e-12, atol=0)
                assert np.allclose(e_t, st.blkB[blo:nb].sum(axis=(1, 2)) / (den * N), rtol=1e-12, atol=0)
            # entries outside the rings are refused
            with pytest.raises(qisg.QisgError):
                inst.walk_history(m, 1)
            if m > hist_len:
                with pytest.raises(qisg.QisgError):
                    inst.walk_history(lo - 1, 1)
        # a state reset restarts the measurement count
        S, wa, t = inst.spins(), inst.permutation(), inst.sweep_count()
        inst.set_state(S, wa, t)
        inst.sweep(2)
        st.n_meas = 0
        st.hist = None
        st.blkA = st.blkB = None
        st.sumA[...] = 0
        st.sumB[...] = 0
        st.sumq[...] = 0
        st.sumq2[...] = 0
        oracle.run(st, 2, pt_every=1, measure_every=me)
        assert np.array_equal(inst.walk_history(0, 1), st.hist[:1])
