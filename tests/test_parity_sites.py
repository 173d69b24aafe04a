"""GPU parity of the SITES packing (the paper's multi-site coding with its
daemon-bit rule, Sec. 2.1.1 and Appendices B-C) against the CPU oracle,
through the C ABI: the host tables, full runs bit for bit, resume, and at the
paper's lattice shape one sweep of sampled systems."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from tests.gpu_util import assert_same_state, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qisg():
    need_gpu()
    from paper_2402_03920_gb300 import qisg as q
    q.load()
    return q


def _ladder(lo, hi, n):
    k = np.array([lo] if n == 1 else [lo + (hi - lo) * s / (n - 1) for s in range(n)], dtype=np.float64)
    return np.stack([k, k], axis=1)


def _make(qisg, L, Lt, ladder, n_rep, n_samples, seed, **kw):
    cfg = qisg.Config(L, Lt, ladder, n_rep, n_samples, seed, layout=qisg.QISG_LAYOUT_SITES, **kw)
    return qisg.Instance(cfg)


def _state(ladder, L, Lt, n_rep, seed, n_a, tau_ap=False):
    return oracle.new_state(L, Lt, ladder[:, 0], ladder[:, 1], n_rep, seed, a_lo=0, n_a=n_a,
                            tau_ap=tau_ap, daemon=True)


def _oracle_overlaps(st):
    q = np.zeros((st.n_a, st.n_slots, st.n_rep * (st.n_rep - 1) // 2), dtype=np.int64)
    for a in range(st.n_a):
        for s in range(st.n_slots):
            p = 0
            for r1 in range(st.n_rep):
                for r2 in range(r1 + 1, st.n_rep):
                    S1 = st.S[a, r1, st.walker_at[a, r1, s]].astype(np.int64)
                    S2 = st.S[a, r2, st.walker_at[a, r2, s]].astype(np.int64)
                    q[a, s, p] = int((S1 * S2).sum())
                    p += 1
    return q


def _nstar_lut(cum, lut, bits, R):
    e = int(lut[R >> (64 - bits)])
    n, span = e & 0xFF, e >> 8
    return n + sum(1 for q in range(n, n + span) if R >= int(cum[q]))


def test_daemon_tables_match_oracle(qisg):
    """The library's cumulative tables equal the oracle's (decimal
    arithmetic) bit for bit, and its prefix index gives the oracle's n* at
    every cut point, next to it, at cell edges and at random words."""
    rng = np.random.default_rng(4)
    ks = [0.0, 1e-3, 0.2, 0.29, 0.3125, 0.5, 1.0, 3.0, 16.0] + list(rng.uniform(0.05, 1.5, size=12))
    for k in ks:
        cum, lut = qisg.daemon_tables(k, 12)
        ref = oracle.daemon_cumulative(k)
        assert np.array_equal(cum, ref), k
    for k in (0.29, 0.5, 2.0):
        cum, lut = qisg.daemon_tables(k, 12)
        words = [0, 2 ** 64 - 1] + [int(v) for v in cum] + [max(int(v) - 1, 0) for v in cum]
        words += [h << 52 for h in range(0, 4096, 7)] + [((h + 1) << 52) - 1 for h in range(0, 4096, 7)]
        words += [int.from_bytes(rng.bytes(8), "little") for _ in range(3000)]
        for R in words:
            assert _nstar_lut(cum, lut, 12, R) == oracle.daemon_nstar(cum, R), (k, R)


@pytest.mark.parametrize("L,Lt,n_slots,n_rep,n_samples,pt_every,measure_every,tau_ap,graphs", [
    (4, 64, 4, 2, 1, 1, 0, 0, 1),
    (6, 128, 3, 3, 2, 1, 5, 0, 1),
    (4, 64, 8, 4, 3, 2, 3, 1, 1),      # antiperiodic, PT every 2nd sweep
    (2, 64, 2, 2, 1, 1, 2, 0, 0),      # L = 2 (double bonds), no graphs
    (8, 192, 5, 2, 2, 1, 0, 1, 1),     # M = 6
    (12, 320, 2, 2, 1, 1, 4, 0, 1),    # 720 colour words: several blocks, ragged tail
])
def test_sites_bit_exact(qisg, L, Lt, n_slots, n_rep, n_samples, pt_every, measure_every, tau_ap, graphs):
    ladder = _ladder(0.2, 0.5, n_slots)
    seed = 11 + L + Lt
    inst = _make(qisg, L, Lt, ladder, n_rep, n_samples, seed, pt_every=pt_every,
                 measure_every=measure_every, tau_antiperiodic=tau_ap)
    st = _state(ladder, L, Lt, n_rep, seed, n_samples, tau_ap=bool(tau_ap))
    with inst:
        inst.set_graphs(bool(graphs))
        assert inst.layout() == (qisg.QISG_LAYOUT_SITES, 32)
        assert_same_state(inst, st, what="start")
        for n in (1, 3, 8):
            inst.sweep(n)
            oracle.run(st, n, pt_every=pt_every, measure_every=measure_every)
            assert_same_state(inst, st, what=f"after {st.t} sweeps")
        if measure_every:
            sA, sB, sq, sq2, nm = inst.measurements()
            assert nm == st.n_meas
            assert np.array_equal(sA, st.sumA) and np.array_equal(sB, st.sumB)
            assert np.array_equal(sq, st.sumq) and np.array_equal(sq2, st.sumq2)
        if n_rep > 1:
            assert np.array_equal(inst.overlaps(), _oracle_overlaps(st))


@pytest.mark.parametrize("n_slots,n_rep", [(1, 1), (32, 1), (2, 3)])
def test_sites_edge_cases(qisg, n_slots, n_rep):
    """One slot and one replica (no PT pairs, no overlaps), the longest
    ladder, and an odd replica count."""
    ladder = _ladder(0.1, 0.6, n_slots)
    inst = _make(qisg, 4, 64, ladder, n_rep, 2, 5, measure_every=2)
    st = _state(ladder, 4, 64, n_rep, 5, 2)
    with inst:
        for n in (1, 4):
            inst.sweep(n)
            oracle.run(st, n, pt_every=1, measure_every=2)
            assert_same_state(inst, st, what=f"after {st.t}")


def test_sites_resume_from_state(qisg):
    """qisg_set_state with an oracle state (spins, permutation, sweep count)
    continues on the oracle's trajectory."""
    ladder = _ladder(0.25, 0.45, 4)
    st = _state(ladder, 4, 64, 2, 9, 2)
    oracle.run(st, 5)
    inst = _make(qisg, 4, 64, ladder, 2, 2, 9)
    with inst:
        inst.set_state(st.S, st.walker_at, st.t)
        assert_same_state(inst, st, what="resumed")
        inst.sweep(6)
        oracle.run(st, 6)
        assert_same_state(inst, st, what="after resume")


def test_sites_rejects_what_the_rule_cannot_run(qisg):
    lad = qisg.ladder_linear(0.2, 0.5, 4, 1.0)      # k_tau != k
    with pytest.raises(qisg.QisgError):
        _make(qisg, 4, 64, lad, 1, 1, 1)
    with pytest.raises(qisg.QisgError):             # L_tau not a multiple of 64
        _make(qisg, 4, 96, _ladder(0.2, 0.5, 4), 1, 1, 1)
    with pytest.raises(qisg.QisgError):             # 64-bit words
        _make(qisg, 4, 64, _ladder(0.2, 0.5, 4), 1, 1, 1, word_bits=64)


@pytest.mark.parametrize("L,Lt,n_samples,n_rep,n_slots", [(16, 8192, 16, 4, 16), (24, 2048, 16, 4, 16)])
def test_sites_paper_shape_sampled_systems(qisg, L, Lt, n_samples, n_rep, n_slots):
    """The paper's lattice shapes in the configuration and launch shape the
    benchmark times (16 samples x 4 replicas x 16 slots): after 3 sweeps
    without PT, sweep 3 of two systems of one sampled disorder sample is
    redone by the oracle from the device state and compared bit for bit; the
    device energies of that sample's 64 systems equal the oracle's recount."""
    ladder = _ladder(0.2, 0.5, n_slots)
    seed = 17
    a = 9
    inst = _make(qisg, L, Lt, ladder, n_rep, n_samples, seed, pt_every=0)
    cum = oracle.daemon_tables(ladder[:, 0])
    with inst:
        inst.sweep(3)
        S3 = inst.spins(a, 1)
        J = inst.couplings(a, 1)
        inst.sweep(1)
        S4 = inst.spins(a, 1)
        A, B = inst.energies()
    J = J.reshape(1, L * L, 2)
    for (r, w) in ((0, 0), (n_rep - 1, n_slots - 1)):
        S = np.ascontiguousarray(S3[0, r, w])
        oracle.daemon_sweep_system(L, Lt, seed, a, r, w, 3, J[0], S, cum)   # no PT: walker w at slot w
        assert np.array_equal(S, S4[0, r, w]), (r, w)
    Ao, Bo = oracle.energies(L, Lt, J, S4)
    assert np.array_equal(A[a:a + 1], Ao) and np.array_equal(B[a:a + 1], Bo)
