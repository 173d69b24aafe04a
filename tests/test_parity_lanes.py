"""GPU parity of the LANES packing (one word = the replica x walker systems of
one sample) against the CPU oracle, through the C ABI."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from tests.gpu_util import assert_same_state, make, need_gpu, oracle_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qisg():
    need_gpu()
    from paper_2402_03920_gb300 import qisg as q
    q.load()
    return q


def test_device_philox_matches_oracle(qisg):
    torch = need_gpu()
    rng = np.random.default_rng(1)
    n = 4096
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    ctr[:4] = 0
    ctr[4:8] = 0xFFFFFFFF
    key[:8:2] = 0
    c_d = torch.from_numpy(ctr.view(np.int32)).cuda()
    k_d = torch.from_numpy(key.view(np.int32)).cuda()
    o_d = torch.zeros((n, 4), dtype=torch.int32, device="cuda")
    qisg.philox4x32_10_device(c_d.data_ptr(), k_d.data_ptr(), o_d.data_ptr(), n,
                              torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    out = o_d.cpu().numpy().view(np.uint32)
    for i in list(range(0, n, 37)) + [0, 4, n - 1]:
        assert list(out[i]) == list(oracle.philox4x32_10(ctr[i], key[i])), i


def test_threshold_table_matches_oracle(qisg):
    inst, ladder = make(qisg, 4, 4, 0.2, 0.5, 32, 0.8, 2, 1, 3, layout=qisg.QISG_LAYOUT_LANES)
    with inst:
        T = inst.thresholds()
    assert np.array_equal(T, oracle.thresholds(ladder[:, 0], ladder[:, 1]))


def test_plain_small_full_run_bit_exact(qisg):
    """L=8, L_tau=32, one sample, 4 replicas x 8 slots (32 systems per
    uint32), 1000 sweeps with PT every sweep; compared after 1, 2, 10, 100
    and 1000 sweeps so that a mismatch points at the first bad sweep."""
    inst, ladder = make(qisg, 8, 32, 0.25, 0.45, 8, 1.0, 4, 1, 1, word_bits=32,
                        layout=qisg.QISG_LAYOUT_LANES, measure_every=10)
    st = oracle_state(ladder, 8, 32, 4, 1)
    with inst:
        assert inst.layout() == (qisg.QISG_LAYOUT_LANES, 32)
        assert_same_state(inst, st, what="start")
        done = 0
        for upto in (1, 2, 10, 100, 1000):
            inst.sweep(upto - done)
            oracle.run(st, upto - done, pt_every=1, measure_every=10)
            done = upto
            assert_same_state(inst, st, what=f"after {upto} sweeps")
        sA, sB, sq, sq2, nm = inst.measurements()
        assert nm == st.n_meas == 100
        assert np.array_equal(sA, st.sumA) and np.array_equal(sB, st.sumB)
        assert np.array_equal(sq, st.sumq) and np.array_equal(sq2, st.sumq2)
        e_s, e_t, q2 = inst.slot_means()
        o_s, o_t, o_q2 = oracle.slot_means(st)
        np.testing.assert_allclose(e_s, o_s, rtol=1e-12, atol=0)
        np.testing.assert_allclose(e_t, o_t, rtol=1e-12, atol=0)
        np.testing.assert_allclose(q2, o_q2, rtol=1e-12, atol=0)
        q = inst.overlaps()
        assert np.array_equal(q, _oracle_overlaps(st))


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


@pytest.mark.parametrize("L,Lt,n_slots,n_rep,W,n_samples", [
    (2, 4, 4, 4, 32, 1),      # the enumeration lattice: double bonds in x and y
    (4, 8, 5, 3, 32, 2),      # odd slot count, odd replica count, two samples
    (6, 6, 12, 4, 32, 1),     # two word groups (2 replicas per word); 108 sites/colour
    (6, 10, 16, 5, 64, 3),    # 64-bit words, ragged replica group
    (10, 4, 7, 2, 64, 2),
])
def test_small_geometries_bit_exact(qisg, L, Lt, n_slots, n_rep, W, n_samples):
    inst, ladder = make(qisg, L, Lt, 0.2, 0.5, n_slots, 0.9, n_rep, n_samples, 11 + L, word_bits=W,
                        layout=qisg.QISG_LAYOUT_LANES)
    st = oracle_state(ladder, L, Lt, n_rep, 11 + L, 0, n_samples)
    with inst:
        for n in (1, 9, 40):
            inst.sweep(n)
            oracle.run(st, n)
            assert_same_state(inst, st, what=f"L={L} Lt={Lt} after {st.t}")


def test_per_sample_launch_equals_batched_launch(qisg):
    a, ladder = make(qisg, 8, 16, 0.25, 0.45, 8, 1.0, 4, 5, 9, layout=qisg.QISG_LAYOUT_LANES,
                     per_sample_launch=1)
    b, _ = make(qisg, 8, 16, 0.25, 0.45, 8, 1.0, 4, 5, 9, layout=qisg.QISG_LAYOUT_LANES)
    with a, b:
        a.sweep(30)
        b.sweep(30)
        assert np.array_equal(a.spins(), b.spins())
        assert np.array_equal(a.permutation(), b.permutation())
        assert a.launch_count() > b.launch_count()


def test_explicit_pt_matches_fused(qisg):
    a, _ = make(qisg, 6, 8, 0.25, 0.45, 6, 1.0, 4, 2, 4, layout=qisg.QISG_LAYOUT_LANES)
    b, _ = make(qisg, 6, 8, 0.25, 0.45, 6, 1.0, 4, 2, 4, layout=qisg.QISG_LAYOUT_LANES, pt_every=0)
    with a, b:
        with pytest.raises(qisg.QisgError):
            b.pt_swap()   # no sweep yet
        for _ in range(12):
            a.sweep(1)
            b.sweep(1)
            b.pt_swap()
        assert np.array_equal(a.spins(), b.spins())
        assert np.array_equal(a.permutation(), b.permutation())


def test_resume_is_bit_exact(qisg):
    a, ladder = make(qisg, 6, 8, 0.25, 0.45, 6, 1.0, 4, 2, 4, layout=qisg.QISG_LAYOUT_LANES)
    b, _ = make(qisg, 6, 8, 0.25, 0.45, 6, 1.0, 4, 2, 99, layout=qisg.QISG_LAYOUT_LANES)
    with a, b:
        a.sweep(10)
        S, wa, t = a.spins(), a.permutation(), a.sweep_count()
        a.sweep(10)
        # b has other couplings: give it a's, then a's state
        b2, _ = make(qisg, 6, 8, 0.25, 0.45, 6, 1.0, 4, 2, 4, layout=qisg.QISG_LAYOUT_LANES)
        with b2:
            b2.set_state(S, wa, t)
            b2.sweep(10)
            assert np.array_equal(a.spins(), b2.spins())
            assert np.array_equal(a.permutation(), b2.permutation())
            assert np.array_equal(a.energies()[0], b2.energies()[0])


@pytest.mark.parametrize("W,n_slots,n_rep", [(0, 6, 4), (32, 16, 4), (64, 20, 5)])
def test_arbitrary_state_and_couplings_against_oracle(qisg, W, n_slots, n_rep):
    """Random couplings, spins and permutation set through the ABI (packed on
    the device), then run on both sides (the path the gauge and flip
    symmetries exercise); one and two word groups per site."""
    from paper_2402_03920_gb300.workloads import random_permutations, random_spins
    L, Lt, n_a = 6, 8, 2
    inst, ladder = make(qisg, L, Lt, 0.2, 0.5, n_slots, 1.1, n_rep, n_a, 5,
                        layout=qisg.QISG_LAYOUT_LANES, word_bits=W)
    J = random_spins((n_a, L * L, 2), 1)
    S = random_spins((n_a, n_rep, n_slots, L * L * Lt), 2)
    wa = random_permutations(n_a * n_rep, n_slots, 3).reshape(n_a, n_rep, n_slots)
    st = oracle_state(ladder, L, Lt, n_rep, 5, 0, n_a)
    st.J, st.S, st.walker_at, st.t = J.copy(), S.copy(), wa.copy(), 17
    oracle.refresh_energies(st)
    with inst:
        inst.set_couplings(J)
        inst.set_state(S, wa, 17)
        assert np.array_equal(inst.couplings(), J)
        assert_same_state(inst, st, what="after set_state")
        inst.sweep(25)
        oracle.run(st, 25)
        assert_same_state(inst, st, what="arbitrary state")


def test_production_shape_sampled(qisg):
    """The 32-sample L=16, L_tau=256, 16-slot workload in the per-instance
    launch form the benchmark times: all samples on the GPU, samples 0 and 31
    replayed by the oracle for 6 sweeps."""
    from paper_2402_03920_gb300.workloads import PRODUCTION as w
    inst, ladder = make(qisg, w.L, w.L_tau, w.k_lo, w.k_hi, w.n_slots, w.gamma, w.n_replicas,
                        w.n_samples, w.seed, word_bits=64, layout=qisg.QISG_LAYOUT_LANES,
                        per_sample_launch=1, measure_every=w.measure_every)
    with inst:
        inst.sweep(6)
        for a in (0, 31):
            st = oracle_state(ladder, w.L, w.L_tau, w.n_replicas, w.seed, a, 1)
            oracle.run(st, 6, measure_every=w.measure_every)
            assert_same_state(inst, st, a_lo=a, what=f"sample {a}")


@pytest.mark.parametrize("W,per_sample", [(64, 0), (32, 1)])
def test_antiperiodic_tau_bit_exact(qisg, W, per_sample):
    """Antiperiodic boundary along tau in the LANES packing against the oracle."""
    L, Lt, n_slots, n_rep, n_samples = 4, 6, 8, 4 if W == 64 else 2, 3
    inst, ladder = make(qisg, L, Lt, 0.2, 0.5, n_slots, 0.9, n_rep, n_samples, 29, word_bits=W,
                        layout=qisg.QISG_LAYOUT_LANES, measure_every=3, per_sample_launch=per_sample,
                        tau_antiperiodic=1)
    st = oracle_state(ladder, L, Lt, n_rep, 29, 0, n_samples, tau_ap=True)
    with inst:
        assert_same_state(inst, st, what="start")
        for n in (1, 5, 12):
            inst.sweep(n)
            oracle.run(st, n, pt_every=1, measure_every=3)
            assert_same_state(inst, st, what=f"W={W} after {st.t}")
        sA, sB, sq, sq2, nm = inst.measurements()
        assert nm == st.n_meas
        assert np.array_equal(sA, st.sumA) and np.array_equal(sB, st.sumB)


@pytest.mark.parametrize("W,L,Lt,n_slots,n_rep,pt_every,measure_every", [
    (32, 4, 4, 1, 1, 1, 2),      # one slot, one replica
    (64, 4, 2, 8, 8, 1, 3),      # L_tau = 2, a full 64-lane word
    (32, 6, 6, 8, 2, 3, 1),      # PT every 3rd sweep
])
def test_edge_cases_bit_exact(qisg, W, L, Lt, n_slots, n_rep, pt_every, measure_every):
    inst, ladder = make(qisg, L, Lt, 0.2, 0.5, n_slots, 0.9, n_rep, 2, 37 + L, word_bits=W,
                        layout=qisg.QISG_LAYOUT_LANES, pt_every=pt_every, measure_every=measure_every)
    st = oracle_state(ladder, L, Lt, n_rep, 37 + L, 0, 2)
    with inst:
        for n in (1, 7, 24):
            inst.sweep(n)
            oracle.run(st, n, pt_every=pt_every, measure_every=measure_every)
            assert_same_state(inst, st, what=f"after {st.t}")
        sA, sB, sq, sq2, nm = inst.measurements()
        assert nm == st.n_meas
        assert np.array_equal(sA, st.sumA) and np.array_equal(sB, st.sumB)
