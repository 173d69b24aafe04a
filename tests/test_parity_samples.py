"""GPU parity of the SAMPLES packing (one word = 32 or 64 samples at one
replica x slot, shared draw) against the CPU oracle and against the LANES
packing, through the C ABI."""
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


@pytest.mark.parametrize("L,Lt,n_slots,n_rep,W,n_samples", [
    (4, 8, 8, 4, 32, 32),      # one full 32-sample word
    (2, 4, 4, 4, 32, 5),       # the enumeration lattice, mostly padding lanes
    (6, 6, 5, 3, 64, 70),      # two 64-sample words, the second ragged; padded replica
    (4, 10, 9, 5, 32, 40),     # two replica groups (5 = 4 + 1)
    (8, 4, 16, 2, 64, 64),
])
def test_small_geometries_bit_exact(qisg, L, Lt, n_slots, n_rep, W, n_samples):
    inst, ladder = make(qisg, L, Lt, 0.2, 0.5, n_slots, 0.9, n_rep, n_samples, 3 + L, word_bits=W,
                        layout=qisg.QISG_LAYOUT_SAMPLES, measure_every=4)
    st = oracle_state(ladder, L, Lt, n_rep, 3 + L, 0, n_samples)
    with inst:
        assert inst.layout() == (qisg.QISG_LAYOUT_SAMPLES, W)
        assert_same_state(inst, st, what="start")
        for n in (1, 3, 28):
            inst.sweep(n)
            oracle.run(st, n, pt_every=1, measure_every=4)
            assert_same_state(inst, st, what=f"L={L} Lt={Lt} W={W} after {st.t}")
        sA, sB, sq, sq2, nm = inst.measurements()
        assert nm == st.n_meas
        assert np.array_equal(sA, st.sumA) and np.array_equal(sB, st.sumB)
        if n_rep > 1:
            assert np.array_equal(sq, st.sumq) and np.array_equal(sq2, st.sumq2)


def test_samples_equals_lanes(qisg):
    """Two packings, one trajectory: the result does not depend on how the
    systems are packed into words."""
    kw = dict(measure_every=5)
    a, _ = make(qisg, 8, 16, 0.2, 0.5, 16, 1.0, 4, 33, 12, layout=qisg.QISG_LAYOUT_SAMPLES,
                word_bits=64, **kw)
    b, _ = make(qisg, 8, 16, 0.2, 0.5, 16, 1.0, 4, 33, 12, layout=qisg.QISG_LAYOUT_LANES,
                word_bits=64, **kw)
    with a, b:
        a.sweep(40)
        b.sweep(40)
        assert np.array_equal(a.permutation(), b.permutation())
        assert np.array_equal(a.spins(), b.spins())
        for x, y in zip(a.energies(), b.energies()):
            assert np.array_equal(x, y)
        ma, mb = a.measurements(), b.measurements()
        for x, y in zip(ma, mb):
            assert np.array_equal(np.asarray(x), np.asarray(y))
        assert np.array_equal(a.overlaps(), b.overlaps())


def test_explicit_pt_and_resume(qisg):
    a, _ = make(qisg, 6, 8, 0.25, 0.45, 6, 1.0, 4, 40, 4, layout=qisg.QISG_LAYOUT_SAMPLES)
    b, _ = make(qisg, 6, 8, 0.25, 0.45, 6, 1.0, 4, 40, 4, layout=qisg.QISG_LAYOUT_SAMPLES, pt_every=0)
    with a, b:
        for _ in range(8):
            a.sweep(1)
            b.sweep(1)
            b.pt_swap()
        assert np.array_equal(a.spins(), b.spins())
        assert np.array_equal(a.permutation(), b.permutation())
        S, wa, t = a.spins(), a.permutation(), a.sweep_count()
        a.sweep(7)
        c, _ = make(qisg, 6, 8, 0.25, 0.45, 6, 1.0, 4, 40, 4, layout=qisg.QISG_LAYOUT_SAMPLES)
        with c:
            c.set_state(S, wa, t)
            c.sweep(7)
            assert np.array_equal(a.spins(), c.spins())
            assert np.array_equal(a.permutation(), c.permutation())


@pytest.mark.parametrize("W,n_rep,n_a", [(32, 4, 36), (64, 3, 70), (32, 5, 33)])
def test_arbitrary_state_against_oracle(qisg, W, n_rep, n_a):
    """Random couplings, spins and permutation through qisg_set_state (packed
    on the device), including a ragged last word group and replica counts
    that leave padding replicas in the last quad."""
    from paper_2402_03920_gb300.workloads import random_permutations, random_spins
    L, Lt, n_slots = 4, 6, 7
    inst, ladder = make(qisg, L, Lt, 0.2, 0.5, n_slots, 1.1, n_rep, n_a, 8,
                        layout=qisg.QISG_LAYOUT_SAMPLES, word_bits=W)
    J = random_spins((n_a, L * L, 2), 4)
    S = random_spins((n_a, n_rep, n_slots, L * L * Lt), 5)
    wa = random_permutations(n_a * n_rep, n_slots, 6).reshape(n_a, n_rep, n_slots)
    st = oracle_state(ladder, L, Lt, n_rep, 8, 0, n_a)
    st.J, st.S, st.walker_at, st.t = J.copy(), S.copy(), wa.copy(), 5
    oracle.refresh_energies(st)
    with inst:
        inst.set_couplings(J)
        inst.set_state(S, wa, 5)
        assert np.array_equal(inst.couplings(), J)
        assert_same_state(inst, st, what="after set_state")
        inst.sweep(12)
        oracle.run(st, 12)
        assert_same_state(inst, st, what="after 12 sweeps")


def test_production_shape_batched_sampled(qisg):
    """32 samples, L=16, L_tau=256, 16 slots, in the batched form the
    benchmark times (SAMPLES, 32-bit words, measurements every 10 sweeps):
    samples 0 and 31 replayed by the oracle after 6 and after 30 sweeps
    (spins, energies, permutation and their measurement sums), and all
    samples against the per-instance LANES form."""
    from concurrent.futures import ThreadPoolExecutor
    from paper_2402_03920_gb300.workloads import PRODUCTION as w
    a, ladder = make(qisg, w.L, w.L_tau, w.k_lo, w.k_hi, w.n_slots, w.gamma, w.n_replicas,
                     w.n_samples, w.seed, layout=qisg.QISG_LAYOUT_SAMPLES,
                     measure_every=w.measure_every)
    b, _ = make(qisg, w.L, w.L_tau, w.k_lo, w.k_hi, w.n_slots, w.gamma, w.n_replicas,
                w.n_samples, w.seed, word_bits=64, layout=qisg.QISG_LAYOUT_LANES,
                per_sample_launch=1, measure_every=w.measure_every)
    states = {s: oracle_state(ladder, w.L, w.L_tau, w.n_replicas, w.seed, s, 1) for s in (0, 31)}

    def advance(item, n):
        return oracle.run(item, n, measure_every=w.measure_every, n_threads=1)

    with a, b:
        assert a.layout() == (qisg.QISG_LAYOUT_SAMPLES, 32)
        for n in (6, 24):
            a.sweep(n)
            with ThreadPoolExecutor(max_workers=2) as ex:
                list(ex.map(lambda st: advance(st, n), states.values()))
            sA, sB, sq, sq2, nm = a.measurements()
            for s, st in states.items():
                assert_same_state(a, st, a_lo=s, what=f"sample {s} after {st.t}")
                assert nm == st.n_meas
                assert np.array_equal(sA[s], st.sumA[0]) and np.array_equal(sB[s], st.sumB[0])
                assert np.array_equal(sq[s], st.sumq[0]) and np.array_equal(sq2[s], st.sumq2[0])
        b.sweep(30)
        assert np.array_equal(a.permutation(), b.permutation())
        assert np.array_equal(a.energies()[0], b.energies()[0])
        assert np.array_equal(a.energies()[1], b.energies()[1])
        ma, mb = a.measurements(), b.measurements()
        for x, y in zip(ma, mb):
            assert np.array_equal(np.asarray(x), np.asarray(y))


def test_batched_full_size_sampled(qisg):
    """1024 samples x 4 replicas x 32 slots, L=24, L_tau=512 (4.8 GB of
    packed spins), in the launch form the benchmark times: 8 samples chosen
    by a fixed seed are replayed by the oracle for the benchmark's 20
    sweeps."""
    from paper_2402_03920_gb300.workloads import BATCHED as w
    inst, ladder = make(qisg, w.L, w.L_tau, w.k_lo, w.k_hi, w.n_slots, w.gamma, w.n_replicas,
                        w.n_samples, w.seed, word_bits=64, layout=qisg.QISG_LAYOUT_SAMPLES)
    picks = sorted(np.random.default_rng(2024).choice(w.n_samples, size=8, replace=False).tolist())
    from concurrent.futures import ThreadPoolExecutor

    def replay(s):
        st = oracle_state(ladder, w.L, w.L_tau, w.n_replicas, w.seed, s, 1)
        return oracle.run(st, 20, n_threads=1)

    with inst:
        inst.sweep(20)
        with ThreadPoolExecutor(max_workers=8) as ex:
            states = list(ex.map(replay, picks))
        for s, st in zip(picks, states):
            assert_same_state(inst, st, a_lo=s, what=f"sample {s}")


@pytest.mark.parametrize("layout", ["LANES", "SAMPLES"])
def test_extreme_ladder_exact_paths(qisg, layout):
    """A ladder from k = 0.05 to k = 12 with k_tau from Gamma = 0.3: the PT
    exponents reach |m dk| > 700 (the exact power chain, with overflow and
    underflow) and the Metropolis table holds zero thresholds (flips that
    are never accepted)."""
    import numpy as np
    lay = qisg.QISG_LAYOUT_LANES if layout == "LANES" else qisg.QISG_LAYOUT_SAMPLES
    ladder = qisg.ladder_linear(0.05, 12.0, 6, 0.3)
    T = oracle.thresholds(ladder[:, 0], ladder[:, 1])
    assert (T == 0).any()
    n_a = 1 if layout == "LANES" else 33
    cfg = qisg.Config(6, 8, ladder, 4, n_a, 77, layout=lay, measure_every=3)
    st = oracle_state(ladder, 6, 8, 4, 77, 0, n_a)
    with qisg.Instance(cfg) as inst:
        for n in (1, 5, 30):
            inst.sweep(n)
            oracle.run(st, n, pt_every=1, measure_every=3)
            assert_same_state(inst, st, what=f"{layout} after {st.t}")
        sA = inst.measurements()[0]
        assert np.array_equal(sA, st.sumA)


def test_graph_replay_equals_direct_launches(qisg):
    """Sweeps replayed from the captured cycle graph (cycle = 5 sweeps here)
    give the trajectory of direct launches, with live kernel timing."""
    import numpy as np
    kw = dict(layout=qisg.QISG_LAYOUT_SAMPLES, measure_every=5, word_bits=32)
    a, _ = make(qisg, 6, 8, 0.2, 0.5, 8, 1.0, 4, 40, 21, **kw)
    b, _ = make(qisg, 6, 8, 0.2, 0.5, 8, 1.0, 4, 40, 21, **kw)
    with a, b:
        b.set_graphs(False)
        a.sweep(3)            # not at a cycle boundary: direct launches
        a.profile(True)
        a.sweep(17)           # 2 replays + ...
        ms, timed, launched = a.profile_read(qisg.KERNEL_SWEEP)
        a.profile(False)
        a.sweep(5)
        b.sweep(25)
        assert launched == 2 * 17 and timed == launched and ms > 0
        assert a.sweep_count() == b.sweep_count() == 25
        assert np.array_equal(a.spins(), b.spins())
        assert np.array_equal(a.permutation(), b.permutation())
        for x, y in zip(a.measurements(), b.measurements()):
            assert np.array_equal(np.asarray(x), np.asarray(y))
        assert a.launch_count() == b.launch_count()


@pytest.mark.parametrize("word_bits,n_cand", [(64, 8), (32, 24)])
def test_autotune_keeps_trajectory(qisg, word_bits, n_cand):
    import numpy as np
    kw = dict(layout=qisg.QISG_LAYOUT_SAMPLES, word_bits=word_bits)
    a, _ = make(qisg, 8, 16, 0.2, 0.5, 8, 1.0, 4, word_bits, 5, **kw)
    b, _ = make(qisg, 8, 16, 0.2, 0.5, 8, 1.0, 4, word_bits, 5, **kw)
    with a, b:
        g = a.autotune(1)
        assert g in (0, 1, 2, 4, 8, 16, 32, 64)
        n = a.sweep_count()
        assert n == n_cand * 2
        a.sweep(6)
        b.sweep(n + 6)
        assert np.array_equal(a.spins(), b.spins())
        assert np.array_equal(a.permutation(), b.permutation())


@pytest.mark.parametrize("W,tiles", [(32, ((1, 4), (0, 0))), (32, ((2, 2), (0, 1))), (32, ((4, 1), (0, 0))),
                                     (32, ((1, 4), (0, 2))), (32, ((2, 1), (0, 2))),
                                     (64, ((0, 0), (0, 0))), (64, ((1, 1), (0, 0)))])
def test_antiperiodic_tau_bit_exact(qisg, W, tiles):
    """Antiperiodic boundary along tau (the wrap tau bond counts -S S): every
    red and blue kernel form against the oracle with the same boundary."""
    L, Lt, n_slots, n_rep, n_samples = 4, 6, 5, 4, W
    inst, ladder = make(qisg, L, Lt, 0.2, 0.5, n_slots, 0.9, n_rep, n_samples, 23, word_bits=W,
                        layout=qisg.QISG_LAYOUT_SAMPLES, measure_every=3, tau_antiperiodic=1)
    st = oracle_state(ladder, L, Lt, n_rep, 23, 0, n_samples, tau_ap=True)
    with inst:
        inst.set_tiles(*tiles)
        assert_same_state(inst, st, what="start")
        for n in (1, 5, 12):
            inst.sweep(n)
            oracle.run(st, n, pt_every=1, measure_every=3)
            assert_same_state(inst, st, what=f"W={W} tiles={tiles} after {st.t}")
        sA, sB, sq, sq2, nm = inst.measurements()
        assert nm == st.n_meas
        assert np.array_equal(sA, st.sumA) and np.array_equal(sB, st.sumB)
        assert np.array_equal(sq, st.sumq) and np.array_equal(sq2, st.sumq2)


@pytest.mark.parametrize("L,variant,tiles", [(16, 0, (1, 2)), (16, 0, (1, 0)), (8, 1, (2, 4)), (16, 2, (1, 1)),
                                             (16, 2, (4, 5)), (16, 2, (0, 64)), (16, 2, (2, 0)), (16, 0, (4, 3)),
                                             (8, 0, (1, 3)), (8, 0, (2, 0))])
def test_blue_variants_bit_exact(qisg, L, variant, tiles):
    """Each 32-bit blue kernel (replica quads, column walk, replica quads with
    bounded registers) and red tile on a lattice of several blocks per
    (sample word, slot) with a ragged second word: the oracle's trajectory.
    L_tau / 2 = 13 sites per column and colour.  At L = 16 (a plane of 256
    columns, a block per segment) walks of at most 2, 3 or 5 sites split a
    column into segments of unequal length (7 x 2 -> 2,2,2,2,2,2,1; 5 x 3 ->
    3,3,3,2,2; 3 x 5 -> 5,4,4), 64 gives one segment, and 0 the default
    segmentation; at L = 8 (64 columns) segments have one length."""
    Lt, n_slots, n_rep, n_samples = 26, 6, 5, 45
    inst, ladder = make(qisg, L, Lt, 0.2, 0.5, n_slots, 0.9, n_rep, n_samples, 71, word_bits=32,
                        layout=qisg.QISG_LAYOUT_SAMPLES, measure_every=2)
    st = oracle_state(ladder, L, Lt, n_rep, 71, 0, n_samples)
    with inst:
        inst.set_tiles(tiles, (0, variant))
        assert inst.tiles() == (tiles, (0, variant))
        for n in (1, 4, 9):
            inst.sweep(n)
            oracle.run(st, n, pt_every=1, measure_every=2)
            assert_same_state(inst, st, what=f"variant={variant} tiles={tiles} after {st.t}")
        sA, sB, sq, sq2, nm = inst.measurements()
        assert nm == st.n_meas
        assert np.array_equal(sA, st.sumA) and np.array_equal(sB, st.sumB)
        assert np.array_equal(sq, st.sumq) and np.array_equal(sq2, st.sumq2)


@pytest.mark.parametrize("W,L,Lt,n_slots,n_rep,n_samples,pt_every,measure_every", [
    (32, 4, 4, 1, 1, 32, 1, 2),      # one slot (no PT pair), one replica (no overlap pair)
    (64, 4, 6, 32, 4, 64, 1, 5),     # the largest ladder (32 slots)
    (32, 4, 2, 6, 4, 32, 1, 3),      # L_tau = 2: both tau bonds join the same pair of sites
    (32, 6, 8, 6, 4, 20, 3, 1),      # PT every 3rd sweep, odd graph cycle (doubled for the two buffers)
    (64, 4, 8, 6, 3, 64, 0, 4),      # no PT at all
    (32, 2, 4, 3, 2, 7, 2, 3),       # the smallest lattice, ragged lanes
])
def test_edge_cases_bit_exact(qisg, W, L, Lt, n_slots, n_rep, n_samples, pt_every, measure_every):
    inst, ladder = make(qisg, L, Lt, 0.2, 0.5, n_slots, 0.9, n_rep, n_samples, 31 + L, word_bits=W,
                        layout=qisg.QISG_LAYOUT_SAMPLES, pt_every=pt_every, measure_every=measure_every)
    st = oracle_state(ladder, L, Lt, n_rep, 31 + L, 0, n_samples)
    with inst:
        inst.sweep(0)                     # a no-op
        assert inst.sweep_count() == 0
        assert_same_state(inst, st, what="start")
        for n in (1, 7, 24):
            inst.sweep(n)
            oracle.run(st, n, pt_every=pt_every, measure_every=measure_every)
            assert_same_state(inst, st, what=f"after {st.t}")
        sA, sB, sq, sq2, nm = inst.measurements()
        assert nm == st.n_meas
        assert np.array_equal(sA, st.sumA) and np.array_equal(sB, st.sumB)
        if n_rep > 1:
            assert np.array_equal(sq, st.sumq) and np.array_equal(sq2, st.sumq2)


@pytest.mark.parametrize("W", [32, 64])
def test_launch_overlap_keeps_trajectory(qisg, W):
    """Programmatic dependent launch on (the default) and off, graphs on and
    off: one trajectory, measurements included, and the oracle's."""
    kw = dict(layout=qisg.QISG_LAYOUT_SAMPLES, word_bits=W, measure_every=3)
    a, ladder = make(qisg, 6, 8, 0.2, 0.5, 9, 1.0, 5, 40, 8, **kw)
    b, _ = make(qisg, 6, 8, 0.2, 0.5, 9, 1.0, 5, 40, 8, **kw)
    st = oracle_state(ladder, 6, 8, 5, 8, 0, 40)
    with a, b:
        a.set_launch_overlap(True)
        b.set_launch_overlap(False)
        a.set_graphs(False)
        for n in (2, 13, 30):
            a.sweep(n)
            b.sweep(n)
            oracle.run(st, n, pt_every=1, measure_every=3)
            assert_same_state(a, st, what=f"overlap on, after {st.t}")
        a.set_graphs(True)
        a.sweep(12)
        b.sweep(12)
        assert np.array_equal(a.spins(), b.spins()) and np.array_equal(a.permutation(), b.permutation())
        for x, y in zip(a.measurements(), b.measurements()):
            assert np.array_equal(np.asarray(x), np.asarray(y))


@pytest.mark.parametrize("variant", [0, 2])
def test_pt_in_blue_pass_equals_pt_launch_and_oracle(qisg, variant):
    """The PT pass run in the blue pass's last blocks (8 samples x 4
    replicas = 32 chains, 8 waiting blocks) against the PT pass of its own
    launch and the oracle, with measurements every 3 sweeps."""
    L, Lt, n_slots, n_rep, n_samples = 16, 32, 6, 4, 8
    kw = dict(word_bits=32, layout=qisg.QISG_LAYOUT_SAMPLES, measure_every=3)
    a, ladder = make(qisg, L, Lt, 0.2, 0.5, n_slots, 0.9, n_rep, n_samples, 41, **kw)
    b, _ = make(qisg, L, Lt, 0.2, 0.5, n_slots, 0.9, n_rep, n_samples, 41, **kw)
    st = oracle_state(ladder, L, Lt, n_rep, 41, 0, n_samples)
    with a, b:
        a.set_tiles((0, 0), (0, variant))
        b.set_tiles((0, 0), (0, variant))
        a.set_pt_in_blue(True)
        b.set_pt_in_blue(False)
        for n in (1, 5, 14):
            a.sweep(n)
            b.sweep(n)
            oracle.run(st, n, pt_every=1, measure_every=3)
            assert_same_state(a, st, what=f"in blue, after {st.t}")
            assert np.array_equal(a.spins(), b.spins())
            assert np.array_equal(a.permutation(), b.permutation())
        for x, y in zip(a.measurements(), b.measurements()):
            assert np.array_equal(np.asarray(x), np.asarray(y))
        assert a.launch_count() < b.launch_count()   # no PT launches in a


def test_pt_in_blue_pass_wait_bound():
    """A 1 ns bound on the waiting blocks: the pass either completes (the
    state equal to the PT launch's) or reports ETIMEOUT; it never hangs."""
    need_gpu()
    from paper_2402_03920_gb300 import qisg
    qisg.load()
    kw = dict(word_bits=32, layout=qisg.QISG_LAYOUT_SAMPLES, measure_every=0)
    a, _ = make(qisg, 16, 64, 0.2, 0.5, 8, 0.9, 4, 8, 43, **kw)
    b, _ = make(qisg, 16, 64, 0.2, 0.5, 8, 0.9, 4, 8, 43, **kw)
    with a, b:
        a.set_pt_in_blue(True, wait_ns=1)
        b.set_pt_in_blue(False)
        b.sweep(20)
        try:
            a.sweep(20)
            a.sync()
        except qisg.QisgError as e:
            assert e.code == -4   # QISG_ETIMEOUT
        else:
            assert np.array_equal(a.spins(), b.spins())
            assert np.array_equal(a.permutation(), b.permutation())


def test_pt_in_blue_pass_with_pt_every_and_graph_off(qisg):
    """PT every 3rd sweep (the blue pass runs the chains only on those
    sweeps), with and without the sweep graph, against the oracle."""
    L, Lt, n_slots, n_rep, n_samples = 16, 16, 5, 4, 6
    kw = dict(word_bits=32, layout=qisg.QISG_LAYOUT_SAMPLES, measure_every=4, pt_every=3)
    a, ladder = make(qisg, L, Lt, 0.2, 0.5, n_slots, 0.9, n_rep, n_samples, 47, **kw)
    b, _ = make(qisg, L, Lt, 0.2, 0.5, n_slots, 0.9, n_rep, n_samples, 47, **kw)
    st = oracle_state(ladder, L, Lt, n_rep, 47, 0, n_samples)
    with a, b:
        a.set_pt_in_blue(True)
        b.set_pt_in_blue(True)
        b.set_graphs(False)
        for n in (2, 7, 13):
            a.sweep(n)
            b.sweep(n)
            oracle.run(st, n, pt_every=3, measure_every=4)
            assert_same_state(a, st, what=f"pt_every=3 after {st.t}")
            assert np.array_equal(a.spins(), b.spins())
            assert np.array_equal(a.permutation(), b.permutation())
        sA, sB, sq, sq2, nm = a.measurements()
        assert nm == st.n_meas
        assert np.array_equal(sA, st.sumA) and np.array_equal(sq2, st.sumq2)
