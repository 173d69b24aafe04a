"""The persistent form of the batched sweep (one cooperative launch per run
of sweeps: red | barrier | blue | barrier | PT | barrier, replayed from a
CUDA graph) against the per-pass launches and the oracle."""
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


@pytest.mark.parametrize("tiles,me,ap,graphs", [((1, 4), 3, 0, True), ((2, 8), 0, 1, True), ((4, 2), 4, 0, False),
                                                ((2, 32), 5, 1, True), ((1, 1), 2, 0, True)])
def test_persistent_equals_oracle(qisg, tiles, me, ap, graphs):
    L, Lt, n_slots, n_rep, n_a, seed = 6, 16, 7, 5, 40, 19
    inst, ladder = make(qisg, L, Lt, 0.2, 0.5, n_slots, 0.9, n_rep, n_a, seed, word_bits=32,
                        layout=qisg.QISG_LAYOUT_SAMPLES, measure_every=me, tau_antiperiodic=ap)
    st = oracle_state(ladder, L, Lt, n_rep, seed, 0, n_a, tau_ap=bool(ap))
    with inst:
        inst.set_persistent(True)
        inst.set_graphs(graphs)
        inst.set_tiles(tiles, (0, 0))
        for n in (1, 6, 23, 70):
            inst.sweep(n)
            oracle.run(st, n, pt_every=1, measure_every=me)
            assert_same_state(inst, st, what=f"tiles={tiles} me={me} after {st.t}")
        sA, sB, sq, sq2, nm = inst.measurements()
        assert nm == st.n_meas
        assert np.array_equal(sA, st.sumA) and np.array_equal(sq2, st.sumq2)


@pytest.mark.parametrize("tiles", [(1, 5), (2, 0), (4, 3)])
def test_persistent_uneven_walks_equal_oracle(qisg, tiles):
    """The persistent form at L = 16 (a block per segment of 128 columns)
    with L_tau / 2 = 13 sites per column and colour: walks of at most 5 or 3
    sites give segments of unequal length (5,4,4 and 3,3,3,2,2), 0 the
    default segmentation for the persistent grid."""
    L, Lt, n_slots, n_rep, n_a, seed = 16, 26, 5, 4, 36, 29
    inst, ladder = make(qisg, L, Lt, 0.2, 0.5, n_slots, 0.9, n_rep, n_a, seed, word_bits=32,
                        layout=qisg.QISG_LAYOUT_SAMPLES, measure_every=3)
    st = oracle_state(ladder, L, Lt, n_rep, seed, 0, n_a)
    with inst:
        inst.set_persistent(True)
        inst.set_tiles(tiles, (0, 0))
        for n in (1, 7, 16):
            inst.sweep(n)
            oracle.run(st, n, pt_every=1, measure_every=3)
            assert_same_state(inst, st, what=f"tiles={tiles} after {st.t}")
        sA, sB, sq, sq2, nm = inst.measurements()
        assert nm == st.n_meas
        assert np.array_equal(sA, st.sumA) and np.array_equal(sq2, st.sumq2)


def test_persistent_autotune_and_switching(qisg):
    """The autotuner's persistent candidates, and switching the form on and
    off mid-run, keep the trajectory of plain launches."""
    kw = dict(layout=qisg.QISG_LAYOUT_SAMPLES, word_bits=32, measure_every=4)
    a, _ = make(qisg, 8, 16, 0.2, 0.5, 10, 1.0, 4, 64, 23, **kw)
    b, _ = make(qisg, 8, 16, 0.2, 0.5, 10, 1.0, 4, 64, 23, **kw)
    with a, b:
        a.set_persistent(True)
        g = a.autotune(1)
        assert g in (0, 1, 2, 4, 8, 16, 32)
        n = a.sweep_count()
        a.sweep(9)
        a.set_persistent(False)
        a.sweep(5)
        a.set_persistent(True)
        a.sweep(12)
        b.sweep(n + 26)
        assert np.array_equal(a.spins(), b.spins())
        assert np.array_equal(a.permutation(), b.permutation())
        for x, y in zip(a.measurements(), b.measurements()):
            assert np.array_equal(np.asarray(x), np.asarray(y))


def test_persistent_refusals_and_timeout(qisg):
    with make(qisg, 4, 8, 0.2, 0.5, 6, 1.0, 4, 40, 3, layout=qisg.QISG_LAYOUT_SAMPLES, word_bits=64)[0] as w64:
        with pytest.raises(qisg.QisgError):
            w64.set_persistent(True)
    with make(qisg, 4, 8, 0.2, 0.5, 6, 1.0, 4, 40, 3, layout=qisg.QISG_LAYOUT_SAMPLES, word_bits=32,
              pt_every=2)[0] as pt2:
        with pytest.raises(qisg.QisgError):
            pt2.set_persistent(True)
    # a barrier wait bounded to 1 ns runs out: the launch ends, the handle reports ETIMEOUT
    inst, _ = make(qisg, 8, 32, 0.2, 0.5, 16, 1.0, 4, 64, 3, layout=qisg.QISG_LAYOUT_SAMPLES, word_bits=32)
    with inst:
        inst.set_persistent(True, wait_ns=1)
        inst.sweep(40)
        with pytest.raises(qisg.QisgError) as e:
            inst.sync()
        assert e.value.code == -4


def test_persistent_full_size_sampled(qisg):
    """The 1024-sample workload (L=24, L_tau=512, 4 replicas x 32 slots) in
    the persistent form with the autotuner's schedule, 20 sweeps: 8 samples
    chosen by a fixed seed replayed by the oracle."""
    from concurrent.futures import ThreadPoolExecutor
    from paper_2402_03920_gb300.workloads import BATCHED as w
    inst, ladder = make(qisg, w.L, w.L_tau, w.k_lo, w.k_hi, w.n_slots, w.gamma, w.n_replicas,
                        w.n_samples, w.seed, word_bits=32, layout=qisg.QISG_LAYOUT_SAMPLES)
    picks = sorted(np.random.default_rng(2024).choice(w.n_samples, size=8, replace=False).tolist())

    def replay(s):
        st = oracle_state(ladder, w.L, w.L_tau, w.n_replicas, w.seed, s, 1)
        return oracle.run(st, 20, n_threads=1)

    with inst:
        inst.set_persistent(True)
        inst.set_tiles((2, 16), (0, 0))
        inst.sweep(20)
        with ThreadPoolExecutor(max_workers=8) as ex:
            states = list(ex.map(replay, picks))
        for s, st in zip(picks, states):
            assert_same_state(inst, st, a_lo=s, what=f"sample {s}")


def test_persistent_production_shape_default_schedule(qisg):
    """The 32-sample L=16, L_tau=256 workload (4 replicas x 16 slots) in the
    persistent form on the default schedule (walks of unequal length filling
    the persistent grid) and with the blue variant bounded to four blocks
    per SM, 20 sweeps with measurements every 10: samples 0 and 17 replayed
    by the oracle, and the whole state equal to the per-pass launches."""
    from concurrent.futures import ThreadPoolExecutor
    from paper_2402_03920_gb300.workloads import PRODUCTION as w
    kw = dict(layout=qisg.QISG_LAYOUT_SAMPLES, word_bits=32, measure_every=w.measure_every)
    a, ladder = make(qisg, w.L, w.L_tau, w.k_lo, w.k_hi, w.n_slots, w.gamma, w.n_replicas, w.n_samples,
                     w.seed, **kw)
    b, _ = make(qisg, w.L, w.L_tau, w.k_lo, w.k_hi, w.n_slots, w.gamma, w.n_replicas, w.n_samples,
                w.seed, **kw)

    def replay(s):
        st = oracle_state(ladder, w.L, w.L_tau, w.n_replicas, w.seed, s, 1)
        return oracle.run(st, 20, measure_every=w.measure_every, n_threads=1)

    with a, b:
        a.set_persistent(True)
        a.sweep(20)
        b.set_tiles((2, 0), (0, 2))
        b.sweep(20)
        with ThreadPoolExecutor(max_workers=2) as ex:
            states = list(ex.map(replay, (0, 17)))
        for s, st in zip((0, 17), states):
            assert_same_state(a, st, a_lo=s, what=f"sample {s}")
        assert np.array_equal(a.spins(), b.spins())
        assert np.array_equal(a.permutation(), b.permutation())
        for x, y in zip(a.measurements(), b.measurements()):
            assert np.array_equal(np.asarray(x), np.asarray(y))
