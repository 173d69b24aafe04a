"""The batched form (one persistent kernel over instances of uneven size)
against the oracle, per instance, through the C ABI."""
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


def _oracle_instance(L, Lt, ladder, n_rep, seed, sweeps):
    st = oracle.new_state(L, Lt, ladder[:, 0], ladder[:, 1], n_rep, seed)
    oracle.run(st, sweeps)
    return st


def test_uneven_batch_bit_exact(qisg):
    """Six instances of different L, L_tau, ladder length, Gamma and replica
    count (the 4-replica tile and the general one) in one batch: every one
    matches its own oracle run after 1, 4 and 25 sweeps."""
    rng = np.random.default_rng(3)
    specs = []
    for i, n_rep in enumerate((4, 1, 3, 2, 4, 3)):
        L = int(rng.choice([2, 4, 6, 8]))
        Lt = int(rng.choice([4, 8, 16]))
        n_slots = int(rng.integers(3, 33))
        gamma = float(rng.uniform(0.8, 1.2))
        specs.append((L, Lt, qisg.ladder_linear(0.2, 0.5, n_slots, gamma), n_rep, 100 + i))
    with qisg.Batch(8, 64 << 20) as b:
        slots = [b.admit(L, Lt, lad, nr, seed) for (L, Lt, lad, nr, seed) in specs]
        done = 0
        for upto in (1, 4, 25):
            b.run(upto - done)
            done = upto
            for slot, (L, Lt, lad, nr, seed) in zip(slots, specs):
                st = _oracle_instance(L, Lt, lad, nr, seed, upto)
                A, B, wa, S = b.results(slot, spins=True)
                assert np.array_equal(wa, st.walker_at[0]), (slot, upto)
                assert np.array_equal(S, st.S[0]), (slot, upto)
                assert np.array_equal(A, st.A[0]) and np.array_equal(B, st.B[0])
                assert b.status(slot)[0] == upto


def test_targets_admission_and_retire(qisg):
    """Instances stop at their sweep target; retiring frees memory that a
    queued instance then gets; a late instance runs from its own start."""
    lad = qisg.ladder_linear(0.25, 0.45, 8, 1.0)
    need = qisg.Batch.instance_bytes(6, 8, lad, 4)
    assert need > 0
    with qisg.Batch(4, 2 * need + 512) as b:
        s0 = b.admit(6, 8, lad, 4, 11, n_sweeps=5)
        s1 = b.admit(6, 8, lad, 4, 12, n_sweeps=0)
        assert b.try_admit(6, 8, lad, 4, 13) is None      # arena full
        b.run(9)
        assert b.status(s0) == (5, True)
        assert b.status(s1) == (9, False)
        st0 = _oracle_instance(6, 8, lad, 4, 11, 5)
        assert np.array_equal(b.results(s0, spins=True)[3], st0.S[0])
        b.retire(s0)
        s2 = b.admit(6, 8, lad, 4, 13, n_sweeps=3)
        b.run(4)
        assert b.status(s2) == (3, True)
        st1 = _oracle_instance(6, 8, lad, 4, 12, 13)
        st2 = _oracle_instance(6, 8, lad, 4, 13, 3)
        assert np.array_equal(b.results(s1, spins=True)[3], st1.S[0])
        assert np.array_equal(b.results(s2, spins=True)[3], st2.S[0])


def test_batch_equals_handles_and_schedule_invariance(qisg):
    """Larger instances against qisg_create handles (LANES and SAMPLES), under
    two schedules and the autotuner."""
    specs = [(16, 64, 12, 1.1, 7), (12, 128, 20, 0.9, 8), (8, 256, 32, 1.0, 9)]
    refs = []
    for (L, Lt, ns, g, seed) in specs:
        lad = qisg.ladder_linear(0.2, 0.5, ns, g)
        with qisg.Instance(qisg.Config(L, Lt, lad, 4, 1, seed, layout=qisg.QISG_LAYOUT_LANES)) as h:
            h.sweep(30)
            refs.append((h.spins()[0], h.permutation()[0], h.energies()[0][0]))
    for sched in ((1, 0), (8, 1), None):
        with qisg.Batch(4, 256 << 20) as b:
            slots = [b.admit(L, Lt, qisg.ladder_linear(0.2, 0.5, ns, g), 4, seed)
                     for (L, Lt, ns, g, seed) in specs]
            if sched is None:
                rows, order = b.autotune(2)        # runs 10 x 2 sweeps
                b.run(30 - 20)
            else:
                b.set_schedule(*sched)
                b.run(30)
            for slot, (S, wa, A) in zip(slots, refs):
                A2, _, wa2, S2 = b.results(slot, spins=True)
                assert np.array_equal(S2, S) and np.array_equal(wa2, wa) and np.array_equal(A2, A)


_UNEVEN_REPLAYS = {}


@pytest.mark.parametrize("rows,order", [(16, 0), (4, 1)])
def test_uneven_batch_full_size_sampled(qisg, rows, order):
    """The benchmark's batch (512 uneven instances, one persistent kernel) in
    two tile schedules: after 20 sweeps, instances covering every L and
    every L_tau of the mix (the smallest of each) and the largest one are
    replayed by the oracle and compared bit for bit."""
    from concurrent.futures import ThreadPoolExecutor
    from paper_2402_03920_gb300.workloads import uneven_batch
    specs = uneven_batch(512, seed=2024, sweeps=100)
    size = [sp.L * sp.L * sp.L_tau * sp.n_slots * sp.n_replicas for sp in specs]
    picks = {int(np.argmax(size))}
    for key in ("L", "L_tau"):
        for v in sorted({getattr(sp, key) for sp in specs}):
            picks.add(min((i for i, sp in enumerate(specs) if getattr(sp, key) == v), key=lambda i: size[i]))
    picks = sorted(picks)
    assert {specs[i].L for i in picks} == {8, 12, 16, 20, 24}
    assert {specs[i].L_tau for i in picks} == {64, 128, 256, 512, 1024}
    n = 20

    def replay(i):
        if i not in _UNEVEN_REPLAYS:   # the same replay serves both schedules
            sp = specs[i]
            lad = qisg.ladder_linear(sp.k_lo, sp.k_hi, sp.n_slots, sp.gamma)
            st = oracle.new_state(sp.L, sp.L_tau, lad[:, 0], lad[:, 1], sp.n_replicas, sp.seed)
            _UNEVEN_REPLAYS[i] = oracle.run(st, n, n_threads=1)
        return _UNEVEN_REPLAYS[i]

    with qisg.Batch(512, 0) as b:
        slots = [b.admit(sp.L, sp.L_tau, qisg.ladder_linear(sp.k_lo, sp.k_hi, sp.n_slots, sp.gamma), sp.n_replicas,
                         sp.seed) for sp in specs]
        b.set_schedule(rows, order)
        b.run(n)
        with ThreadPoolExecutor(max_workers=len(picks)) as ex:
            states = list(ex.map(replay, picks))
        for i, st in zip(picks, states):
            A, B, wa, S = b.results(slots[i], spins=True)
            assert np.array_equal(wa, st.walker_at[0]), i
            assert np.array_equal(S, st.S[0]), i
            assert np.array_equal(A, st.A[0]) and np.array_equal(B, st.B[0]), i


def test_barrier_wait_runs_out(qisg):
    """A grid-barrier wait bounded to 1 ns runs out (the blocks of the
    persistent launch never reach a barrier together that fast): the launch
    ends and the next synchronising call reports ETIMEOUT.  A fresh batch
    then runs normally and matches the oracle.  Nothing here waits unbounded
    or faults: the kernel gives up and returns."""
    lad = qisg.ladder_linear(0.2, 0.5, 16, 1.0)
    with qisg.Batch(8, 256 << 20) as b:
        for i in range(6):
            b.admit(16, 64, lad, 4, 40 + i)
        b.set_wait_limit(1)
        b.run(50)
        with pytest.raises(qisg.QisgError) as e:
            b.sync()
        assert e.value.code == -4
    with qisg.Batch(2, 64 << 20) as b:
        s = b.admit(8, 16, lad, 4, 41)
        b.run(6)
        b.sync()
        A, B, wa, S = b.results(s, spins=True)
        st = _oracle_instance(8, 16, lad, 4, 41, 6)
        assert np.array_equal(S, st.S[0]) and np.array_equal(wa, st.walker_at[0])


def test_antiperiodic_instances_in_the_mix(qisg):
    """Instances with the antiperiodic boundary along tau (Sec. 1) next to
    periodic ones in one persistent launch: each matches the oracle with its
    own boundary."""
    specs = [(6, 8, 7, 1.0, 71, 1), (8, 16, 12, 0.9, 72, 0), (4, 32, 20, 1.1, 73, 1), (6, 4, 5, 1.2, 74, 1)]
    with qisg.Batch(4, 64 << 20) as b:
        slots = [b.admit(L, Lt, qisg.ladder_linear(0.2, 0.5, ns, g), 4, seed, tau_antiperiodic=ap)
                 for (L, Lt, ns, g, seed, ap) in specs]
        b.run(17)
        for slot, (L, Lt, ns, g, seed, ap) in zip(slots, specs):
            lad = qisg.ladder_linear(0.2, 0.5, ns, g)
            st = oracle.new_state(L, Lt, lad[:, 0], lad[:, 1], 4, seed, tau_ap=bool(ap))
            oracle.run(st, 17)
            A, B, wa, S = b.results(slot, spins=True)
            assert np.array_equal(S, st.S[0]) and np.array_equal(wa, st.walker_at[0]), slot
            assert np.array_equal(A, st.A[0]) and np.array_equal(B, st.B[0]), slot
