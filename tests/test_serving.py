"""Serving loop: continuous batching under a memory budget; every request's
result is the same alone and in the mix, and matches the oracle."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def _requests(n, seed):
    from paper_2402_03920_gb300.serving import Request
    rng = np.random.default_rng(seed)
    out, t = [], 0.0
    for i in range(n):
        t += float(rng.exponential(0.002))
        out.append(Request(rid=i, L=int(rng.choice([2, 4, 6, 8])), L_tau=int(rng.choice([4, 8, 16, 32])),
                           n_slots=int(rng.integers(4, 33)), gamma=float(rng.uniform(0.8, 1.2)),
                           sweeps=int(rng.integers(3, 40)), seed=500 + i, arrival=t))
    return out


def test_alone_equals_mix_and_oracle():
    need_gpu()
    from paper_2402_03920_gb300 import qisg
    from paper_2402_03920_gb300.serving import Server
    reqs = _requests(14, 1)
    per = max(qisg.Batch.instance_bytes(r.L, r.L_tau, qisg.ladder_linear(0.2, 0.5, r.n_slots, r.gamma))
              for r in reqs)
    # room for about three instances at a time: requests queue and join as
    # others finish (continuous batching)
    srv = Server(capacity=8, mem_budget=3 * per + 4096, chunk_sweeps=7, keep_spins=True)
    try:
        stats = srv.serve(reqs, realtime=True)
    finally:
        srv.close()
    assert stats.completed == len(reqs)
    assert 1 < stats.max_active <= 8
    s = stats.summary()
    assert s["p50_latency_s"] <= s["p99_latency_s"]
    for r in reqs:
        res = srv.results[r.rid]
        lad = qisg.ladder_linear(r.k_lo, r.k_hi, r.n_slots, r.gamma)
        # alone: a fresh batch holding only this request
        with qisg.Batch(1, 16 << 20) as b:
            slot = b.admit(r.L, r.L_tau, lad, r.n_replicas, r.seed, r.sweeps)
            b.run(r.sweeps + 5)
            A, B, wa, S = b.results(slot, spins=True)
        assert np.array_equal(res.spins, S) and np.array_equal(res.walker_at, wa), r.rid
        assert np.array_equal(res.A, A) and np.array_equal(res.B, B)
        # and the oracle's replay
        st = oracle.new_state(r.L, r.L_tau, lad[:, 0], lad[:, 1], r.n_replicas, r.seed)
        oracle.run(st, r.sweeps)
        assert np.array_equal(res.spins, st.S[0]) and np.array_equal(res.walker_at, st.walker_at[0]), r.rid


def test_full_size_stream_sampled_replay():
    """A Poisson stream of the full request distribution (L 8..24, L_tau
    32..1024, 8..32 slots, Gamma in [0.8, 1.2]) through the serving loop,
    with each request's sweep count capped by an update budget so that the
    oracle can replay it; 16 completed requests, chosen by a fixed seed and
    always including the largest L and the largest L_tau, are replayed by
    the oracle (one host core each) and compared bit for bit."""
    need_gpu()
    from concurrent.futures import ThreadPoolExecutor
    from paper_2402_03920_gb300 import qisg
    from paper_2402_03920_gb300.serving import Request, Server
    from paper_2402_03920_gb300.workloads import poisson_requests
    budget = 1.2e9   # spin updates per replayed request
    reqs = []
    for i, sp in enumerate(poisson_requests(64, rate=400.0, seed=11)):
        per_sweep = sp.L * sp.L * sp.L_tau * sp.n_slots * sp.n_replicas
        sweeps = int(min(sp.sweeps, max(12, budget // per_sweep)))
        reqs.append(Request(rid=i, L=sp.L, L_tau=sp.L_tau, n_slots=sp.n_slots, gamma=sp.gamma, sweeps=sweeps,
                            seed=sp.seed, arrival=sp.arrival))
    srv = Server(capacity=64, mem_budget=4 << 30, chunk_sweeps=25, keep_spins=True)
    try:
        stats = srv.serve(reqs, realtime=True)
    finally:
        srv.close()
    assert stats.completed == len(reqs) and stats.max_active > 1
    rng = np.random.default_rng(16)
    big_L = max(range(len(reqs)), key=lambda i: (reqs[i].L, reqs[i].L_tau))
    big_T = max(range(len(reqs)), key=lambda i: (reqs[i].L_tau, reqs[i].L))
    rest = [i for i in range(len(reqs)) if i not in (big_L, big_T)]
    picks = sorted({big_L, big_T, *rng.choice(rest, size=14, replace=False).tolist()})
    assert reqs[big_L].L == 24 and reqs[big_T].L_tau == 1024

    def replay(i):
        r = reqs[i]
        lad = qisg.ladder_linear(r.k_lo, r.k_hi, r.n_slots, r.gamma)
        st = oracle.new_state(r.L, r.L_tau, lad[:, 0], lad[:, 1], r.n_replicas, r.seed)
        return oracle.run(st, r.sweeps, n_threads=1)

    with ThreadPoolExecutor(max_workers=16) as ex:
        states = list(ex.map(replay, picks))
    for i, st in zip(picks, states):
        res = srv.results[reqs[i].rid]
        assert np.array_equal(res.walker_at, st.walker_at[0]), i
        assert np.array_equal(res.spins, st.S[0]), i
        assert np.array_equal(res.A, st.A[0]) and np.array_equal(res.B, st.B[0]), i
