"""Host scheduling of the serving loop, without a GPU: the Server runs
against a stand-in batch with the same calls (admission by an arena budget,
sweep counters, retirement), so FIFO admission, head-of-line blocking,
rejection of requests that can never fit, retirement and the accounting
are checked on their own."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2402_03920_gb300.serving import Request, Server, updates_of


class FakeBatch:
    """Arena of `budget` bytes, `capacity` slots; an instance takes one byte
    per spin plus a fixed header, and advances by the sweeps of each run."""

    HEADER = 64

    def __init__(self, capacity, budget):
        self.capacity, self.budget, self.used = capacity, budget, 0
        self.slots = {}            # slot -> dict(req fields, done, target, bytes)
        self.admit_log = []        # seeds in admission order
        self.runs = []             # (n_sweeps, active seeds) per run
        self.max_bytes = 0

    def nbytes(self, L, L_tau, n_slots, n_rep):
        return L * L * L_tau * n_slots * n_rep + self.HEADER

    def try_admit(self, L, L_tau, ladder, n_rep, seed, n_sweeps, tau_antiperiodic=0):
        b = self.nbytes(L, L_tau, ladder.shape[0], n_rep)
        free = [k for k in range(self.capacity) if k not in self.slots]
        if not free or self.used + b > self.budget:
            return None
        k = free[0]
        self.slots[k] = dict(L=L, Lt=L_tau, n_slots=ladder.shape[0], n_rep=n_rep, seed=seed, done=0,
                             target=n_sweeps, bytes=b)
        self.used += b
        self.max_bytes = max(self.max_bytes, self.used)
        self.admit_log.append(seed)
        return k

    def run(self, n):
        self.runs.append((n, sorted(v["seed"] for v in self.slots.values())))
        for v in self.slots.values():
            v["done"] = min(v["target"], v["done"] + n)

    def sync(self):
        pass

    def status(self, k):
        v = self.slots[k]
        return v["done"], v["done"] >= v["target"]

    def results(self, k, spins=False):
        v = self.slots[k]
        A = np.full((v["n_rep"], v["n_slots"]), v["seed"], dtype=np.int64)
        wa = np.tile(np.arange(v["n_slots"], dtype=np.int32), (v["n_rep"], 1))
        S = np.ones((v["n_rep"], v["n_slots"], v["L"] ** 2 * v["Lt"]), dtype=np.int8) if spins else None
        return A, -A, wa, S

    def retire(self, k):
        self.used -= self.slots.pop(k)["bytes"]

    def close(self):
        pass


def _req(rid, L, Lt, n_slots, sweeps, arrival=0.0):
    return Request(rid=rid, L=L, L_tau=Lt, n_slots=n_slots, gamma=1.0, sweeps=sweeps, seed=rid,
                   arrival=arrival)


def _size(r):
    return r.L * r.L * r.L_tau * r.n_slots * r.n_replicas + FakeBatch.HEADER


def test_fifo_admission_blocks_behind_the_head():
    """A request that does not fit yet holds back the ones behind it, even
    those that would fit (first come, first served)."""
    small0, big1, small2 = _req(0, 4, 8, 4, 5), _req(1, 8, 16, 8, 3), _req(2, 4, 8, 4, 2)
    fb = FakeBatch(8, budget=_size(big1) + _size(small0) - 1)   # big1 and small0 never together
    srv = Server(chunk_sweeps=2, batch=fb)
    stats = srv.serve([small0, big1, small2], realtime=False)
    assert stats.completed == 3 and not stats.rejected
    assert fb.admit_log == [0, 1, 2]
    assert stats.refused_for_memory >= 1
    # small2 fits beside small0 but was not admitted before big1
    assert all(not (0 in active and 2 in active) for _, active in fb.runs)
    assert fb.max_bytes <= fb.budget


def test_request_too_large_for_the_arena_is_rejected_not_waited_on():
    big = _req(0, 16, 64, 32, 4)
    ok = _req(1, 4, 8, 4, 3)
    fb = FakeBatch(4, budget=_size(ok) * 3)
    srv = Server(chunk_sweeps=2, batch=fb)
    stats = srv.serve([big, ok], realtime=False, max_wall=30.0)
    assert stats.rejected == [0]
    assert stats.completed == 1 and 1 in srv.results and 0 not in srv.results
    assert stats.summary()["rejected"] == 1


@pytest.mark.parametrize("chunk", [1, 3, 7])
def test_accounting_and_continuous_batching(chunk):
    rng = np.random.default_rng(chunk)
    reqs = [_req(i, int(rng.choice([2, 4, 6])), int(rng.choice([4, 8, 16])), int(rng.integers(2, 9)),
                 int(rng.integers(1, 12))) for i in range(25)]
    fb = FakeBatch(capacity=5, budget=4 * max(_size(r) for r in reqs))
    srv = Server(chunk_sweeps=chunk, batch=fb)
    stats = srv.serve(reqs, realtime=False)
    assert stats.completed == len(reqs) and not stats.rejected
    assert stats.updates == sum(updates_of(r) for r in reqs)
    assert stats.chunks == len(fb.runs) and all(n == chunk for n, _ in fb.runs)
    assert 1 < stats.max_active <= 5
    assert len(stats.latencies) == len(reqs) and min(stats.latencies) >= 0.0
    s = stats.summary()
    assert s["p50_latency_s"] <= s["p99_latency_s"]
    assert not fb.slots and fb.used == 0                  # everything retired, arena empty
    # admission is FIFO, and each request ran for the chunks it needed: it
    # is retired after the first chunk that reaches its sweep count
    assert fb.admit_log == sorted(fb.admit_log)
    for r in reqs:
        runs_active = sum(1 for _, active in fb.runs if r.rid in active)
        assert runs_active == -(-r.sweeps // chunk), r.rid
        res = srv.results[r.rid]
        assert res.A.shape == (r.n_replicas, r.n_slots) and int(res.A[0, 0]) == r.rid
        assert res.admitted <= res.finished
