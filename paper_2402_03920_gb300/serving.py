"""Serving loop: continuous batching of simulation requests on one GPU.

Requests (an L x L x L_tau instance with its own ladder, seed and sweep count)
arrive over time.  The loop keeps one ``qisg_batch`` resident: between chunks
of sweeps it admits queued requests into free slots while the device-memory
arena has room (first come, first served), runs one persistent launch over
every active instance, and retires the requests that reached their sweep
target, reading back their results.  Each instance keeps its own state and
Philox counters on the device, so a request's result is the same whether it
ran alone or alongside others.

All simulation work runs in the library's kernels; this module only decides
what is admitted and when (host scheduling).
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import qisg


@dataclass
class Request:
    rid: int
    L: int
    L_tau: int
    n_slots: int
    gamma: float
    sweeps: int
    seed: int
    arrival: float = 0.0           # seconds after the start of the run
    n_replicas: int = 4
    k_lo: float = 0.2
    k_hi: float = 0.5
    tau_antiperiodic: int = 0      # boundary along tau (Sec. 1)


@dataclass
class Result:
    rid: int
    A: np.ndarray
    B: np.ndarray
    walker_at: np.ndarray
    spins: np.ndarray | None
    arrival: float
    admitted: float
    finished: float

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


@dataclass
class Stats:
    completed: int = 0
    updates: int = 0
    wall: float = 0.0
    chunks: int = 0
    latencies: list = field(default_factory=list)
    max_active: int = 0
    refused_for_memory: int = 0     # admission attempts deferred because the arena was full
    rejected: list = field(default_factory=list)   # rids that cannot fit even in an empty batch

    def summary(self) -> dict:
        lat = np.array(self.latencies) if self.latencies else np.zeros(1)
        return {"completed": self.completed, "wall_s": self.wall, "chunks": self.chunks,
                "updates": self.updates,
                "ps_per_update": self.wall * 1e12 / max(self.updates, 1),
                "p50_latency_s": float(np.percentile(lat, 50)),
                "p99_latency_s": float(np.percentile(lat, 99)),
                "max_active": self.max_active, "refused_for_memory": self.refused_for_memory,
                "rejected": len(self.rejected)}


def updates_of(req: Request) -> int:
    return req.L * req.L * req.L_tau * req.n_replicas * req.n_slots * req.sweeps


class Server:
    """One resident batch, admission by memory, continuous batching.

    ``batch`` defaults to a new ``qisg.Batch(capacity, mem_budget, stream)``;
    any object with the same admit/run/status/results/retire calls can stand
    in for it (the scheduling logic is tested that way on the host)."""

    def __init__(self, capacity: int = 256, mem_budget: int = 8 << 30, chunk_sweeps: int = 50,
                 keep_spins: bool = False, stream: int | None = None, batch=None):
        self.batch = batch if batch is not None else qisg.Batch(capacity, mem_budget, stream)
        self.chunk = chunk_sweeps
        self._t0 = time.perf_counter()
        self.keep_spins = keep_spins
        self.queue: list[Request] = []
        self.active: dict[int, tuple[Request, float]] = {}   # slot -> (request, admitted at)
        self.results: dict[int, Result] = {}
        self.stats = Stats()

    def close(self):
        self.batch.close()

    def submit(self, req: Request):
        self.queue.append(req)

    def _admit(self, now: float):
        while self.queue:
            req = self.queue[0]
            lad = qisg.ladder_linear(req.k_lo, req.k_hi, req.n_slots, req.gamma)
            slot = self.batch.try_admit(req.L, req.L_tau, lad, req.n_replicas, req.seed, req.sweeps,
                                        req.tau_antiperiodic)
            if slot is None and not self.active:
                # refused by an empty batch: it never fits, and waiting would
                # block the queue for good
                self.queue.pop(0)
                self.stats.rejected.append(req.rid)
                continue
            if slot is None:
                self.stats.refused_for_memory += 1
                break          # wait for memory to free up (FIFO)
            self.queue.pop(0)
            self.active[slot] = (req, now)
        self.stats.max_active = max(self.stats.max_active, len(self.active))

    def _retire(self, now: float):
        for slot in list(self.active):
            done_sweeps, done = self.batch.status(slot)
            if not done:
                continue
            req, admitted = self.active.pop(slot)
            A, B, wa, S = self.batch.results(slot, spins=self.keep_spins)
            self.batch.retire(slot)
            self.results[req.rid] = Result(req.rid, A, B, wa, S, req.arrival, admitted, now)
            self.stats.completed += 1
            self.stats.updates += updates_of(req)
            self.stats.latencies.append(now - req.arrival)

    def step(self, now: float):
        """Admit, run one chunk, retire."""
        self._admit(now)
        if self.active:
            self.batch.run(self.chunk)
            self.batch.sync()
            self.stats.chunks += 1
        self._retire(self.clock())

    def clock(self) -> float:
        """Seconds since the start of the current ``serve`` run."""
        return time.perf_counter() - self._t0

    def serve(self, requests: list[Request], realtime: bool = True, max_wall: float = 3600.0) -> Stats:
        """Feed requests at their arrival times (seconds from start) and run
        until all are done.  With realtime=False every request is available at
        once (offline batch)."""
        pending = sorted(requests, key=lambda r: r.arrival)
        self._t0 = time.perf_counter()
        i = 0
        while i < len(pending) or self.queue or self.active:
            now = self.clock()
            while i < len(pending) and (not realtime or pending[i].arrival <= now):
                r = pending[i]
                if not realtime:
                    r.arrival = 0.0
                self.submit(r)
                i += 1
            if not self.queue and not self.active:
                # idle until the next arrival
                if i < len(pending):
                    time.sleep(max(0.0, min(0.01, pending[i].arrival - now)))
                continue
            self.step(now)
            if now > max_wall:
                raise TimeoutError("serving run exceeded its wall-clock budget")
        self.stats.wall = self.clock()
        return self.stats
