"""Seeded synthetic workloads (shapes and sizes only; no arithmetic of the
method).  Both the tests and ``bench.py`` draw their inputs from here; the
couplings, start spins and Monte Carlo numbers themselves come from Philox
under each workload's seed.

The paper's production runs (Sec. 2.1, Sec. 4, Appendix E) use L = 16..24,
L_tau = 2048..8192, k near 0.29 and 6 replicas on samples that are not
public; these recipes stand in for them with +-J disorder at p = 1/2.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class Workload:
    name: str
    L: int
    L_tau: int
    k_lo: float
    k_hi: float
    n_slots: int
    gamma: float
    n_replicas: int
    n_samples: int
    seed: int
    sweeps: int
    measure_every: int = 0
    word_bits: int = 0


# One sample, L=8, L_tau=32, 4 replicas x 8 slots, k in [0.25, 0.45], Gamma=1,
# 1000 sweeps, 32 systems per uint32 word.
PLAIN_SMALL = Workload("plain L8 Ltau32 4rep 8slots 1sample", 8, 32, 0.25, 0.45, 8, 1.0, 4, 1, 1,
                       1000, 0, 32)

# 32 samples, L=16, L_tau=256, 4 replicas x 16 slots, k in [0.2, 0.5],
# Gamma=1, 10^4 sweeps, PT every sweep, measurements every 10 sweeps.
PRODUCTION = Workload("production L16 Ltau256 4rep 16slots 32samples", 16, 256, 0.2, 0.5, 16, 1.0,
                      4, 32, 1, 10_000, 10, 64)

# 1024 samples x 4 replicas x 32 slots, L=24, L_tau=512, 2000 sweeps.
BATCHED = Workload("batched L24 Ltau512 4rep 32slots 1024samples", 24, 512, 0.2, 0.5, 32, 1.0, 4,
                   1024, 1, 2000, 0, 64)

# The exact-enumeration lattice.
ENUM = Workload("enumeration L2 Ltau4", 2, 4, 0.25, 0.45, 4, 1.0, 4, 1, 6, 0)


@dataclass(frozen=True)
class InstanceSpec:
    """One independent simulation of a batch or a serving stream."""
    L: int
    L_tau: int
    n_slots: int
    gamma: float
    sweeps: int
    seed: int
    n_replicas: int = 4
    k_lo: float = 0.2
    k_hi: float = 0.5
    arrival: float = 0.0


def uneven_batch(n: int = 512, seed: int = 2024, sweeps: int = 1000):
    """Instances with L in {8,12,16,20,24}, L_tau in {64..1024} (powers of
    two), 8..32 slots, Gamma uniform in [0.8, 1.2], one seed per instance."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        out.append(InstanceSpec(
            L=int(rng.choice([8, 12, 16, 20, 24])),
            L_tau=int(rng.choice([64, 128, 256, 512, 1024])),
            n_slots=int(rng.integers(8, 33)),
            gamma=float(rng.uniform(0.8, 1.2)),
            sweeps=sweeps,
            seed=i + 1))
    return out


def poisson_requests(n: int = 5000, rate: float = 200.0, seed: int = 7):
    """Poisson arrivals (rate per second) of requests with L in {8..24}
    (even), L_tau in {32..1024} (powers of two), 8..32 slots, 100..5000
    sweeps, Gamma uniform in [0.8, 1.2], one seed per request."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += float(rng.exponential(1.0 / rate))
        out.append(InstanceSpec(
            L=int(rng.choice(np.arange(8, 25, 2))),
            L_tau=int(rng.choice([32, 64, 128, 256, 512, 1024])),
            n_slots=int(rng.integers(8, 33)),
            gamma=float(rng.uniform(0.8, 1.2)),
            sweeps=int(rng.integers(100, 5001)),
            seed=1_000_000 + i,
            arrival=t))
    return out


def random_spins(shape, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return (1 - 2 * rng.integers(0, 2, size=shape)).astype(np.int8)


def random_permutations(n_rows: int, n_slots: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.stack([rng.permutation(n_slots) for _ in range(n_rows)]).astype(np.int32)
