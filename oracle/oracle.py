"""ctypes driver for the plain-C oracle (test infrastructure only).

Every function here marshals numpy arrays into ``qisg_oracle.c`` and back;
the arithmetic of the method lives in the C file (except the daemon rule's
cumulative tables, written out below in decimal arithmetic), whose comments cite the
paper passage each step follows (Sec. 1 Eq. (2)-(3), Sec. 2.1, Sec. 2.1.1,
Appendix E.1).  ``build()`` compiles it with gcc; nothing of the product
package is imported.
"""
from __future__ import annotations

import ctypes
import decimal
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qisg_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

N_SEED_BITS = 64


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, OpenMP,
    no floating-point contraction so every product is rounded on its own)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            lib = ctypes.CDLL(path)
            P = ctypes.c_void_p
            i32, i64, u64, f64 = ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
            lib.orc_philox4x32_10.argtypes = [P, P, P]
            lib.orc_philox4x32_10.restype = None
            lib.orc_philox4x32_10_many.argtypes = [i64, P, P, P]
            lib.orc_philox4x32_10_many.restype = None
            lib.orc_ladder_linear.argtypes = [f64, f64, i32, f64, P, P]
            lib.orc_ladder_linear.restype = None
            lib.orc_thresholds.argtypes = [i32, P, P, P]
            lib.orc_thresholds.restype = None
            lib.orc_pt_bases.argtypes = [i32, P, P, P, P, P, P]
            lib.orc_pt_bases.restype = None
            lib.orc_init_couplings.argtypes = [i32, i64, i64, u64, P]
            lib.orc_init_couplings.restype = None
            lib.orc_init_spins.argtypes = [i32, i32, i32, i32, i64, i64, u64, P]
            lib.orc_init_spins.restype = None
            lib.orc_run.argtypes = [i32, i32, i32, i32, i64, i64, u64, P, P, i32, i32,
                                    P, P, P, u64, i64, P, P, P, P, P, P, P, i32, i32, P,
                                    P, i32, P, P]
            lib.orc_run.restype = i32
            lib.orc_energies.argtypes = [i32, i32, i32, i32, i64, P, P, P, P, i32]
            lib.orc_energies.restype = None
            lib.orc_pt_only.argtypes = [i32, i32, i64, u64, P, P, u64, P, P, P]
            lib.orc_pt_only.restype = None
            lib.orc_tau_observables.argtypes = [i32, i32, i32, i32, i64, P, P, P, P, P, P]
            lib.orc_tau_observables.restype = None
            lib.orc_transfer_matvec.argtypes = [i32, f64, f64, P, i32, P, P]
            lib.orc_transfer_matvec.restype = i32
            lib.orc_pow_by_squaring.argtypes = [f64, u64]
            lib.orc_pow_by_squaring.restype = f64
            lib.orc_xoroshiro128pp_step.argtypes = [P]
            lib.orc_xoroshiro128pp_step.restype = None
            lib.orc_daemon_nstar.argtypes = [P, u64]
            lib.orc_daemon_nstar.restype = ctypes.c_uint32
            lib.orc_daemon_bword.argtypes = [u64, i64, i32, i32, ctypes.c_uint32, u64, i32, P]
            lib.orc_daemon_bword.restype = ctypes.c_uint32
            lib.orc_daemon_level.argtypes = [i32, i32, i32]
            lib.orc_daemon_level.restype = i32
            lib.orc_daemon_flip.argtypes = [i32, i32]
            lib.orc_daemon_flip.restype = i32
            lib.orc_daemon_sweep_system.argtypes = [i32, i32, u64, i64, i32, i32, u64, i32, P, P, P]
            lib.orc_daemon_sweep_system.restype = None
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 of one counter (4 x uint32) under one key (2 x uint32)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def philox4x32_10_many(ctr, key) -> np.ndarray:
    """Philox4x32-10 of counters ctr [n][4] under one key (2 x uint32)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros_like(c)
    _load().orc_philox4x32_10_many(len(c), _ptr(c), _ptr(k), _ptr(out))
    return out


def ladder_linear(lo: float, hi: float, n: int, gamma: float):
    k = np.zeros(n, dtype=np.float64)
    kt = np.zeros(n, dtype=np.float64)
    _load().orc_ladder_linear(lo, hi, n, gamma, _ptr(k), _ptr(kt))
    return k, kt


def thresholds(k, ktau) -> np.ndarray:
    k = np.ascontiguousarray(k, dtype=np.float64)
    kt = np.ascontiguousarray(ktau, dtype=np.float64)
    T = np.zeros((len(k), 5, 3), dtype=np.uint32)
    _load().orc_thresholds(len(k), _ptr(k), _ptr(kt), _ptr(T))
    return T


def pt_bases(k, ktau):
    k = np.ascontiguousarray(k, dtype=np.float64)
    kt = np.ascontiguousarray(ktau, dtype=np.float64)
    n = len(k)
    out = [np.zeros(max(n - 1, 1), dtype=np.float64) for _ in range(4)]
    _load().orc_pt_bases(n, _ptr(k), _ptr(kt), *[_ptr(o) for o in out])
    return tuple(o[: max(n - 1, 0)] for o in out)


def pow_by_squaring(b: float, e: int) -> float:
    return _load().orc_pow_by_squaring(float(b), int(e))


# --------------------------------------------------------------------------
# Daemon rule (Sec. 2.1.1, Appendices B and C)
# --------------------------------------------------------------------------

def daemon_cumulative(k: float) -> np.ndarray:
    """cumulative(n), n = 0..254, of Sec. 2.1.1 for coupling k: the 64-bit
    truncation of 2^64 sum_{m <= n} P[m], P[m] = p^pop(m) (1-p)^(8-pop(m)),
    p = e^{-4k}.  The paper evaluates the sum in 128-bit floating point; here
    it is evaluated in decimal arithmetic with 80 significant digits beyond
    those that p^8 = e^{-32k} needs next to 1 (the exact value's
    truncation, which 128-bit arithmetic also gives unless the sum lies
    within about 2^-49 of an integer)."""
    with decimal.localcontext() as ctx:
        ctx.prec = 80 + int(32.0 * float(k) / math.log(10.0)) + 1
        p = (decimal.Decimal(-4) * decimal.Decimal(float(k))).exp()
        q = 1 - p
        scale = decimal.Decimal(2) ** 64
        acc = decimal.Decimal(0)
        out = []
        for n in range(255):
            c = bin(n).count("1")
            acc += (p ** c) * (q ** (8 - c))
            out.append(int((acc * scale).to_integral_value(rounding=decimal.ROUND_FLOOR)))
    return np.array(out, dtype=np.uint64)


def daemon_tables(k) -> np.ndarray:
    """[n_slots][255] cumulative tables of a ladder."""
    return np.ascontiguousarray(np.stack([daemon_cumulative(float(v)) for v in k]), dtype=np.uint64)


def xoroshiro128pp_step(s0: int, s1: int):
    st = np.array([s0, s1], dtype=np.uint64)
    _load().orc_xoroshiro128pp_step(_ptr(st))
    return int(st[0]), int(st[1])


def daemon_nstar(cum: np.ndarray, R: int) -> int:
    return int(_load().orc_daemon_nstar(_ptr(np.ascontiguousarray(cum, dtype=np.uint64)), int(R)))


def daemon_bword(seed: int, a: int, r: int, s: int, wsite: int, t: int, which: int,
                 cum: np.ndarray) -> int:
    return int(_load().orc_daemon_bword(seed, a, r, s, wsite, t, which,
                                        _ptr(np.ascontiguousarray(cum, dtype=np.uint64))))


def daemon_level(b4: int, b8: int, b12: int) -> int:
    return int(_load().orc_daemon_level(b4, b8, b12))


def daemon_flip(u: int, d: int) -> bool:
    return bool(_load().orc_daemon_flip(u, d))


def daemon_sweep_system(L: int, Ltau: int, seed: int, a: int, r: int, s: int, t: int, J_a: np.ndarray,
                        S: np.ndarray, cum: np.ndarray, tau_ap: bool = False) -> None:
    """One daemon-rule sweep t of one system (sample a, replica r, slot s)
    in place: S [N] int8, J_a [L*L][2] of sample a, cum [n_slots][255]."""
    assert S.dtype == np.int8 and S.flags["C_CONTIGUOUS"]
    _load().orc_daemon_sweep_system(L, Ltau, seed, a, r, s, t, int(bool(tau_ap)),
                                    _ptr(np.ascontiguousarray(J_a, dtype=np.int8)), _ptr(S),
                                    _ptr(np.ascontiguousarray(cum, dtype=np.uint64)))


def init_couplings(L: int, a_lo: int, n_a: int, seed: int) -> np.ndarray:
    J = np.zeros((n_a, L * L, 2), dtype=np.int8)
    _load().orc_init_couplings(L, a_lo, n_a, seed, _ptr(J))
    return J


def init_spins(L: int, Ltau: int, n_slots: int, n_rep: int, a_lo: int, n_a: int,
               seed: int) -> np.ndarray:
    S = np.zeros((n_a, n_rep, n_slots, L * L * Ltau), dtype=np.int8)
    _load().orc_init_spins(L, Ltau, n_slots, n_rep, a_lo, n_a, seed, _ptr(S))
    return S


def energies(L: int, Ltau: int, J: np.ndarray, S: np.ndarray, tau_ap: bool = False):
    """A, B (by walker) of configurations S[n_a][n_rep][n_slots][N];
    tau_ap: antiperiodic along tau."""
    n_a, n_rep, n_slots, _ = S.shape
    A = np.zeros((n_a, n_rep, n_slots), dtype=np.int64)
    B = np.zeros_like(A)
    _load().orc_energies(L, Ltau, n_slots, n_rep, n_a, _ptr(np.ascontiguousarray(J)),
                         _ptr(np.ascontiguousarray(S)), _ptr(A), _ptr(B), int(bool(tau_ap)))
    return A, B


def pt_only(a: int, seed: int, k, ktau, t: int, walker_at_a: np.ndarray,
            A_a: np.ndarray, B_a: np.ndarray) -> None:
    """One PT pass of every replica chain of sample a, energies by walker.
    ``walker_at_a`` [n_rep][n_slots] is updated in place."""
    k = np.ascontiguousarray(k, dtype=np.float64)
    kt = np.ascontiguousarray(ktau, dtype=np.float64)
    n_rep, n_slots = walker_at_a.shape
    _load().orc_pt_only(n_slots, n_rep, a, seed, _ptr(k), _ptr(kt), t, _ptr(walker_at_a),
                        _ptr(np.ascontiguousarray(A_a, dtype=np.int64)),
                        _ptr(np.ascontiguousarray(B_a, dtype=np.int64)))


def tau_observables(L: int, Ltau: int, S: np.ndarray, walker_at: np.ndarray):
    """Sums over tau_1 of Q~, Q~^2, Q~^4 and of the two squared Fourier
    moduli (Appendix E.1) for the configuration at every slot:
    four arrays [n_a][n_rep][n_slots][L_tau] (int64, int64, int64, float64)."""
    n_a, n_rep, n_slots, _ = S.shape
    shp = (n_a, n_rep, n_slots, Ltau)
    S1, S2, S4 = (np.zeros(shp, dtype=np.int64) for _ in range(3))
    SF = np.zeros(shp, dtype=np.float64)
    _load().orc_tau_observables(L, Ltau, n_slots, n_rep, n_a, _ptr(np.ascontiguousarray(S, dtype=np.int8)),
                                _ptr(np.ascontiguousarray(walker_at, dtype=np.int32)), _ptr(S1), _ptr(S2),
                                _ptr(S4), _ptr(SF))
    return S1, S2, S4, SF


def transfer_matvec(L: int, k: float, ktau: float, J: np.ndarray, parity: int, v: np.ndarray) -> np.ndarray:
    """T v on the even (+1) or odd (-1) parity sector (Sec. 2.2, Appendix D):
    v has 2^(L^2-1) entries; J is [L*L][2] int8 of one sample."""
    vin = np.ascontiguousarray(v, dtype=np.float64)
    out = np.zeros_like(vin)
    rc = _load().orc_transfer_matvec(L, float(k), float(ktau), _ptr(np.ascontiguousarray(J, dtype=np.int8)),
                                     int(parity), _ptr(vin), _ptr(out))
    if rc != 0:
        raise MemoryError("oracle transfer matvec failed")
    return out


@dataclass
class OracleState:
    """State of a set of samples a_lo .. a_lo+n_a-1 of one instance."""
    L: int
    Ltau: int
    k: np.ndarray
    ktau: np.ndarray
    n_rep: int
    a_lo: int
    n_a: int
    seed: int
    J: np.ndarray            # [n_a][L*L][2] int8
    S: np.ndarray            # [n_a][n_rep][n_slots][N] int8, by walker
    walker_at: np.ndarray    # [n_a][n_rep][n_slots] int32
    t: int = 0               # sweeps done
    A: np.ndarray = None     # [n_a][n_rep][n_slots] by slot
    B: np.ndarray = None
    sumA: np.ndarray = None
    sumB: np.ndarray = None
    sumq: np.ndarray = None  # [n_a][n_slots][n_pairs]
    sumq2: np.ndarray = None
    n_meas: int = 0
    tau_ap: bool = False     # antiperiodic along tau
    cum: np.ndarray = None   # daemon rule: [n_slots][255] cumulative tables; None: thresholds
    keep_history: bool = False   # record the PT walk at every measurement (history_betas)
    maxit: int = 0               # measurements per block sum (0: none)
    hist: np.ndarray = None      # [n_meas][n_a][n_rep][n_slots] uint8: slot of every walker
    blkA: np.ndarray = None      # [n_blocks][n_a][n_rep][n_slots] by slot: block sums
    blkB: np.ndarray = None

    @property
    def n_slots(self) -> int:
        return len(self.k)

    @property
    def N(self) -> int:
        return self.L * self.L * self.Ltau


def new_state(L, Ltau, k, ktau, n_rep, seed, a_lo=0, n_a=1, tau_ap=False,
              daemon=False) -> OracleState:
    """daemon: the paper's multi-site daemon rule (needs k_tau = k and
    L_tau a multiple of 64) instead of the threshold table."""
    k = np.ascontiguousarray(k, dtype=np.float64)
    kt = np.ascontiguousarray(ktau, dtype=np.float64)
    n_slots = len(k)
    if daemon and (not np.array_equal(k, kt) or Ltau % 64 != 0):
        raise ValueError("the daemon rule needs k_tau = k and L_tau a multiple of 64")
    J = init_couplings(L, a_lo, n_a, seed)
    S = init_spins(L, Ltau, n_slots, n_rep, a_lo, n_a, seed)
    wa = np.tile(np.arange(n_slots, dtype=np.int32), (n_a, n_rep, 1)).copy()
    st = OracleState(L, Ltau, k, kt, n_rep, a_lo, n_a, seed, J, S, wa, tau_ap=bool(tau_ap),
                     cum=daemon_tables(k) if daemon else None)
    alloc_obs(st)
    refresh_energies(st)
    return st


def refresh_energies(st: OracleState) -> None:
    """Set st.A, st.B (by slot) from the current configurations."""
    Aw, Bw = energies(st.L, st.Ltau, st.J, st.S, st.tau_ap)
    idx = st.walker_at.astype(np.int64)
    st.A = np.take_along_axis(Aw, idx, axis=2)
    st.B = np.take_along_axis(Bw, idx, axis=2)


def alloc_obs(st: OracleState) -> None:
    n_pairs = st.n_rep * (st.n_rep - 1) // 2
    shp = (st.n_a, st.n_rep, st.n_slots)
    st.A = np.zeros(shp, dtype=np.int64)
    st.B = np.zeros(shp, dtype=np.int64)
    st.sumA = np.zeros(shp, dtype=np.int64)
    st.sumB = np.zeros(shp, dtype=np.int64)
    st.sumq = np.zeros((st.n_a, st.n_slots, max(n_pairs, 1)), dtype=np.int64)
    st.sumq2 = np.zeros_like(st.sumq)


def _grow(arr, rows: int, shape_tail, dtype):
    """arr with at least `rows` leading rows (new rows zero)."""
    if arr is not None and arr.shape[0] >= rows:
        return arr
    out = np.zeros((max(rows, 1),) + tuple(shape_tail), dtype=dtype)
    if arr is not None:
        out[: arr.shape[0]] = arr
    return out


def run(st: OracleState, n_sweeps: int, pt_every: int = 1, measure_every: int = 0,
        n_threads: int = 0) -> OracleState:
    """Advance the state by n_sweeps sweeps (in place)."""
    lib = _load()
    n_meas = ctypes.c_int64(st.n_meas)
    new_meas = 0
    if measure_every > 0:
        new_meas = (st.t + n_sweeps) // measure_every - st.t // measure_every
    tail = (st.n_a, st.n_rep, st.n_slots)
    if st.keep_history:
        st.hist = _grow(st.hist, st.n_meas + new_meas, tail, np.uint8)
    if st.maxit > 0:
        nb = -(-(st.n_meas + new_meas) // st.maxit)
        st.blkA = _grow(st.blkA, nb, tail, np.int64)
        st.blkB = _grow(st.blkB, nb, tail, np.int64)
    rc = lib.orc_run(st.L, st.Ltau, st.n_slots, st.n_rep, st.a_lo, st.n_a, st.seed,
                     _ptr(st.k), _ptr(st.ktau), pt_every, measure_every,
                     _ptr(st.J), _ptr(st.S), _ptr(st.walker_at), st.t, n_sweeps,
                     _ptr(st.A), _ptr(st.B), _ptr(st.sumA), _ptr(st.sumB),
                     _ptr(st.sumq), _ptr(st.sumq2), ctypes.byref(n_meas), n_threads, int(st.tau_ap),
                     _ptr(st.cum) if st.cum is not None else None,
                     _ptr(st.hist) if st.keep_history else None, int(st.maxit),
                     _ptr(st.blkA) if st.maxit > 0 else None, _ptr(st.blkB) if st.maxit > 0 else None)
    if rc == -2:
        raise ValueError("the daemon rule needs k_tau = k, L_tau % 64 == 0 and fewer than 2^24 samples")
    if rc != 0:
        raise MemoryError("oracle run failed")
    st.t += n_sweeps
    st.n_meas = n_meas.value
    return st


def slot_means(st: OracleState, n_samples_total: int | None = None):
    """FP64 per-slot means over (sample, replica, measurement), summed in the
    fixed order sample, replica (slot-major output): e_s = A/(2N),
    e_t = B/N and the mean squared overlap q^2/N^2 over replica pairs."""
    n_pairs = st.n_rep * (st.n_rep - 1) // 2
    N = float(st.N)
    m = float(st.n_meas)
    e_s = np.zeros(st.n_slots)
    e_t = np.zeros(st.n_slots)
    q2 = np.zeros(st.n_slots)
    for s in range(st.n_slots):
        sa = 0.0
        sb = 0.0
        for a in range(st.n_a):
            for r in range(st.n_rep):
                sa += float(st.sumA[a, r, s])
                sb += float(st.sumB[a, r, s])
        e_s[s] = sa / (m * st.n_a * st.n_rep * 2.0 * N)
        e_t[s] = sb / (m * st.n_a * st.n_rep * N)
        sq = 0.0
        for a in range(st.n_a):
            for p in range(n_pairs):
                sq += float(st.sumq2[a, s, p])
        q2[s] = sq / (m * st.n_a * max(n_pairs, 1) * N * N)
    return e_s, e_t, q2
