"""Python binding of libqisg (ctypes; argument marshalling only).

Every call here forwards to the C ABI of ``include/qisg.h``; every step of
the sweep, PT and measurement path runs in the library's CUDA kernels.  The
binding only converts numpy arrays and the torch stream into plain pointers.
If the library cannot be loaded the import fails loudly: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import _build_lib

QISG_LAYOUT_AUTO, QISG_LAYOUT_LANES, QISG_LAYOUT_SAMPLES, QISG_LAYOUT_SITES = 0, 1, 2, 3
KERNEL_SWEEP, KERNEL_PT, KERNEL_MEASURE, KERNEL_PERMUTE, KERNEL_BLUE, KERNEL_RED = 0, 1, 2, 3, 4, 5
PROFILE_ONLY = 0x100
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ETIMEOUT", -5: "ECORRUPT", -6: "ESTATE"}


class QisgError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"QISG_{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Slot(ctypes.Structure):
    _fields_ = [("k", ctypes.c_double), ("k_tau", ctypes.c_double)]


class Opts(ctypes.Structure):
    _fields_ = [("word_bits", ctypes.c_int), ("cuda_stream", ctypes.c_void_p),
                ("mem_budget", ctypes.c_size_t), ("pt_every", ctypes.c_int),
                ("measure_every", ctypes.c_int), ("layout", ctypes.c_int),
                ("per_sample_launch", ctypes.c_int), ("tau_antiperiodic", ctypes.c_int),
                ("history_len", ctypes.c_int), ("maxit", ctypes.c_int), ("blocks_len", ctypes.c_int)]


_lib = None


def library_path() -> str:
    return _build_lib.LIB


def load(build_if_missing: bool = True):
    """Load libqisg.so (building it first when asked and stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build_lib.build() if build_if_missing else _build_lib.LIB
    if not os.path.exists(path):
        raise ImportError(f"libqisg.so not found at {path}; run the build first")
    lib = ctypes.CDLL(path)
    P, I, I64, U64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    sig = {
        "qisg_opts_default": (None, [P]),
        "qisg_ladder_linear": (I, [D, D, I, D, P]),
        "qisg_create": (I, [P, I, I, P, I, I, I64, U64, P]),
        "qisg_sweep": (I, [P, I64]),
        "qisg_pt_swap": (I, [P]),
        "qisg_energies": (I, [P, P, P]),
        "qisg_overlaps": (I, [P, P]),
        "qisg_permutation": (I, [P, P]),
        "qisg_get_spins": (I, [P, I64, I64, P]),
        "qisg_get_couplings": (I, [P, I64, I64, P]),
        "qisg_set_couplings": (I, [P, P]),
        "qisg_set_state": (I, [P, P, P, U64]),
        "qisg_pt_given": (I, [P, P, P, U64, I]),
        "qisg_measurements": (I, [P, P, P, P, P, P]),
        "qisg_slot_means": (I, [P, P, P, P]),
        "qisg_thresholds": (I, [P, P]),
        "qisg_walk_history": (I, [P, I64, I64, P]),
        "qisg_tau_observables": (I, [P, I64, I64, P, P, P, P]),
        "qisg_checkpoint_save": (I, [P, ctypes.c_char_p]),
        "qisg_checkpoint_load": (I, [P, ctypes.c_char_p]),
        "qisg_checkpoint_verify": (I, [ctypes.c_char_p, P]),
        "qisg_block_sums": (I, [P, I64, I64, P, P]),
        "qisg_block_means": (I, [P, I64, I64, P, P]),
        "qisg_sweep_count": (I, [P, P]),
        "qisg_layout": (I, [P, P, P]),
        "qisg_launch_count": (I, [P, P]),
        "qisg_sync": (I, [P]),
        "qisg_destroy": (None, [P]),
        "qisg_strerror": (ctypes.c_char_p, [I]),
        "qisg_last_error": (ctypes.c_char_p, []),
        "qisg_philox4x32_10": (I, [P, P, P, I64, P]),
        "qisg_profile": (I, [P, I]),
        "qisg_set_graphs": (I, [P, I]),
        "qisg_set_persistent": (I, [P, I, I64]),
        "qisg_set_launch_overlap": (I, [P, I]),
        "qisg_set_pt_in_blue": (I, [P, I, I64]),
        "qisg_autotune": (I, [P, I, P]),
        "qisg_get_tiles": (I, [P, P, P]),
        "qisg_set_tiles": (I, [P, P, P]),
        "qisg_batch_create": (I, [P, I, ctypes.c_size_t, P]),
        "qisg_batch_admit": (I, [P, P, P]),
        "qisg_batch_retire": (I, [P, I]),
        "qisg_batch_run": (I, [P, I64]),
        "qisg_batch_set_schedule": (I, [P, I, I]),
        "qisg_batch_set_wait_limit": (I, [P, I64]),
        "qisg_batch_autotune": (I, [P, I, P, P]),
        "qisg_batch_status": (I, [P, I, P, P]),
        "qisg_batch_results": (I, [P, I, P, P, P, P]),
        "qisg_batch_info": (I, [P, P, P, P]),
        "qisg_batch_instance_bytes": (ctypes.c_size_t, [P]),
        "qisg_batch_sync": (I, [P]),
        "qisg_batch_destroy": (None, [P]),
        "qisg_profile_read": (I, [P, I, P, P, P]),
        "qisg_daemon_tables": (I, [D, I, P, P]),
        "qisg_overlaps_noalloc": (I, [P, I, I, I, I, I, I64, P, P]),
        "qisg_transfer_matvec": (I, [P, P, I, D, D, P, I, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    """Names the binding expects the library to export."""
    return ["qisg_opts_default", "qisg_ladder_linear", "qisg_create", "qisg_sweep", "qisg_pt_swap",
            "qisg_energies", "qisg_overlaps", "qisg_permutation", "qisg_get_spins",
            "qisg_get_couplings", "qisg_set_couplings", "qisg_set_state", "qisg_pt_given", "qisg_measurements",
            "qisg_slot_means", "qisg_walk_history", "qisg_block_sums", "qisg_block_means", "qisg_tau_observables",
            "qisg_checkpoint_save", "qisg_checkpoint_load", "qisg_checkpoint_verify",
            "qisg_thresholds", "qisg_sweep_count", "qisg_layout",
            "qisg_launch_count", "qisg_sync", "qisg_destroy", "qisg_strerror", "qisg_last_error",
            "qisg_philox4x32_10", "qisg_profile", "qisg_profile_read", "qisg_set_graphs", "qisg_set_persistent",
            "qisg_set_launch_overlap",
            "qisg_autotune", "qisg_get_tiles", "qisg_set_tiles", "qisg_batch_create", "qisg_batch_admit", "qisg_batch_retire",
            "qisg_batch_run", "qisg_batch_set_schedule", "qisg_batch_set_wait_limit", "qisg_batch_autotune",
            "qisg_batch_status",
            "qisg_batch_results", "qisg_batch_info", "qisg_batch_instance_bytes", "qisg_batch_sync",
            "qisg_batch_destroy", "qisg_daemon_tables", "qisg_overlaps_noalloc", "qisg_transfer_matvec"]


def _check(rc: int):
    if rc != 0:
        msg = load().qisg_last_error()
        raise QisgError(rc, msg.decode() if msg else "")


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def ladder_linear(lo: float, hi: float, n: int, gamma: float) -> np.ndarray:
    """[n][2] array of (k, k_tau), k linear in [lo, hi], k_tau from
    exp(-2 k_tau) = tanh(k Gamma)."""
    arr = (Slot * n)()
    _check(load().qisg_ladder_linear(lo, hi, n, gamma, ctypes.cast(arr, ctypes.c_void_p)))
    return np.array([[s.k, s.k_tau] for s in arr], dtype=np.float64)


def daemon_tables(k: float, lut_bits: int = 12):
    """cumulative(0..254) (uint64) and the prefix index (uint16, 2^lut_bits
    entries) of the SITES daemon rule for coupling k."""
    cum = np.zeros(255, dtype=np.uint64)
    lut = np.zeros(1 << lut_bits, dtype=np.uint16)
    _check(load().qisg_daemon_tables(float(k), int(lut_bits), _ptr(cum), _ptr(lut)))
    return cum, lut


def _sized(arr, dtype, n: int, what: str) -> np.ndarray:
    """Contiguous copy (or view) of `arr` as `dtype`, which must hold exactly
    n elements: the library reads that many from the pointer."""
    a = np.ascontiguousarray(arr, dtype=dtype)
    if a.size != n:
        raise ValueError(f"{what}: expected {n} elements, got {a.size}")
    return a


def _ladder_array(ladder) -> np.ndarray:
    """The ladder as contiguous float64 [n_slots][2] (k, k_tau) rows."""
    lad = np.ascontiguousarray(ladder, dtype=np.float64)
    if lad.ndim != 2 or lad.shape[1] != 2 or lad.shape[0] < 1:
        raise ValueError(f"ladder: expected [n_slots][2] (k, k_tau) rows, got shape {lad.shape}")
    return lad


def ladder_equal(lo: float, hi: float, n: int) -> np.ndarray:
    """[n][2] ladder with k_tau = k (the paper's single coupling, Sec. 1),
    k linear in [lo, hi]: the ladders the SITES daemon rule takes."""
    k = np.array([lo] if n == 1 else [lo + (hi - lo) * s / (n - 1) for s in range(n)], dtype=np.float64)
    return np.stack([k, k], axis=1)


def current_stream_ptr() -> int | None:
    """cudaStream_t of torch's current stream (torch is used for streams only)."""
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:  # pragma: no cover - torch is optional for the binding
        pass
    return None


@dataclass
class Config:
    L: int
    L_tau: int
    ladder: np.ndarray          # [n_slots][2] (k, k_tau)
    n_replicas: int
    n_samples: int
    seed: int
    word_bits: int = 0
    pt_every: int = 1
    measure_every: int = 0
    layout: int = QISG_LAYOUT_AUTO
    per_sample_launch: int = 0
    tau_antiperiodic: int = 0
    mem_budget: int = 0
    history_len: int = 0
    maxit: int = 0
    blocks_len: int = 0


class Instance:
    """One qisg_handle: n_samples x n_replicas chains of an n_slots ladder."""

    def __init__(self, cfg: Config, stream: int | None = None):
        lib = load()
        self.cfg = cfg
        ladder = _ladder_array(cfg.ladder)
        self.n_slots = ladder.shape[0]
        self.L, self.L_tau = cfg.L, cfg.L_tau
        self.N = cfg.L * cfg.L * cfg.L_tau
        self.n_rep, self.n_samples = cfg.n_replicas, cfg.n_samples
        opts = Opts()
        lib.qisg_opts_default(ctypes.byref(opts))
        opts.word_bits = cfg.word_bits
        opts.cuda_stream = stream if stream is not None else current_stream_ptr()
        opts.mem_budget = cfg.mem_budget
        opts.pt_every = cfg.pt_every
        opts.measure_every = cfg.measure_every
        opts.layout = cfg.layout
        opts.per_sample_launch = cfg.per_sample_launch
        opts.tau_antiperiodic = cfg.tau_antiperiodic
        opts.history_len = cfg.history_len
        opts.maxit = cfg.maxit
        opts.blocks_len = cfg.blocks_len
        self._h = ctypes.c_void_p()
        _check(lib.qisg_create(ctypes.byref(self._h), cfg.L, cfg.L_tau, _ptr(ladder), self.n_slots,
                               cfg.n_replicas, cfg.n_samples, cfg.seed, ctypes.byref(opts)))

    # -- lifecycle ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().qisg_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- path --------------------------------------------------------------
    def sweep(self, n: int = 1):
        _check(load().qisg_sweep(self._h, n))

    def pt_swap(self):
        _check(load().qisg_pt_swap(self._h))

    def sync(self):
        _check(load().qisg_sync(self._h))

    # -- results -----------------------------------------------------------
    @property
    def n_pairs(self) -> int:
        return self.n_rep * (self.n_rep - 1) // 2

    def energies(self):
        A = np.zeros((self.n_samples, self.n_rep, self.n_slots), dtype=np.int64)
        B = np.zeros_like(A)
        _check(load().qisg_energies(self._h, _ptr(A), _ptr(B)))
        return A, B

    def overlaps(self) -> np.ndarray:
        q = np.zeros((self.n_samples, self.n_slots, max(self.n_pairs, 1)), dtype=np.int64)
        _check(load().qisg_overlaps(self._h, _ptr(q)))
        return q[:, :, : self.n_pairs]

    def permutation(self) -> np.ndarray:
        wa = np.zeros((self.n_samples, self.n_rep, self.n_slots), dtype=np.int32)
        _check(load().qisg_permutation(self._h, _ptr(wa)))
        return wa

    def spins(self, a_lo: int = 0, n_a: int | None = None) -> np.ndarray:
        n_a = self.n_samples - a_lo if n_a is None else n_a
        S = np.zeros((n_a, self.n_rep, self.n_slots, self.N), dtype=np.int8)
        _check(load().qisg_get_spins(self._h, a_lo, n_a, _ptr(S)))
        return S

    def couplings(self, a_lo: int = 0, n_a: int | None = None) -> np.ndarray:
        n_a = self.n_samples - a_lo if n_a is None else n_a
        J = np.zeros((n_a, self.L * self.L, 2), dtype=np.int8)
        _check(load().qisg_get_couplings(self._h, a_lo, n_a, _ptr(J)))
        return J

    def set_couplings(self, J: np.ndarray):
        J = _sized(J, np.int8, self.n_samples * self.L * self.L * 2, "J [n_samples][L*L][2]")
        _check(load().qisg_set_couplings(self._h, _ptr(J)))

    def set_state(self, S: np.ndarray, walker_at: np.ndarray, sweep: int):
        n_cs = self.n_samples * self.n_rep * self.n_slots
        S = _sized(S, np.int8, n_cs * self.N, "S [n_samples][n_replicas][n_slots][N]")
        wa = _sized(walker_at, np.int32, n_cs, "walker_at [n_samples][n_replicas][n_slots]")
        _check(load().qisg_set_state(self._h, _ptr(S), _ptr(wa), sweep))

    def pt_given(self, U: np.ndarray, walker_at: np.ndarray, t: int, wide: bool = False) -> np.ndarray:
        """One PT pass of the handle's PT kernel on given bond counts U
        [n_samples][n_replicas][n_slots walkers][2]; returns the permutation
        after the pass (test entry: the handle then needs set_state)."""
        n_cs = self.n_samples * self.n_rep * self.n_slots
        U = _sized(U, np.int64, n_cs * 2, "U [n_samples][n_replicas][n_slots][2]")
        wa = _sized(walker_at, np.int32, n_cs, "walker_at [n_samples][n_replicas][n_slots]").copy()
        _check(load().qisg_pt_given(self._h, _ptr(U), _ptr(wa), t, int(bool(wide))))
        return wa.reshape(self.n_samples, self.n_rep, self.n_slots)

    def measurements(self):
        ncs = (self.n_samples, self.n_rep, self.n_slots)
        nq = (self.n_samples, self.n_slots, max(self.n_pairs, 1))
        sA, sB = np.zeros(ncs, np.int64), np.zeros(ncs, np.int64)
        sq, sq2 = np.zeros(nq, np.int64), np.zeros(nq, np.int64)
        nm = ctypes.c_int64()
        _check(load().qisg_measurements(self._h, _ptr(sA), _ptr(sB), _ptr(sq), _ptr(sq2),
                                        ctypes.byref(nm)))
        return sA, sB, sq[:, :, : self.n_pairs], sq2[:, :, : self.n_pairs], nm.value

    def slot_means(self):
        e_s, e_t, q2 = (np.zeros(self.n_slots) for _ in range(3))
        _check(load().qisg_slot_means(self._h, _ptr(e_s), _ptr(e_t), _ptr(q2)))
        return e_s, e_t, q2

    def checkpoint_save(self, path: str):
        _check(load().qisg_checkpoint_save(self._h, os.fsencode(path)))

    def checkpoint_load(self, path: str):
        _check(load().qisg_checkpoint_load(self._h, os.fsencode(path)))

    def tau_observables(self, a_lo: int = 0, n_a: int | None = None):
        """Sums over tau_1 of Q~, Q~^2, Q~^4 and the squared Fourier moduli of
        q~ (Appendix E.1) for the configuration at every slot of samples
        a_lo .. a_lo+n_a-1: four arrays [n_a][n_replicas][n_slots][L_tau]."""
        n_a = self.n_samples - a_lo if n_a is None else n_a
        shp = (n_a, self.n_rep, self.n_slots, self.L_tau)
        S1, S2, S4 = (np.zeros(shp, dtype=np.int64) for _ in range(3))
        SF = np.zeros(shp, dtype=np.float64)
        _check(load().qisg_tau_observables(self._h, a_lo, n_a, _ptr(S1), _ptr(S2), _ptr(S4), _ptr(SF)))
        return S1, S2, S4, SF

    def walk_history(self, first: int, n: int) -> np.ndarray:
        """Slot of every walker at measurements first .. first+n-1:
        [n][n_samples][n_replicas][n_slots] uint8."""
        out = np.zeros((n, self.n_samples, self.n_rep, self.n_slots), dtype=np.uint8)
        _check(load().qisg_walk_history(self._h, first, n, _ptr(out)))
        return out

    def block_sums(self, first: int, n: int):
        """Sums of A and B over blocks first .. first+n-1 of maxit
        measurements: two int64 [n][n_samples][n_replicas][n_slots]."""
        A = np.zeros((n, self.n_samples, self.n_rep, self.n_slots), dtype=np.int64)
        B = np.zeros_like(A)
        _check(load().qisg_block_sums(self._h, first, n, _ptr(A), _ptr(B)))
        return A, B

    def block_means(self, first: int, n: int):
        e_s = np.zeros((n, self.n_slots))
        e_t = np.zeros((n, self.n_slots))
        _check(load().qisg_block_means(self._h, first, n, _ptr(e_s), _ptr(e_t)))
        return e_s, e_t

    def thresholds(self) -> np.ndarray:
        T = np.zeros((self.n_slots, 5, 3), dtype=np.uint32)
        _check(load().qisg_thresholds(self._h, _ptr(T)))
        return T

    def sweep_count(self) -> int:
        t = ctypes.c_uint64()
        _check(load().qisg_sweep_count(self._h, ctypes.byref(t)))
        return t.value

    def layout(self):
        lay, wb = ctypes.c_int(), ctypes.c_int()
        _check(load().qisg_layout(self._h, ctypes.byref(lay), ctypes.byref(wb)))
        return lay.value, wb.value

    def set_graphs(self, enable: bool):
        _check(load().qisg_set_graphs(self._h, 1 if enable else 0))

    def set_launch_overlap(self, enable: bool):
        """Programmatic dependent launch of the SAMPLES sweep kernels."""
        _check(load().qisg_set_launch_overlap(self._h, 1 if enable else 0))

    def set_pt_in_blue(self, enable: bool, wait_ns: int = 0):
        """Run each sweep's PT pass in the blue pass's last blocks (the default)."""
        _check(load().qisg_set_pt_in_blue(self._h, 1 if enable else 0, wait_ns))

    def set_persistent(self, enable: bool, wait_ns: int = 0):
        """One cooperative launch per run of sweeps (SAMPLES, 32-bit words)."""
        _check(load().qisg_set_persistent(self._h, 1 if enable else 0, wait_ns))

    def autotune(self, sweeps_per_candidate: int = 2) -> int:
        """Pick the fastest sweep tile on the live state (advances the run)."""
        g = ctypes.c_int()
        _check(load().qisg_autotune(self._h, sweeps_per_candidate, ctypes.byref(g)))
        return g.value

    def tiles(self):
        """((red tile, blue tile), (red variant, blue variant)) of the sweep schedule."""
        t, pf = (ctypes.c_int * 2)(), (ctypes.c_int * 2)()
        _check(load().qisg_get_tiles(self._h, t, pf))
        return (t[0], t[1]), (pf[0], pf[1])

    def set_tiles(self, tiles, variants=(0, 0)):
        t, pf = (ctypes.c_int * 2)(*tiles), (ctypes.c_int * 2)(*variants)
        _check(load().qisg_set_tiles(self._h, t, pf))

    def profile(self, enable: bool, kinds=None):
        """Time launches with event pairs; `kinds` limits it to those kernel kinds."""
        if not enable:
            code = 0
        elif kinds is None:
            code = 1
        else:
            code = PROFILE_ONLY
            for k in kinds:
                code |= 1 << int(k)
        _check(load().qisg_profile(self._h, code))

    def profile_read(self, kind: int):
        """(total ms, launches timed, launches) of one kernel kind."""
        ms, nt, nl = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
        _check(load().qisg_profile_read(self._h, kind, ctypes.byref(ms), ctypes.byref(nt),
                                        ctypes.byref(nl)))
        return ms.value, nt.value, nl.value

    def launch_count(self) -> int:
        n = ctypes.c_int64()
        _check(load().qisg_launch_count(self._h, ctypes.byref(n)))
        return n.value


def philox4x32_10_device(ctr_dev_ptr: int, key_dev_ptr: int, out_dev_ptr: int, n: int,
                         stream: int | None = None):
    """Device Philox on device buffers (pointers from torch tensors)."""
    _check(load().qisg_philox4x32_10(ctr_dev_ptr, key_dev_ptr, out_dev_ptr, n, stream))


def transfer_matvec(in_ptr: int, out_ptr: int, L: int, k: float, k_tau: float, J: np.ndarray, parity: int,
                    stream: int | None = None):
    """out = T in on a parity sector (device pointers of 2^(L^2-1) doubles,
    e.g. from torch tensors); J host int8 [L*L][2]."""
    Jc = _sized(J, np.int8, L * L * 2, "J [L*L][2]")
    _check(load().qisg_transfer_matvec(in_ptr, out_ptr, L, float(k), float(k_tau), _ptr(Jc), int(parity),
                                       stream if stream is not None else current_stream_ptr()))


class CheckpointInfo(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("L_tau", ctypes.c_int), ("n_slots", ctypes.c_int),
                ("n_replicas", ctypes.c_int), ("n_samples", ctypes.c_int64), ("seed", ctypes.c_uint64),
                ("sweep", ctypes.c_uint64), ("n_meas", ctypes.c_int64), ("pt_every", ctypes.c_int),
                ("measure_every", ctypes.c_int), ("tau_antiperiodic", ctypes.c_int), ("rule", ctypes.c_int)]


def checkpoint_verify(path: str) -> dict:
    """Header of a checkpoint file after its size and CRC checks (host only)."""
    info = CheckpointInfo()
    _check(load().qisg_checkpoint_verify(os.fsencode(path), ctypes.byref(info)))
    return {name: getattr(info, name) for name, _ in CheckpointInfo._fields_}


class InstanceDesc(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("L_tau", ctypes.c_int), ("n_slots", ctypes.c_int),
                ("n_replicas", ctypes.c_int), ("ladder", ctypes.c_void_p),
                ("seed", ctypes.c_uint64), ("n_sweeps", ctypes.c_int64), ("tau_antiperiodic", ctypes.c_int)]


def _desc(L, L_tau, ladder, n_replicas, seed, n_sweeps, tau_antiperiodic=0):
    lad = _ladder_array(ladder)
    d = InstanceDesc(L, L_tau, lad.shape[0], n_replicas, lad.ctypes.data, seed, n_sweeps, int(tau_antiperiodic))
    return d, lad


class Batch:
    """qisg_batch: independent single-sample instances of uneven size, advanced
    together by one persistent kernel per qisg_batch_run."""

    def __init__(self, capacity: int, mem_budget: int = 0, stream: int | None = None):
        lib = load()
        self._b = ctypes.c_void_p()
        _check(lib.qisg_batch_create(ctypes.byref(self._b), capacity, mem_budget,
                                     stream if stream is not None else current_stream_ptr()))
        self.meta = {}

    def close(self):
        if getattr(self, "_b", None) and self._b.value:
            load().qisg_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @staticmethod
    def instance_bytes(L, L_tau, ladder, n_replicas=4) -> int:
        d, _lad = _desc(L, L_tau, ladder, n_replicas, 0, 0)
        return int(load().qisg_batch_instance_bytes(ctypes.byref(d)))

    def admit(self, L, L_tau, ladder, n_replicas, seed, n_sweeps=0, tau_antiperiodic=0) -> int:
        """Slot of the admitted instance; raises QisgError(ENOMEM) when the
        arena or the slots are full."""
        d, lad = _desc(L, L_tau, ladder, n_replicas, seed, n_sweeps, tau_antiperiodic)
        slot = ctypes.c_int()
        _check(load().qisg_batch_admit(self._b, ctypes.byref(d), ctypes.byref(slot)))
        self.meta[slot.value] = (L, L_tau, lad.shape[0], n_replicas)
        return slot.value

    def try_admit(self, *a, **kw):
        try:
            return self.admit(*a, **kw)
        except QisgError as e:
            if e.code == -2:
                return None
            raise

    def retire(self, slot: int):
        _check(load().qisg_batch_retire(self._b, slot))
        self.meta.pop(slot, None)

    def run(self, n_sweeps: int):
        _check(load().qisg_batch_run(self._b, n_sweeps))

    def sync(self):
        _check(load().qisg_batch_sync(self._b))

    def set_schedule(self, tile_rows: int, schedule: int):
        _check(load().qisg_batch_set_schedule(self._b, tile_rows, schedule))

    def set_wait_limit(self, wait_ns: int):
        """Bound of each grid-barrier wait (0: the default)."""
        _check(load().qisg_batch_set_wait_limit(self._b, wait_ns))

    def autotune(self, sweeps_per_candidate: int = 2):
        r, s = ctypes.c_int(), ctypes.c_int()
        _check(load().qisg_batch_autotune(self._b, sweeps_per_candidate, ctypes.byref(r), ctypes.byref(s)))
        return r.value, s.value

    def status(self, slot: int):
        n, d = ctypes.c_uint64(), ctypes.c_int()
        _check(load().qisg_batch_status(self._b, slot, ctypes.byref(n), ctypes.byref(d)))
        return n.value, bool(d.value)

    def results(self, slot: int, spins: bool = False):
        L, Lt, n_slots, n_rep = self.meta[slot]
        A = np.zeros((n_rep, n_slots), dtype=np.int64)
        B = np.zeros_like(A)
        wa = np.zeros((n_rep, n_slots), dtype=np.int32)
        S = np.zeros((n_rep, n_slots, L * L * Lt), dtype=np.int8) if spins else None
        _check(load().qisg_batch_results(self._b, slot, _ptr(A), _ptr(B), _ptr(wa),
                                         _ptr(S) if spins else None))
        return A, B, wa, S

    def info(self):
        fb, fs, ln = ctypes.c_size_t(), ctypes.c_int(), ctypes.c_int64()
        _check(load().qisg_batch_info(self._b, ctypes.byref(fb), ctypes.byref(fs), ctypes.byref(ln)))
        return fb.value, fs.value, ln.value
