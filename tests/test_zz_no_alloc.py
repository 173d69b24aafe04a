"""The allocation-free overlap entry point against the oracle.

qisg_overlaps_noalloc exists for callers that cannot call cudaMalloc (a host
allocator that owns all device memory, a serving loop that must not stall on
an allocation): it counts in a scratch array compiled into the library.  The
configurations come from the CPU oracle (packed into the SAMPLES words here),
and the expected overlaps are the oracle's own measurement of them.  This
file is collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process, where
its first call performs the one-time look-up of the scratch address.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

import oracle
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def _pack_by_slot(S, wa, W):
    """SAMPLES packing [b][s][q][site][4] of spins by walker S[a][r][w][site]
    and the permutation wa[a][r][s]."""
    n_a, n_rep, n_slots, N = S.shape
    n_b, n_q = -(-n_a // W), -(-n_rep // 4)
    by_slot = np.take_along_axis(S, wa[:, :, :, None].astype(np.int64), axis=2)   # [a][r][s][N]
    bits = np.zeros((n_b * W, 4 * n_q, n_slots, N), dtype=np.uint64)
    bits[:n_a, :n_rep] = (by_slot == -1)
    bits = bits.reshape(n_b, W, n_q, 4, n_slots, N)
    words = np.zeros((n_b, n_slots, n_q, N, 4), dtype=np.uint64)
    for lane in range(W):
        words |= np.transpose(bits[:, lane], (0, 3, 1, 4, 2)) << np.uint64(lane)
    return words.astype(np.uint32 if W == 32 else np.uint64)


def _entry():
    from paper_2402_03920_gb300 import qisg
    lib = qisg.load()
    fn = lib.qisg_overlaps_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                   ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    return lib, fn


def _to_device(torch, words, W):
    view = words.view(np.int32 if W == 32 else np.int64)
    return torch.from_numpy(np.ascontiguousarray(view)).cuda()


# N = 6 * 6 * 128 = 4608 sites: two 4096-site chunks, the second ragged
@pytest.mark.parametrize("W,n_samples,n_rep", [(32, 40, 4), (64, 70, 5)])
def test_noalloc_overlaps_match_oracle(W, n_samples, n_rep):
    torch = need_gpu()
    lib, fn = _entry()
    L, Lt, n_slots, seed = 6, 128, 3, 31
    k, kt = oracle.ladder_linear(0.2, 0.5, n_slots, 1.0)
    st = oracle.new_state(L, Lt, k, kt, n_rep, seed, n_a=n_samples)
    stream = torch.cuda.current_stream()
    q_prev = np.zeros_like(st.sumq)
    # two calls in a row on different states; the oracle measures exactly once
    # at the end of each leg (measurement cadence = the sweep count so far)
    for call, n in enumerate((3, 4)):
        oracle.run(st, n, pt_every=1, measure_every=st.t + n)
        q_ref = st.sumq - q_prev
        q_prev = st.sumq.copy()
        d_words = _to_device(torch, _pack_by_slot(st.S, st.walker_at, W), W)
        q_dev = torch.full(q_ref.shape, -7, dtype=torch.int64, device="cuda")
        rc = fn(d_words.data_ptr(), W, L, Lt, n_slots, n_rep, n_samples, q_dev.data_ptr(),
                stream.cuda_stream)
        assert rc == 0, lib.qisg_last_error()
        torch.cuda.synchronize()
        assert np.array_equal(q_dev.cpu().numpy(), q_ref), f"call {call}"


def test_noalloc_many_slots_and_refusals():
    """More (sample block, slot) sets than one grid dimension holds, checked
    against the overlap's definition on random configurations; sizes beyond
    the scratch array are refused before any device work."""
    torch = need_gpu()
    lib, fn = _entry()
    L, Lt, n_slots, n_rep, W = 2, 2, 70000, 2, 32
    N = L * L * Lt
    rng = np.random.default_rng(5)
    S = np.where(rng.random((1, n_rep, n_slots, N)) < 0.5, 1, -1).astype(np.int8)
    wa = np.tile(np.arange(n_slots, dtype=np.int32), (1, n_rep, 1))
    q_ref = np.einsum("si,si->s", S[0, 0].astype(np.int64), S[0, 1].astype(np.int64)).reshape(1, n_slots, 1)
    d_words = _to_device(torch, _pack_by_slot(S, wa, W), W)
    q_dev = torch.full(q_ref.shape, -7, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    rc = fn(d_words.data_ptr(), W, L, Lt, n_slots, n_rep, 1, q_dev.data_ptr(), stream.cuda_stream)
    assert rc == 0, lib.qisg_last_error()
    torch.cuda.synchronize()
    assert np.array_equal(q_dev.cpu().numpy(), q_ref)
    # refused before any launch: q keeps its contents
    q_dev.fill_(-7)
    torch.cuda.synchronize()
    for n_samples, slots, reps in ((1 << 17, 32, 4), (1 << 40, 1, 2), (1, 1 << 20, 2)):
        rc = fn(d_words.data_ptr(), W, L, Lt, slots, reps, n_samples, q_dev.data_ptr(), stream.cuda_stream)
        assert rc == -1
    rc = fn(d_words.data_ptr() + 2, W, L, Lt, 4, n_rep, 1, q_dev.data_ptr(), stream.cuda_stream)
    assert rc == -1   # misaligned words
    torch.cuda.synchronize()
    assert bool((q_dev == -7).all())
