"""The allocation-free overlap entry point against qisg_overlaps.

qisg_overlaps_noalloc exists for callers that cannot call cudaMalloc (a host
allocator that owns all device memory, a serving loop that must not stall on
an allocation): it counts in a scratch array compiled into the library.  This
file is collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process, where
its first call performs the one-time look-up of the scratch address.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

from tests.gpu_util import make, need_gpu

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


@pytest.mark.parametrize("W,n_samples,n_rep", [(32, 40, 4), (64, 70, 5)])
def test_noalloc_overlaps_match_handle(W, n_samples, n_rep):
    torch = need_gpu()
    from paper_2402_03920_gb300 import qisg
    lib = qisg.load()
    fn = lib.qisg_overlaps_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                   ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    L, Lt, n_slots = 4, 8, 6
    inst, _ = make(qisg, L, Lt, 0.2, 0.5, n_slots, 1.0, n_rep, n_samples, 31,
                   layout=qisg.QISG_LAYOUT_SAMPLES, word_bits=W)
    stream = torch.cuda.current_stream()
    with inst:
        for call in range(2):              # two calls in a row on different states
            inst.sweep(3 + call)
            q_ref = inst.overlaps()
            words = _pack_by_slot(inst.spins(), inst.permutation(), W)
            view = words.view(np.int32 if W == 32 else np.int64)
            d_words = torch.from_numpy(np.ascontiguousarray(view)).cuda()
            q_dev = torch.full(q_ref.shape, -7, dtype=torch.int64, device="cuda")
            rc = fn(d_words.data_ptr(), W, L, Lt, n_slots, n_rep, n_samples, q_dev.data_ptr(),
                    stream.cuda_stream)
            assert rc == 0, lib.qisg_last_error()
            torch.cuda.synchronize()
            assert np.array_equal(q_dev.cpu().numpy(), q_ref), f"call {call}"
        # sizes beyond the scratch array are refused before any device work
        big = 1 << 17
        rc = fn(d_words.data_ptr(), W, L, Lt, 32, 4, big, q_dev.data_ptr(), stream.cuda_stream)
        assert rc == -1
