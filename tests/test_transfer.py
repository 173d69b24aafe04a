"""The transfer-matrix product on the GPU (Sec. 2.2, Appendix D) against the
oracle's round-by-round product: both sectors, every lattice size one GPU
holds (2 <= L <= 5, so one, two and three passes over HBM), in place and out
of place, equal and separate couplings.

The kernel evaluates each round as y + jP (x - y) with fused multiply-adds
(jP + jM = 1), the oracle as jP x + jM y: the two differ by rounding.  Each
of the L^2 + 1 steps is a convex combination (jP, jM in (0, 1)), so it adds
at most a few units of 2^-53 of the vector's norm; the test bound,
1e-13 in the max norm relative to the result's max norm, is about 500 such
units for the 26 steps at L = 5 (the 1e-12 relative bound stated for FP64
results, with margin)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L,k,kt,parity,inplace", [(2, 0.3, 0.7, 1, False), (3, 0.29, 0.29, -1, True),
                                                   (4, 0.45, 0.2, 1, False), (4, 0.29, 0.29, -1, True),
                                                   (5, 0.29, 0.29, 1, False), (5, 0.35, 0.5, -1, True)])
def test_transfer_matvec_matches_oracle(L, k, kt, parity, inplace):
    torch = need_gpu()
    from paper_2402_03920_gb300 import qisg
    J = oracle.init_couplings(L, 0, 1, 100 + L)[0]
    n = 1 << (L * L - 1)
    v = np.random.default_rng(L).standard_normal(n)
    want = oracle.transfer_matvec(L, k, kt, J, parity, v)
    d_in = torch.from_numpy(v).cuda()
    d_out = d_in if inplace else torch.empty_like(d_in)
    qisg.transfer_matvec(d_in.data_ptr(), d_out.data_ptr(), L, k, kt, J, parity)
    torch.cuda.synchronize()
    got = d_out.cpu().numpy()
    assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want))


def test_transfer_power_iteration_and_refusals():
    """The leading eigenvalue of the even sector at L = 3 by power iteration
    on the GPU product equals the oracle's; invalid calls are refused."""
    torch = need_gpu()
    from paper_2402_03920_gb300 import qisg
    L, k = 3, 0.29
    J = oracle.init_couplings(L, 0, 1, 5)[0]
    v = torch.ones(1 << 8, dtype=torch.float64, device="cuda")
    w = np.ones(1 << 8)
    for _ in range(200):
        qisg.transfer_matvec(v.data_ptr(), v.data_ptr(), L, k, k, J, 1)
        v /= torch.linalg.norm(v)
        w = oracle.transfer_matvec(L, k, k, J, 1, w)
        w /= np.linalg.norm(w)
    u = torch.empty_like(v)
    qisg.transfer_matvec(v.data_ptr(), u.data_ptr(), L, k, k, J, 1)
    lam_gpu = float(torch.dot(u, v))
    lam = float(w @ oracle.transfer_matvec(L, k, k, J, 1, w))
    assert lam_gpu == pytest.approx(lam, rel=1e-12)
    for bad_L, bad_parity in ((6, 1), (1, 1), (3, 0)):
        Jb = np.ones((bad_L * bad_L, 2), dtype=np.int8)
        with pytest.raises(qisg.QisgError) as e:
            qisg.transfer_matvec(v.data_ptr(), u.data_ptr(), bad_L, k, k, Jb, bad_parity)
        assert e.value.code == -1
    Jz = J.copy()
    Jz[0, 0] = 0                       # a coupling that is not +-1
    with pytest.raises(qisg.QisgError):
        qisg.transfer_matvec(v.data_ptr(), u.data_ptr(), L, k, k, Jz, 1)
