"""The PT kernels against the oracle on decisions placed next to their
acceptance boundary (Sec. 2.1: exchange iff u < P).

The kernels decide most pairs with a float comparison of ln u and ln P and
send the ones inside a margin to the exact power chain.  Here bond counts are
chosen (tests/pt_targets.py) so that ln P falls at, inside, just inside and
just outside that margin (0, 0.3, 0.9, 0.99, 1.01, 1.1, 1.5 and 3 times it,
both sides), at random, and where a factor overflows or underflows, for
small and large |m|, |n| and both energy widths.  qisg_pt_given runs one pass
of the handle's own PT kernel (LANES: by walker, SAMPLES: by slot with the
lane masks) on them; the permutation must equal the oracle's, chain by
chain.  Over all cases and both sweep counters this is more than 10^6
decisions.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from tests import pt_targets as P
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qisg():
    need_gpu()
    from paper_2402_03920_gb300 import qisg as q
    q.load()
    return q


def _ladder(spec):
    if spec[0] == "linear":
        return oracle.ladder_linear(*spec[1:])
    return np.asarray(spec[0], dtype=np.float64), np.asarray(spec[1], dtype=np.float64)


CASES = [
    # name, layout, word bits, ladder, samples, replicas, wide, scan j, count range
    ("lanes-tiny", "LANES", 32, ([0.3, 0.3 + 3.7e-6], [0.5, 0.5 - 2.9e-6]), 1024, 32, 0, False, 2 ** 29),
    ("lanes-mid", "LANES", 32, ([0.3, 0.3 + 1.3e-4], [0.5, 0.5 - 0.9e-4]), 1024, 32, 0, False, 2 ** 29),
    ("lanes-wide", "LANES", 32, ([0.3, 0.3 + 2.1e-9], [0.5, 0.5 - 1.7e-9]), 1024, 32, 1, False, 2 ** 38),
    ("lanes-far", "LANES", 32, ([0.3, 0.3 + 1e-7], [0.5, 0.5 - 1.3e-7]), 512, 32, 1, False, 2 ** 38),
    ("lanes-ladder32", "LANES", 64, ("linear", 0.2, 0.5, 32, 1.0), 2048, 4, 0, True, 2 ** 29),
    ("samples32-ladder32", "SAMPLES", 32, ("linear", 0.2, 0.5, 32, 1.0), 1024, 4, 0, True, 2 ** 29),
    ("samples64-ladder16", "SAMPLES", 64, ("linear", 0.2, 0.5, 16, 0.9), 1000, 5, 0, True, 2 ** 29),
    ("samples64-wide", "SAMPLES", 64, ([0.3 + 2.1e-9 * s for s in range(8)], [0.5 - 1.7e-9 * s for s in range(8)]),
     256, 4, 1, False, 2 ** 38),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_pt_kernel_decisions_match_oracle(qisg, case):
    name, layout, W, spec, n_samples, n_rep, wide, scan, lim = case
    k, kt = _ladder(spec)
    ladder = np.stack([k, kt], axis=1)
    seed = 0x51_7E_ED_01 + len(k)
    lay = qisg.QISG_LAYOUT_LANES if layout == "LANES" else qisg.QISG_LAYOUT_SAMPLES
    rng = np.random.default_rng(len(name))
    n_dec = 0
    near_band = 0
    with qisg.Instance(qisg.Config(2, 2, ladder, n_rep, n_samples, seed, word_bits=W, layout=lay)) as inst:
        assert inst.layout() == (lay, W)
        for t in (7, 123456):
            U, wa0, rel = P.make_case(k, kt, n_samples, n_rep, seed, t, rng, lim, scan)
            got = inst.pt_given(U, wa0, t, wide=bool(wide))
            want = P.oracle_pass(k, kt, seed, t, U, wa0)
            bad = np.argwhere(np.any(got != want, axis=2))
            assert len(bad) == 0, (f"{name} t={t}: {len(bad)} chains differ, first {bad[:3].tolist()}: "
                                   f"got {got[tuple(bad[0])]} want {want[tuple(bad[0])]}")
            n_dec += n_samples * n_rep * (len(k) - 1)
            near_band += int(np.sum((np.abs(rel) > 0.9) & (np.abs(rel) < 1.6)))
        # the handle refuses to sweep on energies it did not count
        with pytest.raises(qisg.QisgError):
            inst.sweep(1)
    assert near_band > 0.1 * n_dec * 0.6 / 2   # decisions at the margin's edge were exercised


def test_pt_given_refuses_bad_input(qisg):
    ladder = np.stack(oracle.ladder_linear(0.2, 0.5, 4, 1.0), axis=1)
    with qisg.Instance(qisg.Config(2, 2, ladder, 2, 3, 9, layout=qisg.QISG_LAYOUT_LANES)) as inst:
        U = np.zeros((3, 2, 4, 2), dtype=np.int64)
        wa = np.tile(np.arange(4, dtype=np.int32), (3, 2, 1))
        bad = wa.copy()
        bad[1, 0, 2] = bad[1, 0, 1]
        with pytest.raises(qisg.QisgError) as e:
            inst.pt_given(U, bad, 0)
        assert e.value.code == -5
        big = U.copy()
        big[0, 0, 0, 0] = 1 << 29
        with pytest.raises(qisg.QisgError) as e:
            inst.pt_given(big, wa, 0)
        assert e.value.code == -1
        inst.pt_given(big, wa, 0, wide=True)   # allowed with 64-bit differences
