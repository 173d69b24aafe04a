"""qisg_set_state refuses corrupt state buffers with QISG_ECORRUPT before any
device work, and leaves the handle's state as it was."""
from __future__ import annotations

import numpy as np
import pytest

from tests.gpu_util import make, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qisg():
    need_gpu()
    from paper_2402_03920_gb300 import qisg as q
    q.load()
    return q


@pytest.mark.parametrize("layout", ["LANES", "SAMPLES", "SITES"])
def test_set_state_rejects_corrupt_buffers(qisg, layout):
    lay = getattr(qisg, f"QISG_LAYOUT_{layout}")
    if layout == "SITES":
        ladder = qisg.ladder_equal(0.25, 0.45, 4)
        inst = qisg.Instance(qisg.Config(4, 64, ladder, 3, 5, 17, layout=lay))
    else:
        inst, _ = make(qisg, 4, 6, 0.2, 0.5, 4, 1.0, 3, 5, 17, layout=lay)
    with inst:
        inst.sweep(3)
        S0, wa0, (A0, B0), t0 = inst.spins(), inst.permutation(), inst.energies(), inst.sweep_count()
        cases = []
        wa = wa0.copy()
        wa[2, 1, 0] = wa[2, 1, 1]                 # a walker twice in one row
        cases.append((S0, wa))
        wa = wa0.copy()
        wa[4, 0, 3] = inst.n_slots                # a label out of range
        cases.append((S0, wa))
        wa = wa0.copy()
        wa[0, 2, 1] = -1
        cases.append((S0, wa))
        for bad in (0, 2, -3, 127):
            S = S0.copy()
            S[1, 2, 3, 5] = bad                   # a spin that is not +-1
            cases.append((S, wa0))
        for S, wa in cases:
            with pytest.raises(qisg.QisgError) as e:
                inst.set_state(S, wa, 99)
            assert e.value.code == -5, qisg.load().qisg_last_error()
        # nothing changed
        assert inst.sweep_count() == t0
        assert np.array_equal(inst.spins(), S0) and np.array_equal(inst.permutation(), wa0)
        A, B = inst.energies()
        assert np.array_equal(A, A0) and np.array_equal(B, B0)
        # a valid state is still taken
        inst.set_state(S0, wa0, t0)
        inst.sweep(1)
