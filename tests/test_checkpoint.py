"""Checkpoint save / load on the GPU: a saved run resumes bit for bit (also
in another packing), a file written from the oracle's state loads and then
follows the oracle, a saved file reads back as the oracle's state, and
corrupt or foreign files are refused without touching the handle."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from tests import checkpoint_format as ck
from tests.gpu_util import assert_same_state, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qisg():
    need_gpu()
    from paper_2402_03920_gb300 import qisg as q
    q.load()
    return q


def _cfg(qisg, layout, W, n_samples=40, seed=5, ap=0):
    ladder = qisg.ladder_linear(0.2, 0.5, 6, 1.0)
    lay = getattr(qisg, f"QISG_LAYOUT_{layout}")
    return qisg.Config(6, 8, ladder, 4, n_samples, seed, word_bits=W, layout=lay, measure_every=3,
                       tau_antiperiodic=ap), ladder


def _same(a, b):
    assert np.array_equal(a.spins(), b.spins())
    assert np.array_equal(a.permutation(), b.permutation())
    for x, y in zip(a.energies(), b.energies()):
        assert np.array_equal(x, y)
    for x, y in zip(a.measurements(), b.measurements()):
        assert np.array_equal(np.asarray(x), np.asarray(y))


@pytest.mark.parametrize("save_as,load_as", [(("SAMPLES", 32), ("LANES", 64)), (("LANES", 64), ("SAMPLES", 64)),
                                             (("SAMPLES", 64), ("SAMPLES", 32))])
def test_resume_is_bit_exact_across_packings(qisg, tmp_path, save_as, load_as):
    cfg_a, ladder = _cfg(qisg, *save_as, ap=1)
    cfg_b, _ = _cfg(qisg, *load_as, ap=1)
    p = str(tmp_path / "run.ckpt")
    with qisg.Instance(cfg_a) as a, qisg.Instance(cfg_b) as b:
        a.sweep(7)
        a.checkpoint_save(p)
        b.checkpoint_load(p)
        assert b.sweep_count() == 7
        _same(a, b)
        a.sweep(11)
        b.sweep(11)
        _same(a, b)
    # the file is the oracle's state after 7 sweeps
    st = oracle.new_state(6, 8, ladder[:, 0], ladder[:, 1], 4, 5, n_a=40, tau_ap=True)
    oracle.run(st, 7, pt_every=1, measure_every=3)
    got = ck.read(p)
    assert got["sweep"] == 7 and got["n_meas"] == st.n_meas
    assert np.array_equal(got["S"], st.S) and np.array_equal(got["walker_at"], st.walker_at)
    assert np.array_equal(got["J"], st.J)
    assert np.array_equal(got["sumA"], st.sumA) and np.array_equal(got["sumq2"], st.sumq2)


def test_oracle_written_file_loads_and_follows_the_oracle(qisg, tmp_path):
    cfg, ladder = _cfg(qisg, "SAMPLES", 32, n_samples=33, seed=8)
    st = oracle.new_state(6, 8, ladder[:, 0], ladder[:, 1], 4, 8, n_a=33)
    oracle.run(st, 13, pt_every=1, measure_every=3)
    # a state the handle never produced: random spins and permutations
    rng = np.random.default_rng(4)
    st.S = np.where(rng.random(st.S.shape) < 0.5, 1, -1).astype(np.int8)
    st.walker_at = np.argsort(rng.random(st.walker_at.shape), axis=2).astype(np.int32)
    oracle.refresh_energies(st)
    p = str(tmp_path / "oracle.ckpt")
    ck.write_oracle_state(p, st, measure_every=3)
    with qisg.Instance(cfg) as inst:
        inst.checkpoint_load(p)
        assert_same_state(inst, st, what="after load")
        inst.sweep(10)
        oracle.run(st, 10, pt_every=1, measure_every=3)
        assert_same_state(inst, st, what="10 sweeps after load")
        sA, sB, sq, sq2, nm = inst.measurements()
        assert nm == st.n_meas and np.array_equal(sA, st.sumA) and np.array_equal(sq2, st.sumq2)


def test_corrupt_and_foreign_files_are_refused(qisg, tmp_path):
    cfg, ladder = _cfg(qisg, "SAMPLES", 32)
    other, _ = _cfg(qisg, "SAMPLES", 32, seed=6)
    good = str(tmp_path / "good.ckpt")
    with qisg.Instance(cfg) as a, qisg.Instance(other) as b:
        a.sweep(4)
        a.checkpoint_save(good)
        b.sweep(2)
        S0, wa0, t0 = b.spins(), b.permutation(), b.sweep_count()
        data = bytearray(open(good, "rb").read())
        for i, cut in enumerate((len(data) // 3, len(data) - 1)):
            bad = bytearray(data)
            bad[cut] ^= 0x40
            path = str(tmp_path / f"bad{i}.ckpt")
            open(path, "wb").write(bytes(bad))
            with pytest.raises(qisg.QisgError) as e:
                b.checkpoint_load(path)
            assert e.value.code == -5
        with pytest.raises(qisg.QisgError) as e:    # another seed: another problem
            b.checkpoint_load(good)
        assert e.value.code == -1
        assert b.sweep_count() == t0 and np.array_equal(b.spins(), S0) and np.array_equal(b.permutation(), wa0)
