"""Checkpoint files checked on the host (no GPU): the library's verification
accepts a file written from the documented format (CRC from zlib, the
state from the oracle) and refuses every corrupted variant with
QISG_ECORRUPT before touching any device."""
from __future__ import annotations

import struct
import zlib

import pytest

import oracle
from tests import checkpoint_format as ck


@pytest.fixture(scope="module")
def qisg():
    from paper_2402_03920_gb300 import qisg as q
    q.load()
    return q


@pytest.fixture(scope="module")
def state():
    k, kt = oracle.ladder_linear(0.2, 0.5, 5, 1.0)
    st = oracle.new_state(4, 6, k, kt, 3, 99, n_a=2)
    oracle.run(st, 9, pt_every=1, measure_every=4)
    return st


def _refit_crc(buf: bytearray) -> bytearray:
    body = bytes(buf[:-4])
    buf[-4:] = struct.pack("<I", zlib.crc32(body) & 0xFFFFFFFF)
    return buf


def test_verify_accepts_a_file_from_the_documented_format(qisg, state, tmp_path):
    p = tmp_path / "ok.ckpt"
    ck.write_oracle_state(p, state, measure_every=4)
    info = qisg.checkpoint_verify(str(p))
    assert (info["L"], info["L_tau"], info["n_slots"], info["n_replicas"], info["n_samples"]) == (4, 6, 5, 3, 2)
    assert info["seed"] == 99 and info["sweep"] == 9 and info["n_meas"] == 2 and info["measure_every"] == 4
    back = ck.read(p)
    assert back["sweep"] == 9 and (back["S"] == state.S).all() and (back["walker_at"] == state.walker_at).all()


@pytest.mark.parametrize("how", ["flip_body", "flip_crc", "truncate", "append", "magic", "version",
                                 "padding", "sizes", "empty"])
def test_verify_refuses_corrupt_files(qisg, state, tmp_path, how):
    def corrupt(b: bytearray):
        if how == "flip_body":
            b[len(b) // 2] ^= 0x10
        elif how == "flip_crc":
            b[-1] ^= 0x01
        elif how == "truncate":
            b = b[:-1]
        elif how == "append":
            b = b + b"\0"
        elif how == "magic":
            b[0] = ord("X")
            b = _refit_crc(b)
        elif how == "version":
            b[8] = 2
            b = _refit_crc(b)
        elif how == "padding":
            b[100] = 1
            b = _refit_crc(b)
        elif how == "sizes":
            b[24] = 200            # n_slots beyond the limit
            b = _refit_crc(b)
        elif how == "empty":
            b = bytearray()
        return b
    p = tmp_path / f"{how}.ckpt"
    ck.write_oracle_state(p, state, measure_every=4, corrupt=corrupt)
    with pytest.raises(qisg.QisgError) as e:
        qisg.checkpoint_verify(str(p))
    assert e.value.code == -5, how


def test_verify_missing_file(qisg, tmp_path):
    with pytest.raises(qisg.QisgError) as e:
        qisg.checkpoint_verify(str(tmp_path / "absent.ckpt"))
    assert e.value.code == -1
