"""Writer and reader of the checkpoint file format documented in
include/qisg.h, written from that description (tests only): a file made here
from the oracle's state must load into a handle, and a file the library
writes must read back as the oracle's state."""
from __future__ import annotations

import struct
import zlib

import numpy as np

MAGIC = b"QISGCKP1"
HEADER = struct.Struct("<8sII4iqQQq4i")   # 80 bytes, zero padded to 128


def write(path, *, L, L_tau, k, ktau, n_rep, seed, sweep, J, S, walker_at, sumA, sumB, sumq, sumq2, n_meas,
          pt_every=1, measure_every=0, tau_ap=0, rule=0, corrupt=None):
    """S [n_a][n_rep][n_slots][N] int8 by walker; J [n_a][L*L][2] int8."""
    n_a, _, n_slots, N = S.shape
    head = HEADER.pack(MAGIC, 1, 128, L, L_tau, n_slots, n_rep, n_a, seed, sweep, n_meas, pt_every, measure_every,
                       tau_ap, rule)
    head += b"\0" * (128 - len(head))
    lad = b"".join(struct.pack("<dd", float(a), float(b)) for a, b in zip(k, ktau))
    bits = np.packbits((S.reshape(-1) == -1).astype(np.uint8), bitorder="little").tobytes()
    body = (head + lad + np.ascontiguousarray(J, dtype=np.int8).tobytes() + bits
            + np.ascontiguousarray(walker_at, dtype="<i4").tobytes()
            + np.ascontiguousarray(sumA, dtype="<i8").tobytes() + np.ascontiguousarray(sumB, dtype="<i8").tobytes()
            + np.ascontiguousarray(sumq, dtype="<i8").tobytes() + np.ascontiguousarray(sumq2, dtype="<i8").tobytes())
    data = body + struct.pack("<I", zlib.crc32(body) & 0xFFFFFFFF)
    if corrupt is not None:
        data = corrupt(bytearray(data))
    with open(path, "wb") as f:
        f.write(bytes(data))


def write_oracle_state(path, st, pt_every=1, measure_every=0, **kw):
    n_pairs = st.n_rep * (st.n_rep - 1) // 2
    write(path, L=st.L, L_tau=st.Ltau, k=st.k, ktau=st.ktau, n_rep=st.n_rep, seed=st.seed, sweep=st.t, J=st.J,
          S=st.S, walker_at=st.walker_at, sumA=st.sumA, sumB=st.sumB, sumq=st.sumq[:, :, :n_pairs],
          sumq2=st.sumq2[:, :, :n_pairs], n_meas=st.n_meas, pt_every=pt_every, measure_every=measure_every,
          tau_ap=int(st.tau_ap), rule=int(st.cum is not None), **kw)


def read(path) -> dict:
    data = open(path, "rb").read()
    body, crc = data[:-4], struct.unpack("<I", data[-4:])[0]
    assert zlib.crc32(body) & 0xFFFFFFFF == crc, "CRC mismatch"
    (magic, ver, hb, L, Lt, n_slots, n_rep, n_a, seed, sweep, n_meas, pt_every, measure_every, tau_ap,
     rule) = HEADER.unpack_from(body, 0)
    assert magic == MAGIC and ver == 1 and hb == 128
    N = L * L * Lt
    n_pairs = n_rep * (n_rep - 1) // 2
    o = 128
    lad = np.frombuffer(body, dtype="<f8", count=2 * n_slots, offset=o).reshape(n_slots, 2)
    o += 16 * n_slots
    J = np.frombuffer(body, dtype=np.int8, count=n_a * L * L * 2, offset=o).reshape(n_a, L * L, 2)
    o += J.size
    n_bits = n_a * n_rep * n_slots * N
    nb = (n_bits + 7) // 8
    bits = np.unpackbits(np.frombuffer(body, dtype=np.uint8, count=nb, offset=o), bitorder="little")[:n_bits]
    S = np.where(bits == 1, -1, 1).astype(np.int8).reshape(n_a, n_rep, n_slots, N)
    o += nb
    rows = n_a * n_rep * n_slots
    wa = np.frombuffer(body, dtype="<i4", count=rows, offset=o).reshape(n_a, n_rep, n_slots)
    o += 4 * rows
    sums = []
    for cnt, shape in ((rows, (n_a, n_rep, n_slots)), (rows, (n_a, n_rep, n_slots)),
                       (n_a * n_slots * n_pairs, (n_a, n_slots, n_pairs)), (n_a * n_slots * n_pairs, (n_a, n_slots, n_pairs))):
        sums.append(np.frombuffer(body, dtype="<i8", count=cnt, offset=o).reshape(shape))
        o += 8 * cnt
    assert o == len(body)
    return dict(L=L, L_tau=Lt, ladder=lad, seed=seed, sweep=sweep, n_meas=n_meas, J=J, S=S, walker_at=wa,
                sumA=sums[0], sumB=sums[1], sumq=sums[2], sumq2=sums[3], pt_every=pt_every,
                measure_every=measure_every, tau_ap=tau_ap, rule=rule)
