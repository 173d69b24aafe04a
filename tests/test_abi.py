"""The C-ABI library builds, loads and exports every entry point declared in
include/qisg.h (no GPU needed: nothing here launches a kernel)."""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(qisg_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("qisg_create", "qisg_sweep", "qisg_pt_swap", "qisg_energies", "qisg_overlaps",
                 "qisg_permutation", "qisg_get_spins", "qisg_set_state", "qisg_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2402_03920_gb300 import _build_lib
    path = _build_lib.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2402_03920_gb300 import qisg
    assert set(qisg.exported_symbols()) <= _declared()


def test_host_only_entry_points_without_gpu():
    """Argument checks and host tables need no device."""
    import numpy as np
    from paper_2402_03920_gb300 import qisg
    import oracle
    lad = qisg.ladder_linear(0.2, 0.5, 16, 1.0)
    k, kt = oracle.ladder_linear(0.2, 0.5, 16, 1.0)
    # the library's FP64 ladder is the oracle's, bit for bit
    assert np.array_equal(lad[:, 0], k) and np.array_equal(lad[:, 1], kt)
    with pytest.raises(qisg.QisgError):
        qisg.ladder_linear(0.2, 0.5, 0, 1.0)
    lib = qisg.load()
    h = ctypes.c_void_p()
    sl = np.ascontiguousarray(lad)
    # odd L is rejected before any device work
    rc = lib.qisg_create(ctypes.byref(h), 7, 32, sl.ctypes.data_as(ctypes.c_void_p), 16, 4, 1, 1, None)
    assert rc == -1
    rc = lib.qisg_create(ctypes.byref(h), 8, 31, sl.ctypes.data_as(ctypes.c_void_p), 16, 4, 1, 1, None)
    assert rc == -1
    assert lib.qisg_strerror(-4) == b"bounded device wait expired"


def test_daemon_tables_host_without_gpu():
    """The daemon rule's host tables (fixed point, 126 fractional bits) equal
    the oracle's (decimal arithmetic) bit for bit, and a SITES handle with
    unequal couplings or an unfit L_tau is refused before any device work."""
    import numpy as np
    from paper_2402_03920_gb300 import qisg
    import oracle
    for k in (0.0, 0.05, 0.2, 0.29, 0.4137, 0.5, 1.7, 16.0):
        cum, _ = qisg.daemon_tables(k, 12)
        assert np.array_equal(cum, oracle.daemon_cumulative(k)), k
    lib = qisg.load()
    h = ctypes.c_void_p()
    opts = qisg.Opts()
    lib.qisg_opts_default(ctypes.byref(opts))
    opts.layout = qisg.QISG_LAYOUT_SITES
    unequal = np.ascontiguousarray(qisg.ladder_linear(0.2, 0.5, 4, 1.0))
    equal = np.ascontiguousarray(qisg.ladder_equal(0.2, 0.5, 4))
    rc = lib.qisg_create(ctypes.byref(h), 4, 64, unequal.ctypes.data_as(ctypes.c_void_p), 4, 2, 1, 1,
                         ctypes.byref(opts))
    assert rc == -1
    rc = lib.qisg_create(ctypes.byref(h), 4, 96, equal.ctypes.data_as(ctypes.c_void_p), 4, 2, 1, 1,
                         ctypes.byref(opts))
    assert rc == -1


def test_binding_rejects_misshapen_host_arrays():
    """The library reads exactly the documented number of elements from each
    host pointer, so the binding refuses arrays of another size or shape
    before the call."""
    from paper_2402_03920_gb300 import qisg
    assert qisg._sized(np.ones((2, 3), np.int64), np.int8, 6, "x").dtype == np.int8
    with pytest.raises(ValueError):
        qisg._sized(np.ones(5, np.int8), np.int8, 6, "x")
    assert qisg._ladder_array([[0.2, 0.3], [0.4, 0.5]]).shape == (2, 2)
    for bad in ([0.2, 0.3], np.zeros((2, 3)), np.zeros((0, 2))):
        with pytest.raises(ValueError):
            qisg._ladder_array(bad)
