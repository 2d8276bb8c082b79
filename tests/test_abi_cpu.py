"""C ABI and host-logic tests that need no GPU.

The library must load and export every symbol include/phia.h declares; argument
validation happens on the host before any device work, so its error paths are
exercised here without a GPU.
"""
import os
import re
import threading

import numpy as np
import pytest

from conftest import ROOT
from paper_2407_10205_gb300 import build as pbuild
from paper_2407_10205_gb300 import instances as ins
from paper_2407_10205_gb300 import phia


@pytest.fixture(scope="module")
def lib():
    pbuild.build()
    return phia.load()


def _declared_symbols():
    txt = open(os.path.join(ROOT, "include", "phia.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(phia_[a-z_]+)\s*\(", txt)))


def test_header_symbols_exported(lib):
    names = _declared_symbols()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/phia.h but not exported"
    assert set(names) == set(phia.SIGNATURES), "binding and header disagree"


def _create_rc(lib, J, h, frac=0, o=None):
    import ctypes
    J = np.ascontiguousarray(J, dtype=np.int8)
    h = np.ascontiguousarray(h, dtype=np.int32)
    out = ctypes.c_void_p()
    rc = lib.phia_create(ctypes.byref(out), J.ctypes.data_as(ctypes.c_void_p),
                         h.ctypes.data_as(ctypes.c_void_p), h.shape[0], frac,
                         ctypes.byref(o) if o is not None else None)
    return rc, out


def test_invalid_instances_rejected(lib):
    d = ins.dense_int(10, 5, 5, seed=1)
    J = d.k.copy(); J[2, 7] += 1
    assert _create_rc(lib, J, d.kh)[0] == phia.EINVAL
    assert "symmetric" in phia.last_error()
    J = d.k.copy(); J[3, 3] = 1
    assert _create_rc(lib, J, d.kh)[0] == phia.EINVAL
    assert "diagonal" in phia.last_error()
    h = d.kh.copy(); h[0] = 1 << 24
    assert _create_rc(lib, d.k, h)[0] == phia.ERANGE
    assert _create_rc(lib, d.k, d.kh, frac=31)[0] == phia.EINVAL
    big = ins.dense_int(10, 100, 5, seed=2)
    o = phia.opts(path=phia.PATH_TC, operand=phia.OP_E4M3)
    assert _create_rc(lib, big.k, big.kh, o=o)[0] == phia.ERANGE
    assert "e4m3" in phia.last_error()


def test_large_dense_check_reports_the_first_mismatch(lib):
    """From N = 1024 the host splits the symmetry check over its cores; the mismatch it
    reports is still the first in the serial scan (tile rows of 64, then tile columns,
    then rows and columns), whichever thread finds a mismatch first."""
    d = ins.dense_int(1500, 7, 7, seed=4)
    k = d.k.copy()
    for (i, j) in ((1400, 1450), (700, 900), (65, 1300)):   # tile rows 21, 10 and 1
        k[i, j] = np.int8(k[j, i] + 1)
    for _ in range(3):
        assert _create_rc(lib, k, d.kh)[0] == phia.EINVAL
        assert phia.last_error() == "J_k is not symmetric at (65, 1300)"
    k2 = d.k.copy()
    k2[5, 7] = np.int8(k2[7, 5] - 1)                      # tile row 0, tile column 0
    k2[3, 1499] = np.int8(k2[1499, 3] + 1)                # tile row 0, a later tile column
    assert _create_rc(lib, k2, d.kh)[0] == phia.EINVAL
    assert phia.last_error() == "J_k is not symmetric at (5, 7)"


def _batch_rc(lib, insts):
    import ctypes
    descs = (phia.InstanceDesc * len(insts))()
    keep = []
    for k, c in enumerate(insts):
        arrs = [np.ascontiguousarray(c.row_ptr, np.int32), np.ascontiguousarray(c.col, np.int32),
                np.ascontiguousarray(c.val, np.int8), np.ascontiguousarray(c.kh, np.int32)]
        keep.append(arrs)
        descs[k] = phia.InstanceDesc(c.n, c.frac_bits, None, *(a.ctypes.data for a in arrs), k, 0, 0)
    out = ctypes.c_void_p()
    return lib.phia_batch_create(ctypes.byref(out), len(insts), descs, None)


def test_batch_reports_first_invalid_instance(lib):
    """Batch instances are checked in parallel on the host (before any device call); the
    lowest-numbered failing instance is the one reported, whatever the thread order."""
    insts = [ins.erdos_renyi(60 + 7 * k, 0.1, 127, 31, 4, seed=k) for k in range(24)]
    for bad in (17, 5, 21):              # asymmetric value in three instances
        c = insts[bad]
        c.val[0] = np.int8(c.val[0] + 1 if c.val[0] < 100 else c.val[0] - 1)
    for _ in range(5):
        assert _batch_rc(lib, insts) == phia.EINVAL
        assert phia.last_error().startswith("instance 5: CSR is not symmetric")
    c = insts[2]
    c.kh[3] = 1 << 24                    # now instance 2 fails first, with ERANGE
    assert _batch_rc(lib, insts) == phia.ERANGE
    assert phia.last_error().startswith("instance 2:")


def test_zero_spins_rejected(lib):
    import ctypes
    out = ctypes.c_void_p()
    h = np.zeros(1, dtype=np.int32)
    rc = lib.phia_create(ctypes.byref(out), None, h.ctypes.data_as(ctypes.c_void_p), 0, 0, None)
    assert rc == phia.EINVAL


def test_last_error_is_thread_local(lib):
    d = ins.dense_int(6, 3, 3, seed=3)
    J = d.k.copy(); J[0, 1] += 1
    assert _create_rc(lib, J, d.kh)[0] == phia.EINVAL
    seen = {}

    def other():
        seen["msg"] = phia.last_error()

    t = threading.Thread(target=other); t.start(); t.join()
    assert seen["msg"] == ""
    assert "symmetric" in phia.last_error()


def test_null_handle_calls_fail_cleanly(lib):
    s = phia.schedule(0.1, 1.0, 0.1, 2.0)
    import ctypes
    assert lib.phia_anneal(None, ctypes.byref(s), 4, 10, 1) == phia.EINVAL
    assert lib.phia_best(None, None, None) == phia.EINVAL
    assert lib.phia_sync(None) == phia.EINVAL
    lib.phia_destroy(None)


def test_unpack_bits():
    S = ins.random_spins(5, 70, seed=4)
    W = 3
    bits = np.zeros((5, W), dtype=np.uint32)
    for r in range(5):
        for i in range(70):
            if S[r, i] > 0:
                bits[r, i // 32] |= np.uint32(1 << (i % 32))
    assert np.array_equal(phia.unpack_bits(bits, 70), S)


def test_instance_generators():
    d = ins.sk_pm1(50, seed=1)
    assert np.array_equal(d.k, d.k.T) and not np.diag(d.k).any()
    assert set(np.unique(d.k[~np.eye(50, dtype=bool)])) == {-1, 1}
    d2 = ins.dense_int(60, 7, 7, seed=2)
    assert d2.k.min() >= -7 and d2.k.max() <= 7 and np.array_equal(d2.k, d2.k.T)
    c = ins.erdos_renyi(400, 0.05, 127, 31, 4, seed=3)
    dd = c.to_dense()
    assert np.array_equal(dd.k, dd.k.T) and not np.diag(dd.k).any()
    dens = c.nnz / (400 * 399)
    assert 0.04 < dens < 0.06
    assert all(np.all(np.diff(c.col[c.row_ptr[i]:c.row_ptr[i + 1]]) > 0) for i in range(400))
    b = ins.batched_er(6, seed=4)
    assert all(100 <= x.n <= 3000 for x in b)
    reqs = ins.serving_stream(20, seed=5)
    assert all(reqs[i].arrival_s < reqs[i + 1].arrival_s for i in range(19))
    assert all(64 <= r.instance.n <= 8192 for r in reqs)
