"""phia_create_from_device: a dense instance from device buffers (torch tensors).  Runs
are bit-identical to the same instance created from host arrays on every dense path,
and the device-side checks reject what phia_create rejects, with the same codes."""
import ctypes

import numpy as np
import pytest

from paper_2407_10205_gb300 import instances as ins

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _records(phia, A, R, N):
    return phia.replica_results(A.h, R, N)


@pytest.mark.parametrize("path,kern", [(1, 0), (1, 2), (2, 0)])
def test_device_instance_runs_like_host_instance(gpu_lib, path, kern):
    phia = gpu_lib
    N, R, T = 150, 64, 300
    d = ins.dense_int(N, 7, 7, seed=12)
    sched = phia.schedule(0.01, 0.3, 0.1, 2.0, refresh=40)
    Jd = torch.from_numpy(np.ascontiguousarray(d.k)).cuda()
    hd = torch.from_numpy(np.ascontiguousarray(d.kh.astype(np.int32))).cuda()
    out = []
    for J, h in ((d.k, d.kh), (Jd, hd)):
        with phia.Annealer(J, h, path=path, tc_kernel=kern) as A:
            res = A.anneal(sched, R, T, seed=9)
            out.append((res.energy_k, res.stats.tc_kernel, res.stats.operand, _records(phia, A, R, N)))
    assert out[0][:3] == out[1][:3]
    for u, v in zip(out[0][3], out[1][3]):
        assert np.array_equal(u, v)


def _expect(phia, code, J, h, **kw):
    with pytest.raises(phia.PhiaError) as ei:
        phia.Annealer(J, h, **kw)
    assert ei.value.code == code, str(ei.value)


def test_device_checks_reject_bad_instances(gpu_lib):
    phia = gpu_lib
    N = 70
    d = ins.dense_int(N, 7, 7, seed=2)
    k = np.ascontiguousarray(d.k)
    h = np.ascontiguousarray(d.kh.astype(np.int32))
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    # asymmetric at (3, 40)
    ka = k.copy(); ka[3, 40] = np.int8(ka[40, 3] + 1 if ka[40, 3] < 7 else ka[40, 3] - 1)
    _expect(phia, phia.EINVAL, dev(ka), dev(h))
    # nonzero diagonal
    kd = k.copy(); kd[5, 5] = 1
    _expect(phia, phia.EINVAL, dev(kd), dev(h))
    # |h| >= 2^24
    hb = h.copy(); hb[N - 1] = 1 << 24
    _expect(phia, phia.ERANGE, dev(k), dev(hb))
    # e4m3 forced with |k| = 17 (not exact in e4m3)
    kk = k.copy(); kk[1, 2] = kk[2, 1] = 17
    _expect(phia, phia.ERANGE, dev(kk), dev(h), path=phia.PATH_TC, operand=phia.OP_E4M3)
    # the same |k| = 17 instance is accepted with the automatic operand (bf16)
    with phia.Annealer(dev(kk), dev(h), path=phia.PATH_TC) as A:
        assert A.anneal(phia.schedule(0.01, 0.1, 0.1, 2.0), 8, 10, seed=1).stats.operand == phia.OP_BF16
    # host pointers are refused by the device entry point
    hptr = ctypes.c_void_p()
    rc = phia.load().phia_create_from_device(ctypes.byref(hptr), ctypes.c_void_p(k.ctypes.data),
                                             ctypes.c_void_p(h.ctypes.data), N, 0, None)
    assert rc == phia.EINVAL


def test_device_check_at_larger_n(gpu_lib):
    """N = 3000 (9 M couplings): the device check and the per-iteration kernel."""
    phia = gpu_lib
    N = 3000
    d = ins.sk_pm1(N, 4)
    Jd = torch.from_numpy(np.ascontiguousarray(d.k)).cuda()
    hd = torch.from_numpy(np.ascontiguousarray(d.kh.astype(np.int32))).cuda()
    with phia.Annealer(Jd, hd, path=phia.PATH_TC) as A, phia.Annealer(d.k, d.kh, path=phia.PATH_TC) as B:
        ra = A.anneal(phia.schedule(0.01, 0.1, 0.1, 2.0), 256, 20, seed=3)
        rb = B.anneal(phia.schedule(0.01, 0.1, 0.1, 2.0), 256, 20, seed=3)
        assert ra.energy_k == rb.energy_k and np.array_equal(ra.spins, rb.spins)
