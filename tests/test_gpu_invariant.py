"""At beta = 0 the update of Eq. A7 is the map x' = x + eps v, v' = v - eps x', which
keeps x^2 + v^2 + eps x v exactly in exact arithmetic (pinned in FP64 on the oracle).
On the GPU, every path run for 10^4 iterations keeps it within FP32 drift.

Tolerance: a plain FP32 simulation of the same map on these inputs (fused multiply-adds,
one rounding per line) drifts by at most 1.1e-4 absolute, 1.8e-5 relative, after 10^4
steps; the test allows ten times that, |dH| <= 1e-3 max(H0, 1)."""
import numpy as np
import pytest

from paper_2407_10205_gb300 import instances as ins

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

T, EPS = 10_000, 0.1


def _invariant(x, v):
    e = np.float64(np.float32(EPS))
    x, v = x.astype(np.float64), v.astype(np.float64)
    return x * x + v * v + e * x * v


def _check(phia, A, R, N):
    x, v = ins.random_state(R, N, seed=9)
    H0 = _invariant(x, v)
    xt, vt = torch.from_numpy(x).cuda(), torch.from_numpy(v).cuda()
    phia.run(A.h, phia.schedule(0.0, 0.0, EPS, 2.0), R, 0, T, T, 3, xt, vt)
    torch.cuda.synchronize()
    xg, vg = xt.cpu().numpy(), vt.cpu().numpy()
    assert np.all(np.isfinite(xg)) and np.all(np.isfinite(vg))
    assert np.abs(xg - x).max() > 0.1            # the state moved
    dH = np.abs(_invariant(xg, vg) - H0)
    assert np.all(dH <= 1e-3 * np.maximum(H0, 1.0)), dH.max()


@pytest.mark.parametrize("kern", [1, 2, 3, 4])
def test_beta_zero_invariant_dense(gpu_lib, kern):
    phia = gpu_lib
    N, R = 64, 32
    d = ins.dense_int(N, 7, 7, seed=4)
    with phia.Annealer(d.k, d.kh, path=phia.PATH_TC, tc_kernel=kern) as A:
        _check(phia, A, R, N)


def test_beta_zero_invariant_fp32(gpu_lib):
    phia = gpu_lib
    N, R = 64, 32
    d = ins.dense_int(N, 7, 7, seed=4)
    with phia.Annealer(d.k, d.kh, path=phia.PATH_FP32) as A:
        _check(phia, A, R, N)


def test_beta_zero_invariant_csr(gpu_lib):
    phia = gpu_lib
    N, R = 300, 64
    c = ins.erdos_renyi(N, 0.05, 127, 31, 4, seed=8)
    with phia.Annealer(h_k=c.kh, frac_bits=c.frac_bits, csr=(c.row_ptr, c.col, c.val), path=phia.PATH_CSR) as A:
        _check(phia, A, R, N)
