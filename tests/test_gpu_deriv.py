"""GPU tests of the quadratic stand-in for the derivative factor of Eq. 8 (schedule
deriv = 1): one step from identical state against the FP64 oracle on every path, and
bit-identical runs across the dense kernels (they share the update)."""
import numpy as np
import pytest

import oracle as o
from paper_2407_10205_gb300 import instances as ins

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _state(R, N, eps, seed):
    x, v = ins.random_state(R, N, seed=seed)
    xn = x.astype(np.float64) + eps * v.astype(np.float64)
    bad = np.abs(xn) < 1e-3           # keep the sign away from rounding
    x[bad] = np.where(xn[bad] >= 0, 0.01, -0.01).astype(np.float32)
    v[bad] = 0.0
    return x, v


def _one_step(phia, A, P, R, N, beta, eps, gamma, seed):
    x, v = _state(R, N, eps, seed)
    xt, vt = torch.from_numpy(x).cuda(), torch.from_numpy(v).cuda()
    phia.run(A.h, phia.schedule(beta, beta, eps, gamma, deriv=phia.DERIV_QUADRATIC), R, 0, 1, 1, 5, xt, vt)
    be, bs, _, bits = phia.replica_results(A.h, R, N)
    xg, vg = xt.cpu().numpy(), vt.cpu().numpy()
    S = phia.unpack_bits(bits, N)
    for r in range(0, R, 3):
        xo, vo, so, Io, eo = o.step(P, x[r].astype(np.float64), v[r].astype(np.float64), beta, eps, gamma, deriv=1)
        assert np.array_equal(S[r], so) and be[r] == eo
        assert np.allclose(xg[r], xo, rtol=1e-6, atol=1e-7)
        scale = np.abs(v[r]) + eps * (beta * gamma * P.q * np.abs(Io) + np.abs(xo))
        assert np.all(np.abs(vg[r] - vo) <= 1e-5 * np.maximum(scale, 1e-3))


@pytest.mark.parametrize("kern,N,R", [(1, 60, 40), (2, 600, 30), (4, 100, 20)])
def test_quadratic_step_matches_oracle_dense(gpu_lib, kern, N, R):
    phia = gpu_lib
    d = ins.dense_int(N, 7, 7, seed=N)
    P = o.Instance(d.kh, k=d.k)
    with phia.Annealer(d.k, d.kh, path=phia.PATH_TC, tc_kernel=kern) as A:
        _one_step(phia, A, P, R, N, 0.4, 0.1, 2.0, seed=N + 1)


def test_quadratic_step_matches_oracle_csr(gpu_lib):
    phia = gpu_lib
    N, R = 900, 256
    c = ins.erdos_renyi(N, 0.03, 127, 31, 4, seed=3)
    P = o.Instance(c.kh, row_ptr=c.row_ptr, col=c.col, val=c.val, frac_bits=4)
    with phia.Annealer(h_k=c.kh, frac_bits=c.frac_bits, csr=(c.row_ptr, c.col, c.val), path=phia.PATH_CSR) as A:
        _one_step(phia, A, P, R, N, 0.4, 0.1, 2.0, seed=5)


def test_quadratic_runs_identical_across_dense_kernels(gpu_lib):
    phia = gpu_lib
    N, R, T = 200, 64, 150
    d = ins.dense_int(N, 7, 7, seed=2)
    sched = phia.schedule(0.01, 0.3, 0.1, 2.0, refresh=40, deriv=phia.DERIV_QUADRATIC)
    outs = []
    for kern in (phia.KERNEL_RESIDENT, phia.KERNEL_PER_STEP, phia.KERNEL_INCREMENTAL):
        with phia.Annealer(d.k, d.kh, path=phia.PATH_TC, tc_kernel=kern) as A:
            x = torch.empty((R, N), device="cuda"); v = torch.empty((R, N), device="cuda")
            phia.init_state(A.h, R, 7, x, v)
            phia.run(A.h, sched, R, 0, T, T, 7, x, v)
            outs.append((phia.replica_results(A.h, R, N), x.cpu().numpy(), v.cpu().numpy()))
    for other in outs[1:]:
        for u, w in zip(outs[0][0], other[0]):
            assert np.array_equal(u, w)
        assert np.array_equal(outs[0][1], other[1]) and np.array_equal(outs[0][2], other[2])
    # the mode is live: the exact factor gives another trajectory
    with phia.Annealer(d.k, d.kh, path=phia.PATH_TC, tc_kernel=phia.KERNEL_RESIDENT) as A:
        x = torch.empty((R, N), device="cuda"); v = torch.empty((R, N), device="cuda")
        phia.init_state(A.h, R, 7, x, v)
        phia.run(A.h, phia.schedule(0.01, 0.3, 0.1, 2.0, refresh=40), R, 0, T, T, 7, x, v)
        assert not np.array_equal(x.cpu().numpy(), outs[0][1])


def test_unknown_derivative_mode_is_rejected(gpu_lib):
    phia = gpu_lib
    d = ins.dense_int(20, 7, 7, seed=1)
    with phia.Annealer(d.k, d.kh) as A:
        with pytest.raises(phia.PhiaError) as ei:
            A.anneal(phia.schedule(0.01, 0.1, 0.1, 2.0, deriv=2), 8, 10, seed=1)
        assert ei.value.code == phia.EINVAL
