"""Resident tensor-core kernel at large energy terms: every term s_i (I_i + h_i) of a
32-spin warp at its maximum (a warp sum at and just past 2^15), fields and energies
(Eqs. 2, 6) equal the oracle's exactly, and run records hold Eq. 2 on the returned
spins for every tile size; one step from identical state matches the oracle on two- and
three-tile instances (N = 200, 300, 384)."""
import numpy as np
import pytest

import oracle as o
from paper_2407_10205_gb300 import instances as ins

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _group_bound(k, kh):
    ra = np.abs(k.astype(np.int64)).sum(1) + 2 * np.abs(kh.astype(np.int64))
    return max(int(ra[g:g + 32].sum()) for g in range(0, len(kh), 32))


def _spin_patterns(N, R, seed):
    g = np.random.default_rng(seed)
    S = np.where(g.random((R, N)) < 0.5, -1, 1).astype(np.int8)
    S[0] = 1                     # every term at its maximum in group 0
    S[1] = -1
    S[2, :32], S[2, 32:] = 1, -1
    S[3, :32], S[3, 32:] = -1, 1
    S[4, ::2], S[4, 1::2] = 1, -1
    S[5] = -S[4]
    return S


@pytest.mark.parametrize("h0, below", [(255, True), (256, False)])
def test_energy_terms_at_16_bits(gpu_lib, h0, below):
    phia = gpu_lib
    N, R = 64, 24
    k = np.full((N, N), 16, np.int8)
    np.fill_diagonal(k, 0)
    kh = np.zeros(N, np.int32)
    kh[0], kh[33] = h0, -h0
    assert (_group_bound(k, kh) < 2 ** 15) == below
    P = o.Instance(kh, k=k)
    S = _spin_patterns(N, R, seed=h0)
    with phia.Annealer(k, kh, path=phia.PATH_TC, tc_kernel=phia.KERNEL_RESIDENT) as A:
        f = torch.empty((R, N), dtype=torch.int32, device="cuda")
        e = torch.empty(R, dtype=torch.int64, device="cuda")
        phia.field(A.h, torch.from_numpy(S).cuda(), f, e)
        torch.cuda.synchronize()
        I, E = o.field_batch(P, S)
        assert np.array_equal(f.cpu().numpy(), I) and np.array_equal(e.cpu().numpy(), E)
        # replica 0 (all +1) puts group 0's warp sum at 32 * 1008 + 2 h0
        assert int((S[0, :32].astype(np.int64) * (I[0, :32] + kh[:32])).sum()) == 32 * 1008 + 2 * h0
        # run records: every returned energy equals Eq. 2 on the returned spins
        for tile in (4, 8, 16):
            with phia.Annealer(k, kh, path=phia.PATH_TC, tc_kernel=phia.KERNEL_RESIDENT,
                               tile_replicas=tile) as B:
                B.anneal(phia.schedule(0.01, 0.2, 0.1, 2.0, refresh=30), R, 300, seed=5)
                be, bs, _, bits = phia.replica_results(B.h, R, N)
                Sb = phia.unpack_bits(bits, N)
                for r in range(R):
                    assert be[r] == o.energy_exact(P, Sb[r]) and 0 <= bs[r] < 300


@pytest.mark.parametrize("N,kmax,hmax", [(200, 7, 7), (300, 1, 0), (384, 7, 7)])
def test_resident_runs_match_oracle_records(gpu_lib, N, kmax, hmax):
    """One step from identical state gives the oracle's energies and spins on every
    replica (two and three output tiles; group sums of |terms| below and above 2^15)."""
    phia = gpu_lib
    d = ins.dense_int(N, kmax, hmax, seed=N + 3)
    P = o.Instance(d.kh, k=d.k)
    assert (_group_bound(d.k, d.kh) < 2 ** 15) == (N != 384)
    R = 40
    x, v = ins.random_state(R, N, seed=N)
    xn = x.astype(np.float64) + 0.1 * v.astype(np.float64)
    bad = np.abs(xn) < 1e-3
    x[bad] = np.where(xn[bad] >= 0, 0.01, -0.01).astype(np.float32)
    v[bad] = 0.0
    with phia.Annealer(d.k, d.kh, path=phia.PATH_TC, tc_kernel=phia.KERNEL_RESIDENT) as A:
        xt, vt = torch.from_numpy(x).cuda(), torch.from_numpy(v).cuda()
        phia.run(A.h, phia.schedule(0.3, 0.3, 0.1, 2.0), R, 0, 1, 1, 5, xt, vt)
        be, _, _, bits = phia.replica_results(A.h, R, N)
        S = phia.unpack_bits(bits, N)
    for r in range(R):
        _, _, so, _, eo = o.step(P, x[r].astype(np.float64), v[r].astype(np.float64), 0.3, 0.1, 2.0)
        assert np.array_equal(S[r], so) and be[r] == eo
