"""GPU tests of the incremental-field resident kernel (dense, N <= 384): its field is the
exact integer J s + h kept up to date from the columns of the spins that changed sign,
so every record and every FP32 state must equal the resident tensor-core kernel's, bit
for bit, and the oracle's where the oracle is compared."""
import numpy as np
import pytest

import oracle as o
from paper_2407_10205_gb300 import instances as ins

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _run(phia, d, kern, tile, sched, R, T, seed, pieces=None, op=0):
    N = d.n
    with phia.Annealer(d.k, d.kh, path=phia.PATH_TC, operand=op, tc_kernel=kern, tile_replicas=tile) as A:
        x = torch.empty((R, N), device="cuda"); v = torch.empty((R, N), device="cuda")
        phia.init_state(A.h, R, seed, x, v)
        t0 = 0
        for k, s in enumerate(pieces or [T]):
            phia.run(A.h, sched, R, t0, s, T, seed, x, v, reset_best=(k == 0))
            t0 += s
        torch.cuda.synchronize()
        st = phia.stats_get(A.h)
        return phia.replica_results(A.h, R, N), x.cpu().numpy(), v.cpu().numpy(), st


@pytest.mark.parametrize("N,R,tile,kmax,op", [
    (200, 50, 8, 7, 1), (37, 129, 4, 16, 1), (384, 40, 16, 7, 1), (256, 70, 16, 90, 2), (1, 5, 4, 7, 1),
    (130, 33, 8, 127, 2)])
def test_incremental_equals_resident_tensor_core(gpu_lib, N, R, tile, kmax, op):
    """Same records and states as the tcgen05 resident kernel (N = 384 with 16 requested
    runs 8 replicas per CTA: the tiling differs, the per-replica arithmetic does not)."""
    phia = gpu_lib
    d = ins.dense_int(N, kmax, 7, seed=N + R)
    sched = phia.schedule(0.01, 0.3, 0.1, 2.0, refresh=30)
    a = _run(phia, d, phia.KERNEL_RESIDENT, tile, sched, R, 150, 4, op=op)
    b = _run(phia, d, phia.KERNEL_INCREMENTAL, tile, sched, R, 150, 4, op=op)
    assert a[3].tc_kernel == 1 and b[3].tc_kernel == 4
    for u, w in zip(a[0], b[0]):
        assert np.array_equal(u, w)
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_incremental_resume_bit_identical(gpu_lib):
    phia = gpu_lib
    d = ins.sk_pm1(300, 2)
    sched = phia.schedule(0.01, 0.2, 0.1, 2.0, refresh=17)
    one = _run(phia, d, phia.KERNEL_INCREMENTAL, 8, sched, 60, 90, 3)
    two = _run(phia, d, phia.KERNEL_INCREMENTAL, 8, sched, 60, 90, 3, pieces=[1, 33, 56])
    for u, w in zip(one[0], two[0]):
        assert np.array_equal(u, w)
    assert np.array_equal(one[1], two[1]) and np.array_equal(one[2], two[2])


def test_incremental_stop_at_target_matches_resident(gpu_lib):
    """With stop-at-target both kernels report the same earliest hit.  How far other
    CTAs run past it depends on when they see the hit, so only what every replica
    reaches is compared: the earliest hit step, and each replica's hit step where it
    is at or before that one."""
    phia = gpu_lib
    d = ins.dense_int(64, 7, 7, seed=9)
    P = o.Instance(d.kh, k=d.k)
    target = int(o.anneal(P, 4, 200, 5, 0, 0.02, 0.5, 0.1, 2.0)["best_e"].min())
    sched = phia.schedule(0.02, 0.5, 0.1, 2.0, refresh=20, target=target, stop_at_target=True)
    out = []
    for kern in (phia.KERNEL_RESIDENT, phia.KERNEL_INCREMENTAL):
        with phia.Annealer(d.k, d.kh, path=phia.PATH_TC, tc_kernel=kern, tile_replicas=8) as A:
            res = A.anneal(sched, 40, 400, seed=11)
            out.append((res.stats.hit_step, res.energy_k, phia.replica_results(A.h, 40, 64)[2]))
    H = out[0][0]
    assert H >= 0 and out[1][0] == H
    assert out[0][1] <= target and out[1][1] <= target
    ha, hb = out[0][2], out[1][2]
    early = ((ha >= 0) & (ha <= H)) | ((hb >= 0) & (hb <= H))
    assert early.any() and np.array_equal(ha[early], hb[early])


def test_incremental_energies_are_exact(gpu_lib):
    """Every returned energy is Eq. 2 recomputed exactly on the returned spins."""
    phia = gpu_lib
    N, R = 180, 70
    d = ins.dense_int(N, 16, 50, seed=4)
    P = o.Instance(d.kh, k=d.k)
    with phia.Annealer(d.k, d.kh, path=phia.PATH_TC, tc_kernel=phia.KERNEL_INCREMENTAL) as A:
        res = A.anneal(phia.schedule(0.005, 0.1, 0.1, 2.0, refresh=40), R, 300, seed=3)
        be, bs, _, bits = phia.replica_results(A.h, R, N)
    S = phia.unpack_bits(bits, N)
    for r in range(R):
        assert o.energy_exact(P, S[r]) == be[r]
    assert res.stats.tc_kernel == 4 and res.energy_k == be.min()
