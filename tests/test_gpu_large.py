"""GPU parity tests of the per-iteration tensor-core kernel (TMA-staged J, any N),
through the C ABI against the oracle and against the resident kernel."""
import numpy as np
import pytest

import oracle as o
from paper_2407_10205_gb300 import instances as ins

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _large(phia, d, op, frac=0):
    return phia.Annealer(d.k, d.kh, frac_bits=frac, path=phia.PATH_TC, operand=op, tc_kernel=phia.KERNEL_PER_STEP)


def _field(phia, A, S):
    R, N = S.shape
    f = torch.empty((R, N), dtype=torch.int32, device="cuda")
    e = torch.empty(R, dtype=torch.int64, device="cuda")
    phia.field(A.h, torch.from_numpy(S).cuda(), f, e)
    torch.cuda.synchronize()
    return f.cpu().numpy(), e.cpu().numpy()


@pytest.mark.parametrize("N,R,kmax,hmax,op", [
    (5, 1, 7, 7, 1), (130, 129, 16, 100, 1), (257, 260, 7, 7, 1), (700, 40, 16, 1 << 20, 1),
    (2000, 130, 1, 0, 1), (150, 3, 127, 127, 2), (640, 129, 127, 31, 2),
    (640, 10240, 16, 100, 1)])   # 400 output tiles: several per CTA of the persistent kernel
def test_large_field_bit_exact(gpu_lib, N, R, kmax, hmax, op):
    phia = gpu_lib
    d = ins.dense_int(N, kmax, hmax, seed=N + R)
    S = ins.random_spins(R, N, seed=N * 3 + R)
    with _large(phia, d, op) as A:
        f, e = _field(phia, A, S)
    I, E = o.field_batch(o.Instance(d.kh, k=d.k), S)
    assert np.array_equal(f, I) and np.array_equal(e, E)


@pytest.mark.parametrize("N,kval,op", [(2048, 16, 1), (2048, -16, 1), (8192, 127, 2)])
def test_large_field_extreme_magnitudes(gpu_lib, N, kval, op):
    """All products of one sign at the largest exact |k|, N up to 8192: partial sums
    reach |k| (N - 1) = 1.04e6 in FP32 TMEM accumulation and must stay exact."""
    phia = gpu_lib
    k = np.full((N, N), kval, dtype=np.int8)
    np.fill_diagonal(k, 0)
    d = ins.Dense(k, np.full(N, (1 << 24) - 1, dtype=np.int32))
    S = np.ones((3, N), dtype=np.int8)
    S[1] = -1
    S[2, ::3] = -1
    with _large(phia, d, op) as A:
        f, e = _field(phia, A, S)
    I, E = o.field_batch(o.Instance(d.kh, k=d.k), S)
    assert np.array_equal(f, I) and np.array_equal(e, E)


def test_large_single_step_matches_oracle(gpu_lib):
    phia = gpu_lib
    N, R, eps, gamma, beta = 600, 30, 0.1, 2.0, 0.21
    d = ins.dense_int(N, 7, 7, seed=11)
    P = o.Instance(d.kh, k=d.k)
    x, v = ins.random_state(R, N, seed=12)
    xn = x.astype(np.float64) + eps * v.astype(np.float64)
    bad = np.abs(xn) < 1e-3
    x[bad] = np.where(xn[bad] >= 0, 0.01, -0.01).astype(np.float32)
    v[bad] = 0.0
    with _large(phia, d, 1) as A:
        xt, vt = torch.from_numpy(x).cuda(), torch.from_numpy(v).cuda()
        phia.run(A.h, phia.schedule(beta, beta, eps, gamma), R, 0, 1, 1, 5, xt, vt)
        be, bs, _, bits = phia.replica_results(A.h, R, N)
        xg, vg = xt.cpu().numpy(), vt.cpu().numpy()
    S = phia.unpack_bits(bits, N)
    for r in range(R):
        xo, vo, so, Io, eo = o.step(P, x[r].astype(np.float64), v[r].astype(np.float64), beta, eps, gamma)
        assert np.array_equal(S[r], so) and be[r] == eo and bs[r] == 0
        assert np.allclose(xg[r], xo, rtol=1e-6, atol=1e-7)
        scale = np.abs(v[r]) + eps * (beta * gamma * np.abs(Io) + np.abs(xo))
        assert np.all(np.abs(vg[r] - vo) <= 1e-5 * np.maximum(scale, 1e-3))


@pytest.mark.parametrize("N,op,R", [(200, 1, 50), (130, 2, 140), (256, 1, 40000), (130, 2, 40000)])
def test_large_equals_resident_kernel(gpu_lib, N, op, R):
    """The per-iteration and the resident kernel do the same arithmetic per replica:
    records and final states are bit-identical (R = 40000: over 600 output tiles, so
    each CTA of the persistent per-iteration kernel runs several and reuses both of its
    accumulators)."""
    phia = gpu_lib
    T = 120
    d = ins.dense_int(N, 7 if op == 1 else 90, 7, seed=N)
    sched = phia.schedule(0.01, 0.2, 0.1, 2.0, refresh=30)
    outs = []
    for kern in (phia.KERNEL_RESIDENT, phia.KERNEL_PER_STEP):
        with phia.Annealer(d.k, d.kh, path=phia.PATH_TC, operand=op, tc_kernel=kern) as A:
            x = torch.empty((R, N), device="cuda"); v = torch.empty((R, N), device="cuda")
            phia.init_state(A.h, R, 21, x, v)
            phia.run(A.h, sched, R, 0, T, T, 21, x, v)
            outs.append((phia.replica_results(A.h, R, N), x.cpu().numpy(), v.cpu().numpy(),
                         phia.stats_get(A.h).tc_kernel))
    assert outs[0][3] == 1 and outs[1][3] == 2
    for u, w in zip(outs[0][0], outs[1][0]):
        assert np.array_equal(u, w)
    assert np.array_equal(outs[0][1], outs[1][1]) and np.array_equal(outs[0][2], outs[1][2])


def test_large_resume_bit_identical(gpu_lib):
    phia = gpu_lib
    N, R, T, a = 700, 130, 60, 23
    d = ins.sk_pm1(N, 3)
    sched = phia.schedule(0.01, 0.15, 0.1, 2.0, refresh=10)
    with _large(phia, d, 1) as A:
        x1 = torch.empty((R, N), device="cuda"); v1 = torch.empty((R, N), device="cuda")
        phia.init_state(A.h, R, 9, x1, v1)
        x2, v2 = x1.clone(), v1.clone()
        phia.run(A.h, sched, R, 0, T, T, 9, x1, v1)
        one = phia.replica_results(A.h, R, N)
        phia.run(A.h, sched, R, 0, a, T, 9, x2, v2, reset_best=True)
        phia.run(A.h, sched, R, a, 1, T, 9, x2, v2, reset_best=False)
        phia.run(A.h, sched, R, a + 1, T - a - 1, T, 9, x2, v2, reset_best=False)
        two = phia.replica_results(A.h, R, N)
        torch.cuda.synchronize()
        assert torch.equal(x1, x2) and torch.equal(v1, v2)
        for u, w in zip(one, two):
            assert np.array_equal(u, w)


def test_large_run_invariants(gpu_lib):
    """Every returned energy equals Eq. 2 recomputed exactly on the returned spins."""
    phia = gpu_lib
    N, R = 520, 140
    d = ins.dense_int(N, 16, 50, seed=4)
    P = o.Instance(d.kh, k=d.k)
    with _large(phia, d, 1) as A:
        res = A.anneal(phia.schedule(0.005, 0.1, 0.1, 2.0, refresh=40), R, 300, seed=3)
        be, bs, _, bits = phia.replica_results(A.h, R, N)
    S = phia.unpack_bits(bits, N)
    for r in range(R):
        assert o.energy_exact(P, S[r]) == be[r]
    assert res.energy_k == be.min() and o.energy_exact(P, res.spins) == res.energy_k
    assert res.stats.tc_kernel == 2 and res.stats.spin_updates == R * N * 300


# ------------------------------------------------------------------ kernel variants

VARIANTS = list(range(1, 14))   # x/v ring in shared memory; x/v in registers; + spin-tile multicast over
                                # 2 / 4 CTAs (registers: 3, 4; ring: 5, 6); 7: the whole run in one cooperative
                                # launch with per-replica-tile counters, 8 / 9: the same with the multicast over
                                # 2 / 4 CTAs, 10-13: tile width fixed at 256 / 224 / 128 / 160 (160: three
                                # accumulators; field-only calls use 1)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("N,R,kmax,op", [(2000, 300, 1, 1), (1024, 4096, 16, 1), (520, 1100, 127, 2),
                                          (384, 300, 7, 1)])
def test_large_variants_field_bit_exact(gpu_lib, variant, N, R, kmax, op):
    """Every variant computes the exact field and energy (N = 384: three spin tiles, which a
    cluster of 2 or 4 cannot split, so those fall back to the unclustered form)."""
    phia = gpu_lib
    d = ins.dense_int(N, kmax, 31, seed=N + variant)
    S = ins.random_spins(R, N, seed=N + R)
    with phia.Annealer(d.k, d.kh, path=phia.PATH_TC, operand=op, tc_kernel=phia.KERNEL_PER_STEP,
                       large_variant=variant) as A:
        f, e = _field(phia, A, S)
    I, E = o.field_batch(o.Instance(d.kh, k=d.k), S)
    assert np.array_equal(f, I) and np.array_equal(e, E)


@pytest.mark.parametrize("N,R,op", [(1024, 600, 1), (2000, 4096, 1), (512, 700, 2)])
def test_large_variants_bit_identical_runs(gpu_lib, N, R, op):
    """The variants change where x, v and the spin operand travel, not the arithmetic per
    replica: records and final states of a run with refreshes are bit-identical across all
    of them (and equal the oracle's energies on the returned spins)."""
    phia = gpu_lib
    T = 40
    d = ins.dense_int(N, 7 if op == 1 else 90, 7, seed=N + 1)
    sched = phia.schedule(0.01, 0.2, 0.1, 2.0, refresh=15)
    outs = []
    for variant in VARIANTS:
        with phia.Annealer(d.k, d.kh, path=phia.PATH_TC, operand=op, tc_kernel=phia.KERNEL_PER_STEP,
                           large_variant=variant) as A:
            x = torch.empty((R, N), device="cuda"); v = torch.empty((R, N), device="cuda")
            phia.init_state(A.h, R, 4, x, v)
            phia.run(A.h, sched, R, 0, T, T, 4, x, v)
            outs.append((phia.replica_results(A.h, R, N), x.cpu().numpy(), v.cpu().numpy()))
    for rec, x, v in outs[1:]:
        for u, w in zip(outs[0][0], rec):
            assert np.array_equal(u, w)
        assert np.array_equal(outs[0][1], x) and np.array_equal(outs[0][2], v)
    P = o.Instance(d.kh, k=d.k)
    S = phia.unpack_bits(outs[0][0][3], N)
    for r in range(0, R, max(1, R // 16)):
        assert o.energy_exact(P, S[r]) == outs[0][0][0][r]


@pytest.mark.parametrize("variant", VARIANTS)
def test_large_variants_single_step_matches_oracle(gpu_lib, variant):
    phia = gpu_lib
    N, R, eps, gamma, beta = 1024, 520, 0.1, 2.0, 0.05
    d = ins.dense_int(N, 7, 7, seed=13)
    P = o.Instance(d.kh, k=d.k)
    x, v = ins.random_state(R, N, seed=14)
    xn = x.astype(np.float64) + eps * v.astype(np.float64)
    bad = np.abs(xn) < 1e-3
    x[bad] = np.where(xn[bad] >= 0, 0.01, -0.01).astype(np.float32)
    v[bad] = 0.0
    with phia.Annealer(d.k, d.kh, path=phia.PATH_TC, tc_kernel=phia.KERNEL_PER_STEP, large_variant=variant) as A:
        xt, vt = torch.from_numpy(x).cuda(), torch.from_numpy(v).cuda()
        phia.run(A.h, phia.schedule(beta, beta, eps, gamma), R, 0, 1, 1, 5, xt, vt)
        be, bs, _, bits = phia.replica_results(A.h, R, N)
        xg, vg = xt.cpu().numpy(), vt.cpu().numpy()
    S = phia.unpack_bits(bits, N)
    for r in range(0, R, 13):
        xo, vo, so, Io, eo = o.step(P, x[r].astype(np.float64), v[r].astype(np.float64), beta, eps, gamma)
        assert np.array_equal(S[r], so) and be[r] == eo and bs[r] == 0
        assert np.allclose(xg[r], xo, rtol=1e-6, atol=1e-7)
        scale = np.abs(v[r]) + eps * (beta * gamma * np.abs(Io) + np.abs(xo))
        assert np.all(np.abs(vg[r] - vo) <= 1e-5 * np.maximum(scale, 1e-3))


@pytest.mark.parametrize("variant", [7, 8, 9, 10, 11, 12, 13])
@pytest.mark.parametrize("N,R,op,T", [(2000, 4096, 1, 120), (1024, 600, 1, 200), (4000, 2048, 1, 60),
                                      (4000, 1200, 1, 40), (700, 300, 2, 150), (130, 64, 1, 90)])
def test_overlapped_variant_equals_per_iteration_launches(gpu_lib, variant, N, R, op, T):
    """Variants 7-13 (one cooperative launch per run; CTAs keep their tiles and wait on
    per-replica-tile counters; a records warp settles energies and copies best spins; 8 / 9
    multicast the spin tile over clusters of 2 / 4 CTAs, N = 700 / 130 falling back to
    smaller clusters; 10 / 11 / 12 / 13 fix the tile width at 256 / 224 / 128 / 160
    replicas, 160 with three tensor-memory accumulators) give
    bit for bit the records, hit steps and final x, v of one launch per iteration, with
    refreshes and a target that some replicas reach mid-run; grids of fewer CTAs than SMs
    (N = 1024 / 700 / 130), CTAs with one or more tiles, and each tile width variant 7
    picks by its estimate (224 replicas at N = 2000 x 4096, 160 at 4000 x 1200, 256 at
    4000 x 2048, 128 for the others) included."""
    phia = gpu_lib
    d = ins.dense_int(N, 7 if op == 1 else 90, 7, seed=N + 5)
    P = o.Instance(d.kh, k=d.k)
    sched0 = phia.schedule(0.01, 0.2, 0.1, 2.0, refresh=25)
    outs = []
    for lv in (1, variant):
        with phia.Annealer(d.k, d.kh, path=phia.PATH_TC, operand=op, tc_kernel=phia.KERNEL_PER_STEP,
                           large_variant=lv) as A:
            if not outs:
                # a target between the best energies of the replicas: reached by some, mid-run
                phia.anneal(A.h, sched0, R, T, 9)
                be0 = phia.replica_results(A.h, R, N)[0]
                target = int(np.median(be0))
            sched = phia.schedule(0.01, 0.2, 0.1, 2.0, refresh=25, target=target)
            x = torch.empty((R, N), device="cuda"); v = torch.empty((R, N), device="cuda")
            phia.init_state(A.h, R, 9, x, v)
            phia.run(A.h, sched, R, 0, T, T, 9, x, v)
            outs.append((phia.replica_results(A.h, R, N), x.cpu().numpy(), v.cpu().numpy()))
    (rec1, x1, v1), (rec7, x7, v7) = outs
    for u, w in zip(rec1, rec7):
        assert np.array_equal(u, w)
    assert np.array_equal(x1, x7) and np.array_equal(v1, v7)
    hit = rec7[2]
    assert (hit >= 0).any() and (hit < 0).any()
    S = phia.unpack_bits(rec7[3], N)
    for r in range(0, R, max(1, R // 16)):
        assert o.energy_exact(P, S[r]) == rec7[0][r]


@pytest.mark.parametrize("variant", [7, 9])
def test_overlapped_variant_resumes_bit_identical(gpu_lib, variant):
    """A run split into calls (t0 > 0) equals the same run in one call, on variants 7 and 9."""
    phia = gpu_lib
    N, R, T = 1500, 1024, 90
    d = ins.sk_pm1(N, 4)
    sched = phia.schedule(0.01, 0.2, 0.1, 2.0, refresh=20)
    res = []
    for splits in ((0, T), (0, 33, 61, T)):
        with phia.Annealer(d.k, d.kh, path=phia.PATH_TC, tc_kernel=phia.KERNEL_PER_STEP,
                           large_variant=variant) as A:
            x = torch.empty((R, N), device="cuda"); v = torch.empty((R, N), device="cuda")
            phia.init_state(A.h, R, 3, x, v)
            for k in range(len(splits) - 1):
                phia.run(A.h, sched, R, splits[k], splits[k + 1] - splits[k], T, 3, x, v, reset_best=(k == 0))
            res.append((phia.replica_results(A.h, R, N), x.cpu().numpy(), v.cpu().numpy()))
    for u, w in zip(res[0][0], res[1][0]):
        assert np.array_equal(u, w)
    assert np.array_equal(res[0][1], res[1][1]) and np.array_equal(res[0][2], res[1][2])
