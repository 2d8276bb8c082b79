"""phia_run_noalloc: the allocation-free entry point for callers that cannot allocate
device memory (a device-wide memory pool owns the GPU, or allocation is forbidden in
their time-critical loop).  Checked through the C ABI against phia_run on a handle
that uses the same per-iteration kernel: two calls in a row (the second continuing the
first, reusing the shared scratch) must give the same records and states, for both
operand encodings, both tile widths and sizes next to the scratch limit.  A second
call must not change the device's free memory, and the instance checks of phia_create
must refuse what the fixed-point encoding cannot hold exactly."""
import numpy as np
import pytest

from paper_2407_10205_gb300 import instances as ins

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = [
    # (N, replicas, kmax, operand name, iterations): 128-wide tiles at N = 300; the
    # N = 2000 / 2304-replica case is the largest replica count that fits the scratch with
    # e4m3 at that N; N = 1536 with 3328 replicas picks the 256-wide tile and also sits
    # next to the limit; kmax = 100 under AUTO selects bf16.
    (300, 200, 16, "E4M3", 50), (300, 200, 100, "BF16", 50), (300, 200, 100, "AUTO", 30),
    (2000, 2304, 1, "E4M3", 6), (1536, 3328, 1, "E4M3", 6),
]


def _records(phia, be, bs, hs, bits, x, v):
    return (be.cpu().numpy(), bs.cpu().numpy(), hs.cpu().numpy(), bits.cpu().numpy().view(np.uint32),
            x.cpu().numpy(), v.cpu().numpy())


@pytest.mark.parametrize("N,R,kmax,opname,T", CASES)
def test_noalloc_matches_handle_path_on_two_calls(gpu_lib, N, R, kmax, opname, T):
    phia = gpu_lib
    op = getattr(phia, "OP_" + opname)
    a = T // 3 + 1
    d = ins.dense_int(N, kmax, 31, seed=N + kmax)
    sched = phia.schedule(0.01, 0.2, 0.1, 2.0, refresh=max(2, T // 4))
    W = (N + 31) // 32
    handle_op = phia.OP_BF16 if (opname == "AUTO" and kmax > 16) else op
    with phia.Annealer(d.k, d.kh, path=phia.PATH_TC, operand=handle_op, tc_kernel=phia.KERNEL_PER_STEP) as A:
        x0 = torch.empty((R, N), device="cuda"); v0 = torch.empty((R, N), device="cuda")
        phia.init_state(A.h, R, 5, x0, v0)
        x1, v1 = x0.clone(), v0.clone()
        phia.run(A.h, sched, R, 0, a, T, 5, x1, v1, reset_best=True)
        ref1 = phia.replica_results(A.h, R, N) + (x1.cpu().numpy(), v1.cpu().numpy())
        phia.run(A.h, sched, R, a, T - a, T, 5, x1, v1, reset_best=False)
        ref2 = phia.replica_results(A.h, R, N) + (x1.cpu().numpy(), v1.cpu().numpy())

    Jd = torch.from_numpy(d.k).cuda()
    hd = torch.from_numpy(d.kh).cuda()
    x2, v2 = x0.clone(), v0.clone()
    be = torch.empty(R, dtype=torch.int64, device="cuda")
    bs = torch.empty(R, dtype=torch.int64, device="cuda")
    hs = torch.empty(R, dtype=torch.int64, device="cuda")
    bits = torch.empty((R, W), dtype=torch.int32, device="cuda")
    outs, free = [], []
    for t0, steps, reset in ((0, a, True), (a, T - a, False)):
        phia.run_noalloc(Jd, hd, 0, op, sched, R, t0, steps, T, 5, 0, x2, v2, be, bs, hs, bits, reset_best=reset)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        outs.append(_records(phia, be, bs, hs, bits, x2, v2))
    for ref, got in ((ref1, outs[0]), (ref2, outs[1])):
        for u, w in zip(ref, got):
            assert np.array_equal(u, w)
    assert free[0] == free[1], "a later call changed the device's free memory"


def test_noalloc_rejects_sizes_beyond_its_scratch(gpu_lib):
    phia = gpu_lib
    t = torch.zeros(1, device="cuda")
    J = torch.zeros((2000, 2000), dtype=torch.int8, device="cuda")
    h = torch.zeros(2000, dtype=torch.int32, device="cuda")
    with pytest.raises(phia.PhiaError) as ei:
        phia.run_noalloc(J, h, 0, phia.OP_E4M3, phia.schedule(0.1, 0.2, 0.1, 2.0), 2305, 0, 1, 1, 1, 0,
                         t, t, t, t, t, t)
    assert ei.value.code == phia.ERANGE and "scratch" in str(ei.value) and "2304 replicas" in str(ei.value)


def _small_call(phia, k, kh, op):
    N, R = k.shape[0], 8
    x = torch.zeros((R, N), device="cuda"); v = torch.zeros((R, N), device="cuda")
    rec = [torch.empty(R, dtype=torch.int64, device="cuda") for _ in range(3)]
    bits = torch.empty((R, (N + 31) // 32), dtype=torch.int32, device="cuda")
    phia.run_noalloc(torch.from_numpy(k).cuda(), torch.from_numpy(kh).cuda(), 0, op,
                     phia.schedule(0.1, 0.2, 0.1, 2.0), R, 0, 2, 2, 1, 0, x, v, *rec, bits)


def test_noalloc_checks_the_instance_like_phia_create(gpu_lib):
    """|k| = 17 is not exact in e4m3 (3 mantissa bits): PHIA_ERANGE, not a silently
    rounded field; an asymmetric J or a nonzero diagonal: PHIA_EINVAL; |h| >= 2^24:
    PHIA_ERANGE."""
    phia = gpu_lib
    d = ins.dense_int(40, 7, 7, seed=3)
    k17 = d.k.copy(); k17[3, 5] = k17[5, 3] = 17
    asym = d.k.copy(); asym[1, 2] = np.int8(asym[2, 1] + 1)
    diag = d.k.copy(); diag[4, 4] = 1
    hbig = d.kh.copy(); hbig[7] = 1 << 24
    for k, kh, op, code in ((k17, d.kh, phia.OP_E4M3, phia.ERANGE), (asym, d.kh, phia.OP_BF16, phia.EINVAL),
                            (diag, d.kh, phia.OP_BF16, phia.EINVAL), (d.k, hbig, phia.OP_BF16, phia.ERANGE)):
        with pytest.raises(phia.PhiaError) as ei:
            _small_call(phia, k, kh, op)
        assert ei.value.code == code, str(ei.value)
    _small_call(phia, k17, d.kh, phia.OP_AUTO)   # AUTO takes bf16 here, exact for |k| = 17
