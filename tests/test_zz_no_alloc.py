"""phia_run_noalloc: the allocation-free entry point for callers that cannot allocate
device memory (a device-wide memory pool owns the GPU, or allocation is forbidden in
their time-critical loop).  Checked through the C ABI against phia_run on a handle
that uses the same per-iteration kernel: two calls in a row (the second continuing the
first, reusing the shared scratch) must give the same records and states."""
import numpy as np
import pytest

from paper_2407_10205_gb300 import instances as ins

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_noalloc_matches_handle_path_on_two_calls(gpu_lib):
    phia = gpu_lib
    N, R, T, a = 300, 200, 50, 19
    d = ins.dense_int(N, 16, 31, seed=7)
    sched = phia.schedule(0.01, 0.2, 0.1, 2.0, refresh=15)
    W = (N + 31) // 32
    with phia.Annealer(d.k, d.kh, path=phia.PATH_TC, operand=phia.OP_E4M3, tc_kernel=phia.KERNEL_PER_STEP) as A:
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
    outs = []
    for t0, steps, reset in ((0, a, True), (a, T - a, False)):
        phia.run_noalloc(Jd, hd, 0, phia.OP_E4M3, sched, R, t0, steps, T, 5, 0, x2, v2, be, bs, hs, bits,
                         reset_best=reset)
        outs.append((be.cpu().numpy(), bs.cpu().numpy(), hs.cpu().numpy(), bits.cpu().numpy().view(np.uint32),
                     x2.cpu().numpy(), v2.cpu().numpy()))
    for ref, got in ((ref1, outs[0]), (ref2, outs[1])):
        for u, w in zip(ref, got):
            assert np.array_equal(u, w)


def test_noalloc_rejects_sizes_beyond_its_scratch(gpu_lib):
    phia = gpu_lib
    N, R = 4000, 4096
    t = torch.zeros(1, device="cuda")
    J = torch.zeros((N, N), dtype=torch.int8, device="cuda")
    h = torch.zeros(N, dtype=torch.int32, device="cuda")
    with pytest.raises(phia.PhiaError) as ei:
        phia.run_noalloc(J, h, 0, phia.OP_E4M3, phia.schedule(0.1, 0.2, 0.1, 2.0), R, 0, 1, 1, 1, 0,
                         t, t, t, t, t, t)
    assert ei.value.code == phia.ERANGE and "scratch" in str(ei.value)
