"""The error path of bounded device waits, exercised without faulting the GPU.

Every device-side wait in the library's kernels has a time bound; when it runs out the
kernel records it, skips the work that depended on the wait and returns, and the host
reports PHIA_ETIMEOUT.  Here the per-iteration tensor-core kernel runs with its TMA
producer stalled (it issues no copy, so no copy or tensor-core operation is ever in
flight) and a 2 ms bound: the consumer waits on full operand stages and finished
accumulators can never complete and must give up.  The run must report PHIA_ETIMEOUT,
and the same handle (and a fresh one) must then run a normal anneal correctly on the
same GPU.
"""
import numpy as np
import pytest

import oracle as o
from paper_2407_10205_gb300 import instances as ins

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("variant", [1, 7, 9])
def test_expired_waits_report_etimeout_and_the_gpu_stays_usable(gpu_lib, variant):
    """Variant 1: one launch per iteration; variants 7 and 9: one cooperative launch (9 in
    clusters of 4) whose tile counters and records waits must give up too."""
    phia = gpu_lib
    N, R, T = 256, 256, 3
    d = ins.dense_int(N, 7, 7, seed=13)
    P = o.Instance(d.kh, k=d.k)
    sched = phia.schedule(0.01, 0.1, 0.1, 2.0)
    with phia.Annealer(d.k, d.kh, path=phia.PATH_TC, tc_kernel=phia.KERNEL_PER_STEP, large_variant=variant) as A:
        phia.debug_wait(A.h, 2_000_000, stall_producer=True)
        phia.anneal(A.h, sched, R, T, 5)
        with pytest.raises(phia.PhiaError) as ei:
            phia.best(A.h, N)
        assert ei.value.code == phia.ETIMEOUT
        with pytest.raises(phia.PhiaError) as ei:
            phia.stats_get(A.h)
        assert ei.value.code == phia.ETIMEOUT
        # the context is intact: the same handle, back to normal, anneals correctly
        phia.debug_wait(A.h, 0, stall_producer=False)
        res = A.anneal(sched, R, 40, 5)
        assert res.energy_k == o.energy_exact(P, res.spins)
        be, _, _, bits = phia.replica_results(A.h, R, N)
        S = phia.unpack_bits(bits, N)
        for r in range(0, R, 31):
            assert o.energy_exact(P, S[r]) == be[r]
    torch.cuda.synchronize()
    # and so does another handle on another kernel
    with phia.Annealer(d.k, d.kh, path=phia.PATH_TC, tc_kernel=phia.KERNEL_RESIDENT) as B:
        res = B.anneal(sched, 64, 40, 6)
        assert res.energy_k == o.energy_exact(P, res.spins)


def test_stall_is_refused_where_it_does_not_apply(gpu_lib):
    phia = gpu_lib
    d = ins.dense_int(64, 7, 7, seed=2)
    with phia.Annealer(d.k, d.kh, path=phia.PATH_TC, tc_kernel=phia.KERNEL_RESIDENT) as A:
        with pytest.raises(phia.PhiaError) as ei:
            phia.debug_wait(A.h, 1000, stall_producer=True)
        assert ei.value.code == phia.ENOTSUP
        with pytest.raises(phia.PhiaError) as ei:
            phia.debug_wait(A.h, -1)
        assert ei.value.code == phia.EINVAL
