"""GPU tests of the autotuner (phia_autotune)."""
import numpy as np
import pytest

from paper_2407_10205_gb300 import instances as ins

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_autotune_picks_a_variant_and_caches_it(gpu_lib):
    phia = gpu_lib
    N, R, T = 200, 300, 80
    d = ins.dense_int(N, 7, 7, seed=1)
    sched = phia.schedule(0.01, 0.1, 0.1, 2.0, refresh=50)
    with phia.Annealer(d.k, d.kh, path=phia.PATH_TC) as A:
        res = phia.autotune(A.h, sched, R, probe_iters=50)
        # resident tcgen05 (3 tiles x 2 places for J), int8 mma.sync (2), incremental (3),
        # per-iteration kernel (13 variants)
        assert res.candidates == 24 and res.tc_kernel in (1, 2, 3, 4)
        assert 0 < res.best_us_per_iter <= res.worst_us_per_iter
        A.anneal(sched, R, T, seed=5)
        tuned = phia.replica_results(A.h, R, N)
        assert phia.stats_get(A.h).tc_kernel == res.tc_kernel
    # every variant gives the same records, so the tuned run equals a fixed variant
    with phia.Annealer(d.k, d.kh, path=phia.PATH_TC, tile_replicas=16, coupling_mem=1) as B:
        B.anneal(sched, R, T, seed=5)
        fixed = phia.replica_results(B.h, R, N)
    for u, w in zip(tuned, fixed):
        assert np.array_equal(u, w)
    # a new automatic handle with the same (N, replicas, operand) uses the cached choice
    with phia.Annealer(d.k, d.kh, path=phia.PATH_TC) as C:
        C.anneal(sched, R, T, seed=5)
        assert phia.stats_get(C.h).tc_kernel == res.tc_kernel


def test_autotune_large_n_times_the_per_iteration_variants(gpu_lib):
    phia = gpu_lib
    d = ins.sk_pm1(600, 2)
    with phia.Annealer(d.k, d.kh, path=phia.PATH_TC) as A:
        res = phia.autotune(A.h, phia.schedule(0.01, 0.2, 0.1, 2.0), 128, probe_iters=10)
        assert res.candidates == 13 and res.tc_kernel == 2 and 1 <= res.large_variant <= 13
