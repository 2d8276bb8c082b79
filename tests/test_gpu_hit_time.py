"""Time to target on the device (Table 3, state 5: a hit records its step and the device
clock).  On every path the first hit of a target is stamped with %globaltimer; stats.hit_ns
is the time from the run's start (its record reset) to that record: -1 without a hit,
positive and within the run's device time with one, and no later for a looser target
reached at an earlier step of the same trajectory."""
import pytest

from paper_2407_10205_gb300 import instances as ins

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

R, T = 64, 400


def _sched(phia, target=None):
    return phia.schedule(0.01, 0.3, 0.1, 2.0, refresh=50, target=target)


def _check(phia, run, stats):
    run(_sched(phia))
    st = stats()
    assert st.hit_step == -1 and st.hit_ns == -1
    tight = st.best_energy_k                      # this trajectory's own best: reached at best_step
    loose = tight + max(8, abs(tight) // 4)
    run(_sched(phia, target=tight))
    s1 = stats()
    run(_sched(phia, target=loose))
    s2 = stats()
    assert 0 <= s2.hit_step <= s1.hit_step < T
    for s in (s1, s2):
        assert 0 < s.hit_ns <= s.device_ms * 1e6 + 1e6     # within the run (1 ms for the reset launch)
    assert s2.hit_ns <= s1.hit_ns


@pytest.mark.parametrize("kern", [1, 2, 3, 4])
def test_hit_time_dense(gpu_lib, kern):
    phia = gpu_lib
    d = ins.dense_int(100, 7, 7, seed=6)
    with phia.Annealer(d.k, d.kh, path=phia.PATH_TC, tc_kernel=kern) as A:
        _check(phia, lambda s: phia.anneal(A.h, s, R, T, 3), lambda: phia.stats_get(A.h))


def test_hit_time_fp32(gpu_lib):
    phia = gpu_lib
    d = ins.dense_int(100, 7, 7, seed=6)
    with phia.Annealer(d.k, d.kh, path=phia.PATH_FP32) as A:
        _check(phia, lambda s: phia.anneal(A.h, s, R, T, 3), lambda: phia.stats_get(A.h))


def test_hit_time_csr_batch(gpu_lib):
    phia = gpu_lib
    insts = [ins.erdos_renyi(300, 0.05, 127, 31, 4, seed=11)]
    with phia.Batch(insts) as B:
        def run(s):
            B.anneal(s, 256, T, 5)
            B.sync()
        _check(phia, run, B.stats)
