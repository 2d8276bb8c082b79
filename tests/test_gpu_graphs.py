"""GPU tests of the per-iteration paths' graph replay: step kernels read their iteration
from device memory, so long runs replay instantiated graphs of identical launches.  A
run replayed through graphs must equal the same run cut into short calls that launch
every step directly, and a repeated run (graph taken from the cache) must equal the
first."""
import numpy as np
import pytest

from paper_2407_10205_gb300 import instances as ins

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _run_whole_and_chunked(phia, make, N, R, T, chunks, seed):
    sched = phia.schedule(0.01, 0.2, 0.1, 2.0, refresh=40)
    out = []
    for pieces in ([T], chunks):
        assert sum(pieces) == T
        with make() as A:
            x = torch.empty((R, N), device="cuda"); v = torch.empty((R, N), device="cuda")
            phia.init_state(A.h, R, seed, x, v)
            t0 = 0
            for k, s in enumerate(pieces):
                phia.run(A.h, sched, R, t0, s, T, seed, x, v, reset_best=(k == 0))
                t0 += s
            torch.cuda.synchronize()
            out.append((phia.replica_results(A.h, R, N), x.cpu().numpy(), v.cpu().numpy()))
    (r1, x1, v1), (r2, x2, v2) = out
    for u, w in zip(r1, r2):
        assert np.array_equal(u, w)
    assert np.array_equal(x1, x2) and np.array_equal(v1, v2)


def test_large_graph_replay_equals_direct_launches(gpu_lib):
    """450 iterations in one call (4 graph replays of 100 launches + 50 direct) against
    the same run in calls of at most 37 iterations (every launch direct)."""
    phia = gpu_lib
    N, R, T = 300, 300, 450
    d = ins.dense_int(N, 7, 7, seed=31)
    make = lambda: phia.Annealer(d.k, d.kh, path=phia.PATH_TC, tc_kernel=phia.KERNEL_PER_STEP)
    _run_whole_and_chunked(phia, make, N, R, T, [37] * 12 + [6], seed=8)


def test_csr_graph_replay_equals_direct_launches(gpu_lib):
    phia = gpu_lib
    N, R, T = 900, 256, 430
    c = ins.erdos_renyi(N, 0.02, 127, 31, 4, seed=32)
    make = lambda: phia.Annealer(h_k=c.kh, frac_bits=c.frac_bits, csr=(c.row_ptr, c.col, c.val), path=phia.PATH_CSR)
    _run_whole_and_chunked(phia, make, N, R, T, [43] * 10, seed=9)


@pytest.mark.parametrize("kind", ["large", "csr"])
def test_repeated_run_from_cached_graph(gpu_lib, kind):
    """The same 150-iteration anneal three times on one handle: the first launches
    directly, the second builds the graph, the third replays it from the cache."""
    phia = gpu_lib
    sched = phia.schedule(0.01, 0.2, 0.1, 2.0, refresh=25)
    if kind == "large":
        d = ins.sk_pm1(500, 5)
        A = phia.Annealer(d.k, d.kh, path=phia.PATH_TC, tc_kernel=phia.KERNEL_PER_STEP)
        N = 500
    else:
        c = ins.erdos_renyi(700, 0.03, 127, 31, 4, seed=6)
        A = phia.Annealer(h_k=c.kh, frac_bits=c.frac_bits, csr=(c.row_ptr, c.col, c.val), path=phia.PATH_CSR)
        N = 700
    R = 260
    with A:
        res = []
        for _ in range(3):
            r = A.anneal(sched, R, 150, seed=12)
            res.append((r.energy_k, r.spins.copy(), phia.replica_results(A.h, R, N)))
    for e, s, rr in res[1:]:
        assert e == res[0][0] and np.array_equal(s, res[0][1])
        for u, w in zip(rr, res[0][2]):
            assert np.array_equal(u, w)
