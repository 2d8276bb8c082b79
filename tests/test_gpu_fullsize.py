"""GPU parity at the benchmark's full sizes, in the launch configuration bench.py times
(its workload definitions, seeds and the autotuned kernel choice).  Whole trajectories
of FP32 and FP64 part after sign ties, so full runs are judged on sampled outputs the
oracle computes one by one and on properties that hold at any size:

- every sampled returned energy equals Eq. 2 recomputed exactly on the returned spins;
- the field (Eq. 6) of the returned best states is bit-exact against the oracle;
- one iteration from identical state, for every replica at once (the full launch),
  matches the oracle's FP64 step on sampled replicas within 1e-5 of the update's terms;
- in the batch, sampled instances give bit-identical records to the same instance run
  alone."""
import numpy as np
import pytest

import bench
import oracle as o
from paper_2407_10205_gb300 import instances as ins

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _sched(phia, w):
    return phia.schedule(w["beta0"], w["beta1"], w["eps"], w["gamma"], refresh=w["refresh"])


def _dense_full(phia, name, samples):
    w = bench.WORKLOADS[name]
    d = bench._instance(w)
    N, R, T = w["N"], w["replicas"], w["iterations"]
    P = o.Instance(d.kh, k=d.k)
    sched = _sched(phia, w)
    with phia.Annealer(d.k, d.kh, path=phia.PATH_TC) as A:
        phia.autotune(A.h, sched, R, probe_iters=min(T, 200))      # as bench.py does
        res = A.anneal(sched, R, T, w["run_seed"])
        be, bs, _, bits = phia.replica_results(A.h, R, N)
        S = phia.unpack_bits(bits, N)
        rows = np.linspace(0, R - 1, samples).astype(int)
        # (a) returned energies are exact
        for r in rows:
            assert be[r] == o.energy_exact(P, S[r]) and 0 <= bs[r] < T
        assert res.energy_k == be.min()
        # (b) the field of the returned states, computed by the path's field kernel
        f = torch.empty((R, N), dtype=torch.int32, device="cuda")
        e = torch.empty(R, dtype=torch.int64, device="cuda")
        phia.field(A.h, torch.from_numpy(np.ascontiguousarray(S)).cuda(), f, e)
        torch.cuda.synchronize()
        I, E = o.field_batch(P, S[rows])
        assert np.array_equal(f.cpu().numpy()[rows], I) and np.array_equal(e.cpu().numpy()[rows], E)
        # (c) one iteration from identical state for all R replicas
        x, v = ins.random_state(R, N, seed=N + 7)
        xn = x.astype(np.float64) + w["eps"] * v.astype(np.float64)
        bad = np.abs(xn) < 1e-3
        x[bad] = np.where(xn[bad] >= 0, 0.01, -0.01).astype(np.float32)
        v[bad] = 0.0
        beta = 0.5 * (w["beta0"] + w["beta1"])
        xt, vt = torch.from_numpy(x).cuda(), torch.from_numpy(v).cuda()
        phia.run(A.h, phia.schedule(beta, beta, w["eps"], w["gamma"]), R, 0, 1, 1, 5, xt, vt)
        be1, _, _, bits1 = phia.replica_results(A.h, R, N)
        S1 = phia.unpack_bits(bits1, N)
        xg, vg = xt.cpu().numpy(), vt.cpu().numpy()
    for r in rows:
        xo, vo, so, Io, eo = o.step(P, x[r].astype(np.float64), v[r].astype(np.float64), beta, w["eps"], w["gamma"])
        assert np.array_equal(S1[r], so) and be1[r] == eo
        assert np.allclose(xg[r], xo, rtol=1e-6, atol=1e-7)
        scale = np.abs(v[r]) + w["eps"] * (beta * w["gamma"] * np.abs(Io) + np.abs(xo))
        assert np.all(np.abs(vg[r] - vo) <= 1e-5 * np.maximum(scale, 1e-3))


def test_dense200_full_size(gpu_lib):
    """N = 200 dense, 1024 replicas x 2000 iterations (the default benchmark)."""
    _dense_full(gpu_lib, "dense200", 48)


def test_dense2000_full_size(gpu_lib):
    """N = 2000 complete graph, 4096 replicas x 5000 iterations."""
    _dense_full(gpu_lib, "dense2000", 12)


def test_batched_er_full_size(gpu_lib):
    """256 ER instances, 256 replicas x 2000 iterations in one batch."""
    phia = gpu_lib
    w = bench.WORKLOADS["batched_er"]
    insts = ins.batched_er(w["count"], w["seed"])
    R, T = w["replicas"], w["iterations"]
    sched = _sched(phia, w)
    picks = [0, 37, 128, 255]
    with phia.Batch(insts) as B:
        B.anneal(sched, R, T, w["run_seed"])
        got = {k: B.replica_results(k, R) for k in picks}
    for k in picks:
        c = insts[k]
        P = o.Instance(c.kh, row_ptr=c.row_ptr, col=c.col, val=c.val, frac_bits=c.frac_bits)
        be, bs, _, bits = got[k]
        S = phia.unpack_bits(bits, c.n)
        for r in range(0, R, 51):
            assert be[r] == o.energy_exact(P, S[r]) and 0 <= bs[r] < T
    # the same instance alone (same Philox instance id) gives the same records
    for k in picks[1:3]:
        with phia.Batch([insts[k]], instance_ids=[k]) as A:
            A.anneal(sched, R, T, w["run_seed"])
            alone = A.replica_results(0, R)
        for u, v in zip(got[k], alone):
            assert np.array_equal(u, v)
