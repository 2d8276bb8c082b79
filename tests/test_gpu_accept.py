"""GPU parity of the acceptance test (Table 3, state 4, read as the Metropolis test of
HMC on the Hamiltonian of Eq. 4; schedule accept_test = 1) against the FP64 oracle.

Trajectories of 5 iterations (refresh = 5), 41 iterations in all: tests at the momentum
draws t = 10, 15, ..., 40 (the first trajectory, from the injected state, is kept
untested).  The schedule is chosen so that about half of the tests reject (checked on
the oracle).  From identical FP32 states, per replica: best energy and its step, the
numbers of tests and acceptances, and the final x and v equal the oracle's for >= 90%
of replicas (a replica may differ where FP32 and FP64 decide a sign or a test near its
threshold differently).  The same run compared against the oracle without the test
matches almost no replica, so the bar detects a GPU that skipped the test or applied it
at the wrong place.
"""
import numpy as np
import pytest

import oracle as o
from paper_2407_10205_gb300 import instances as ins

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N, R, T, REFRESH = 100, 64, 41, 5
EPS, GAMMA, BETA0, BETA1 = 0.1, 2.0, 0.005, 0.02
SEED, INST = 3, 4


def _handle(phia, d, path):
    if path == "fp32":
        return phia.Annealer(d.k, d.kh, path=phia.PATH_FP32, instance_id=INST)
    op, tile = {"tc_e4m3_8": (phia.OP_E4M3, 8), "tc_e4m3_16": (phia.OP_E4M3, 16), "tc_e4m3_4": (phia.OP_E4M3, 4),
                "tc_bf16_8": (phia.OP_BF16, 8)}[path]
    return phia.Annealer(d.k, d.kh, path=phia.PATH_TC, operand=op, tc_kernel=phia.KERNEL_RESIDENT,
                         tile_replicas=tile, instance_id=INST)


def _safe_state(seed):
    x, v = ins.random_state(R, N, seed)
    xn = x.astype(np.float64) + EPS * v.astype(np.float64)
    bad = np.abs(xn) < 1e-3
    x[bad] = np.where(xn[bad] >= 0, 0.01, -0.01).astype(np.float32)
    v[bad] = 0.0
    return x, v


@pytest.mark.parametrize("path", ["tc_e4m3_8", "tc_e4m3_16", "tc_e4m3_4", "tc_bf16_8", "fp32"])
def test_acceptance_test_follows_the_oracle(gpu_lib, path):
    phia = gpu_lib
    d = ins.dense_int(N, 7, 7, seed=44)
    P = o.Instance(d.kh, k=d.k)
    x, v = _safe_state(seed=12)
    sched = phia.schedule(BETA0, BETA1, EPS, GAMMA, refresh=REFRESH, accept_test=phia.ACCEPT_METROPOLIS)
    with _handle(phia, d, path) as A:
        xt, vt = torch.from_numpy(x).cuda(), torch.from_numpy(v).cuda()
        phia.run(A.h, sched, R, 0, T, T, SEED, xt, vt)
        be, bs, _, _ = phia.replica_results(A.h, R, N)
        prop, acc = phia.acceptance(A.h, R)
        xg, vg = xt.cpu().numpy(), vt.cpu().numpy()
        st = phia.stats_get(A.h)
    if path != "fp32":
        assert st.tc_kernel == 1
    same = same_plain = 0
    o_prop = o_acc = 0
    for r in range(R):
        kw = dict(refresh=REFRESH, x0=x[r].astype(np.float64), v0=v[r].astype(np.float64))
        ref = o.anneal_replica(P, T, SEED, INST, r, BETA0, BETA1, EPS, GAMMA, accept_test=1, **kw)
        plain = o.anneal_replica(P, T, SEED, INST, r, BETA0, BETA1, EPS, GAMMA, accept_test=0, **kw)
        o_prop += ref["proposed"]
        o_acc += ref["accepted"]
        close = np.allclose(xg[r], ref["x"], atol=2e-3) and np.allclose(vg[r], ref["v"], atol=2e-3)
        same += (ref["best_e"] == be[r] and ref["best_step"] == bs[r] and ref["proposed"] == prop[r]
                 and ref["accepted"] == acc[r] and close)
        same_plain += np.allclose(xg[r], plain["x"], atol=2e-3) and np.allclose(vg[r], plain["v"], atol=2e-3)
    assert o_prop == 7 * R and 0.2 < o_acc / o_prop < 0.8, "the case must mix acceptances and rejections"
    assert (prop == 7).all()
    assert same >= int(0.9 * R), f"{path}: {same}/{R} replicas follow the oracle"
    assert same_plain <= R // 10, f"{path}: {same_plain}/{R} replicas also match a run without the test"


def test_acceptance_off_is_unchanged_and_counts_zero(gpu_lib):
    """accept_test = 0 gives the run of every other test (bit-identical to a schedule
    without the field) and zero counts; with refresh = 0 the test has nothing to test."""
    phia = gpu_lib
    d = ins.dense_int(N, 7, 7, seed=44)
    with _handle(phia, d, "tc_e4m3_8") as A:
        A.anneal(phia.schedule(BETA0, BETA1, EPS, GAMMA, refresh=REFRESH), R, T, 9)
        ref = phia.replica_results(A.h, R, N)
        A.anneal(phia.schedule(BETA0, BETA1, EPS, GAMMA, refresh=0, accept_test=1), R, T, 9)
        prop, acc = phia.acceptance(A.h, R)
        assert (prop == 0).all() and (acc == 0).all()
        A.anneal(phia.schedule(BETA0, BETA1, EPS, GAMMA, refresh=0), R, T, 9)
        b = phia.replica_results(A.h, R, N)
        A.anneal(phia.schedule(BETA0, BETA1, EPS, GAMMA, refresh=0, accept_test=1), R, T, 9)
        c = phia.replica_results(A.h, R, N)
        for u, w in zip(b, c):
            assert np.array_equal(u, w)
        A.anneal(phia.schedule(BETA0, BETA1, EPS, GAMMA, refresh=REFRESH), R, T, 9)
        for u, w in zip(ref, phia.replica_results(A.h, R, N)):
            assert np.array_equal(u, w)


def test_acceptance_test_refused_where_it_does_not_run(gpu_lib):
    phia = gpu_lib
    d = ins.dense_int(N, 7, 7, seed=44)
    sched = phia.schedule(BETA0, BETA1, EPS, GAMMA, refresh=REFRESH, accept_test=1)
    with phia.Annealer(d.k, d.kh, path=phia.PATH_TC, tc_kernel=phia.KERNEL_PER_STEP) as A:
        with pytest.raises(phia.PhiaError) as ei:
            phia.anneal(A.h, sched, R, T, 1)
        assert ei.value.code == phia.ENOTSUP
