"""GPU parity of vanilla GAHMC (exact dynamics by zero crossings; Sec. 2.1 and its
reference [Pakman & Paninski 2013]; the ablation of Sec. 3.2) against the FP64 oracle.

- the hand-worked 2-spin trajectory of tests/golden/gahmc_two_spin.txt: the event
  sequence (a crossing, then a reflection), final spins, best energy, and final x, v
  within FP32 rounding;
- random instances from identical FP32 states: per replica, the whole sequence of wall
  events (which spin, crossed or reflected), the counts, the best energy and the
  trajectory that first reached it, and the final spins equal the oracle's for >= 90% of
  replicas (a replica may differ where FP32 and FP64 order two nearly simultaneous
  events, or decide a crossing at its threshold, differently);
- the exact dynamics conserve H (App. A) within a trajectory: on the GPU to FP32
  rounding;
- returned best energies equal Eq. 2 on the returned best spins.
"""
import math

import numpy as np
import pytest

import oracle as o
from paper_2407_10205_gb300 import instances as ins
from conftest import read_golden

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _f64(text):
    return np.array(text.split(), dtype=np.float64)


def test_gahmc_hand_case_on_the_gpu(gpu_lib):
    phia = gpu_lib
    g = read_golden("gahmc_two_spin.txt")
    k = np.array(g["k"].split(), dtype=np.int8).reshape(2, 2)
    kh = np.zeros(2, dtype=np.int32)
    x = torch.from_numpy(_f64(g["x0"]).astype(np.float32)[None, :]).cuda()
    v = torch.from_numpy(_f64(g["v0"]).astype(np.float32)[None, :]).cuda()
    counts = torch.zeros((1, 2), dtype=torch.int64, device="cuda")
    events = torch.full((1, 4), -(2**31), dtype=torch.int32, device="cuda")
    b = float(g["beta"])
    with phia.Annealer(k, kh, path=phia.PATH_TC) as A:
        phia.gahmc(A.h, phia.gahmc_schedule(b, b, float(g["travel"])), 1, 1, 0, x, v, counts, events)
        e, spins = phia.best(A.h, 2)
    assert list(events.cpu().numpy()[0, :2]) == [int(t) for t in g["events"].split()]
    assert list(counts.cpu().numpy()[0]) == [1, 1]
    assert np.allclose(x.cpu().numpy()[0], _f64(g["x_end"]), atol=2e-6)
    assert np.allclose(v.cpu().numpy()[0], _f64(g["v_end"]), atol=2e-6)
    assert e == int(g["best_e"]) and list(spins) == [int(t) for t in g["s_end"].split()]


CASES = [  # (N, kmax, hmax, frac, trajectories, beta0, beta1)
    (64, 7, 7, 0, 30, 0.01, 0.3), (200, 7, 7, 0, 12, 0.005, 0.1), (130, 127, 31, 4, 10, 0.002, 0.05),
    (1024, 1, 0, 0, 3, 0.01, 0.05),
]


@pytest.mark.parametrize("N,kmax,hmax,frac,K,b0,b1", CASES)
def test_gahmc_event_sequences_follow_the_oracle(gpu_lib, N, kmax, hmax, frac, K, b0, b1):
    phia = gpu_lib
    R, cap, seed, inst = 64, 4096, 21, 6
    d = ins.dense_int(N, kmax, hmax, seed=N + K, frac_bits=frac)
    P = o.Instance(d.kh, k=d.k, frac_bits=frac)
    x0, v0 = ins.random_state(R, N, seed=N, min_abs=1e-3)
    x = torch.from_numpy(x0).cuda()
    v = torch.from_numpy(v0).cuda()
    counts = torch.zeros((R, 2), dtype=torch.int64, device="cuda")
    events = torch.full((R, cap), -(2**31), dtype=torch.int32, device="cuda")
    with phia.Annealer(d.k, d.kh, frac_bits=frac, path=phia.PATH_TC, instance_id=inst) as A:
        phia.gahmc(A.h, phia.gahmc_schedule(b0, b1, math.pi / 2), R, K, seed, x, v, counts, events)
        be, bs, _, bits = phia.replica_results(A.h, R, N)
        st = phia.stats_get(A.h)
    assert st.spin_updates == R * N * K
    ev, cn, xg = events.cpu().numpy(), counts.cpu().numpy(), x.cpu().numpy()
    S = phia.unpack_bits(bits, N)
    same = 0
    for r in range(R):
        ref = o.gahmc_replica(P, K, seed, inst, r, b0, b1, math.pi / 2, x0=x0[r].astype(np.float64),
                              v0=v0[r].astype(np.float64), events_cap=cap)
        assert o.energy_exact(P, S[r]) == be[r], "best energy is not Eq. 2 of the best spins"
        n_ev = int(cn[r].sum())
        same += (n_ev <= cap and np.array_equal(ev[r, :n_ev], ref["events"])
                 and list(cn[r]) == [ref["crossings"], ref["reflections"]]
                 and be[r] == ref["best_e"] and bs[r] == ref["best_traj"]
                 and np.array_equal(np.where(xg[r] >= 0, 1, -1), ref["s"]))
    assert same >= int(0.9 * R), f"{same}/{R} replicas follow the oracle's event sequence"


def test_gahmc_conserves_h_within_a_trajectory_on_the_gpu(gpu_lib):
    phia = gpu_lib
    N, R, beta = 150, 32, 0.3
    d = ins.dense_int(N, 7, 7, seed=8, frac_bits=2)
    P = o.Instance(d.kh, k=d.k, frac_bits=2)
    x0, v0 = ins.random_state(R, N, seed=9, min_abs=1e-3)
    v0 *= 2.0
    x, v = torch.from_numpy(x0).cuda(), torch.from_numpy(v0).cuda()
    counts = torch.zeros((R, 2), dtype=torch.int64, device="cuda")
    with phia.Annealer(d.k, d.kh, frac_bits=2, path=phia.PATH_TC) as A:
        phia.gahmc(A.h, phia.gahmc_schedule(beta, beta, math.pi), R, 1, 1, x, v, counts)
    xg, vg, cn = x.cpu().numpy().astype(np.float64), v.cpu().numpy().astype(np.float64), counts.cpu().numpy()
    assert (cn[:, 0] > 0).all() and (cn[:, 1] > 0).all()
    for r in range(R):
        s0 = np.where(x0[r] >= 0, 1, -1).astype(np.int8)
        s1 = np.where(xg[r] >= 0, 1, -1).astype(np.int8)
        h0 = o.hamiltonian(beta, P.q, o.energy_exact(P, s0), x0[r].astype(np.float64), v0[r].astype(np.float64))
        h1 = o.hamiltonian(beta, P.q, o.energy_exact(P, s1), xg[r], vg[r])
        assert abs(h1 - h0) <= 1e-4 * abs(h0) + 1e-3, (r, h0, h1)
