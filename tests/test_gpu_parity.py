"""GPU parity tests: the CUDA path through the C ABI against the FP64 oracle.

Bar: integer fields and energies bit-exact; one iteration from identical FP32 state
within 1e-5 relative (to the magnitude of the update's terms) in FP32; Philox words
bit-exact; full runs judged by invariants (returned energy = Eq. 2 on the returned
spins, never below the exhaustive minimum) and by success statistics.
"""
import math

import numpy as np
import pytest

import oracle as o
from paper_2407_10205_gb300 import instances as ins

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TC_E4M3 = ("tc", 1)
TC_BF16 = ("tc", 2)
TC_E4M3_TM = ("tc", 1, 2)   # couplings kept in tensor memory
TC_BF16_TM = ("tc", 2, 2)
FP32 = ("fp32", 0)
IMMA8 = ("imma", 8)          # int8 mma.sync kernel, 8 replicas per CTA
IMMA16 = ("imma", 16)


def _handle(phia, d, path, frac=0):
    kind, op = path[0], path[1]
    mem = path[2] if len(path) > 2 else 0
    if kind == "imma":
        return phia.Annealer(d.k, d.kh, frac_bits=frac, path=phia.PATH_TC, tc_kernel=phia.KERNEL_IMMA,
                             tile_replicas=op)
    p = phia.PATH_TC if kind == "tc" else phia.PATH_FP32
    return phia.Annealer(d.k, d.kh, frac_bits=frac, path=p, operand=op, coupling_mem=mem)


def _oinst(d, frac=0):
    return o.Instance(d.kh, k=d.k, frac_bits=frac)


# ------------------------------------------------------------------ Philox

def test_philox_words_bit_exact(gpu_lib):
    phia = gpu_lib
    R, N, seed, inst = 5, 37, 0x1234_5678_9ABC_DEF0, 3
    for d in (0, 17):
        raw = torch.empty((R, N, 4), dtype=torch.int32, device="cuda")
        x = torch.empty((R, N), dtype=torch.float32, device="cuda")
        v = torch.empty((R, N), dtype=torch.float32, device="cuda")
        phia.philox_draws(seed, inst, d, R, N, raw, x, v)
        torch.cuda.synchronize()
        raw = raw.cpu().numpy().view(np.uint32)
        X, V = o.draw_grid(seed, inst, R, N, d)
        for r in range(R):
            for j in range(N):
                assert list(raw[r, j]) == o.philox4x32_10([j, r, d, inst], [seed & 0xFFFFFFFF, seed >> 32])
        xs, vs = x.cpu().numpy(), v.cpu().numpy()
        assert np.all(np.abs(xs - X) <= 4e-6 * (1 + np.abs(X)))
        assert np.all(np.abs(vs - V) <= 4e-6 * (1 + np.abs(V)))


# ------------------------------------------------------------------ field (Eq. 6) and energy (Eq. 2)

FIELD_CASES = [
    # (path, N, R, kmax, hmax)
    (TC_E4M3, 3, 1, 1, 0), (TC_E4M3, 16, 17, 1, 0), (TC_E4M3, 33, 40, 7, 7), (TC_E4M3, 130, 33, 16, 100),
    (TC_E4M3, 200, 64, 7, 7), (TC_E4M3, 257, 20, 16, 1000), (TC_E4M3, 384, 16, 16, 5),
    (TC_BF16, 5, 3, 127, 9), (TC_BF16, 100, 31, 127, 1 << 20), (TC_BF16, 256, 48, 127, 127),
    (FP32, 7, 5, 7, 7), (FP32, 200, 64, 7, 7), (FP32, 333, 19, 127, 50),
    (TC_E4M3_TM, 3, 1, 1, 0), (TC_E4M3_TM, 200, 64, 7, 7), (TC_E4M3_TM, 384, 16, 16, 5),
    (TC_BF16_TM, 5, 3, 127, 9), (TC_BF16_TM, 256, 48, 127, 127),
    (IMMA8, 3, 1, 1, 0), (IMMA8, 33, 40, 127, 1 << 20), (IMMA8, 200, 64, 7, 7), (IMMA16, 256, 37, 127, 127),
    (IMMA16, 100, 16, 127, 9),
]


@pytest.mark.parametrize("path,N,R,kmax,hmax", FIELD_CASES)
def test_field_and_energy_bit_exact(gpu_lib, path, N, R, kmax, hmax):
    phia = gpu_lib
    d = ins.dense_int(N, kmax, hmax, seed=N * 7 + R)
    S = ins.random_spins(R, N, seed=N + 3)
    with _handle(phia, d, path) as A:
        f = torch.empty((R, N), dtype=torch.int32, device="cuda")
        e = torch.empty(R, dtype=torch.int64, device="cuda")
        phia.field(A.h, torch.from_numpy(S).cuda(), f, e)
        torch.cuda.synchronize()
        I, E = o.field_batch(_oinst(d), S)
        assert np.array_equal(f.cpu().numpy(), I)
        assert np.array_equal(e.cpu().numpy(), E)


@pytest.mark.parametrize("path,N,kval", [(TC_E4M3, 384, 16), (TC_E4M3, 384, -16), (TC_BF16, 256, 127),
                                         (TC_BF16, 256, -127), (FP32, 384, 127), (TC_E4M3_TM, 384, 16),
                                         (TC_BF16_TM, 256, -127), (IMMA8, 256, 127), (IMMA16, 256, -127)])
def test_field_extreme_magnitudes(gpu_lib, path, N, kval):
    """Every product of one sign at the largest exact |k|: the accumulator's largest
    partial sums (|I| = |k| (N - 1)) must stay exact; alternating states as well."""
    phia = gpu_lib
    k = np.full((N, N), kval, dtype=np.int8)
    np.fill_diagonal(k, 0)
    # the tensor-core path adds h as an exact int32; the FP32 path needs |I| < 2^24
    hmax = (1 << 24) - 1 if path[0] == "tc" else 1 << 22
    d = ins.Dense(k, np.full(N, hmax, dtype=np.int32))
    S = np.ones((4, N), dtype=np.int8)
    S[1] = -1
    S[2, ::2] = -1
    S[3, : N // 2] = -1
    with _handle(phia, d, path) as A:
        f = torch.empty((4, N), dtype=torch.int32, device="cuda")
        e = torch.empty(4, dtype=torch.int64, device="cuda")
        phia.field(A.h, torch.from_numpy(S).cuda(), f, e)
        torch.cuda.synchronize()
        I, E = o.field_batch(_oinst(d), S)
        assert np.array_equal(f.cpu().numpy(), I)
        assert np.array_equal(e.cpu().numpy(), E)


# ------------------------------------------------------------------ one iteration (Eq. A7)

def _safe_state(R, N, eps, seed):
    """FP32 states whose new positions x + eps v stay away from 0, so the sign is not
    decided by rounding (the paper leaves sgn(0) open; FP32 and FP64 may differ there)."""
    x, v = ins.random_state(R, N, seed)
    xn = x.astype(np.float64) + eps * v.astype(np.float64)
    bad = np.abs(xn) < 1e-3
    x[bad] = np.where(xn[bad] >= 0, 0.01, -0.01).astype(np.float32)
    v[bad] = 0.0
    return x, v


STEP_CASES = [(TC_E4M3, 16, 16, 1, 0, 0), (TC_E4M3, 200, 40, 7, 7, 0), (TC_BF16, 150, 20, 127, 31, 4),
              (TC_E4M3, 333, 17, 16, 16, 3), (FP32, 200, 40, 7, 7, 0), (FP32, 77, 9, 127, 31, 4),
              (IMMA8, 200, 40, 7, 7, 0), (IMMA16, 150, 20, 127, 31, 4)]


@pytest.mark.parametrize("path,N,R,kmax,hmax,frac", STEP_CASES)
def test_single_step_matches_oracle(gpu_lib, path, N, R, kmax, hmax, frac):
    phia = gpu_lib
    eps, gamma, beta = 0.1, 2.0, 0.37
    d = ins.dense_int(N, kmax, hmax, seed=N + R)
    P = _oinst(d, frac)
    x, v = _safe_state(R, N, eps, seed=N * R)
    sched = phia.schedule(beta, beta, eps, gamma)
    with _handle(phia, d, path, frac) as A:
        xt, vt = torch.from_numpy(x).cuda(), torch.from_numpy(v).cuda()
        phia.run(A.h, sched, R, 0, 1, 1, 7, xt, vt)
        be, bs, hs, bits = phia.replica_results(A.h, R, N)
        xg, vg = xt.cpu().numpy(), vt.cpu().numpy()
    S = phia.unpack_bits(bits, N)
    for r in range(R):
        xo, vo, so, Io, eo = o.step(P, x[r].astype(np.float64), v[r].astype(np.float64), beta, eps, gamma)
        assert np.array_equal(S[r], so), "sign readout differs"
        assert be[r] == eo and bs[r] == 0, "energy differs"
        assert np.allclose(xg[r], xo, rtol=1e-6, atol=1e-7)
        # 1e-5 relative to the size of the terms of the momentum update
        scale = np.abs(v[r]) + eps * (beta * gamma * P.q * np.abs(Io) + np.abs(xo))
        assert np.all(np.abs(vg[r] - vo) <= 1e-5 * np.maximum(scale, 1e-3))


def test_initial_state_matches_oracle_draws(gpu_lib):
    phia = gpu_lib
    d = ins.sk_pm1(40, 1)
    R, seed = 6, 99
    with phia.Annealer(d.k, d.kh, path=phia.PATH_TC, instance_id=11) as A:
        x = torch.empty((R, 40), device="cuda"); v = torch.empty((R, 40), device="cuda")
        phia.init_state(A.h, R, seed, x, v)
        torch.cuda.synchronize()
    X, V = o.draw_grid(seed, 11, R, 40, 0)
    assert np.all(np.abs(x.cpu().numpy() - X) <= 4e-6 * (1 + np.abs(X)))
    assert np.all(np.abs(v.cpu().numpy() - V) <= 4e-6 * (1 + np.abs(V)))


# ------------------------------------------------------------------ runs

@pytest.mark.parametrize("path", [TC_E4M3, FP32])
def test_run_invariants_small_sk(gpu_lib, path):
    """N = 16 SK, seed 0 (J in {-1,+1}, h = 0): returned energies equal Eq. 2 on the
    returned spins, never go below the exhaustive minimum, and most replicas reach it."""
    phia = gpu_lib
    d = ins.sk_pm1(16, 0)
    P = _oinst(d)
    emin, _, _ = o.brute_force(P)
    R = 64
    with _handle(phia, d, path) as A:
        res = A.anneal(phia.schedule(0.05, 2.0, 0.2, 2.0), R, 1000, seed=1)
        be, bs, hs, bits = phia.replica_results(A.h, R, 16)
    S = phia.unpack_bits(bits, 16)
    for r in range(R):
        assert o.energy_exact(P, S[r]) == be[r]
    assert (be >= emin).all() and res.energy_k == be.min()
    assert o.energy_exact(P, res.spins) == res.energy_k
    assert np.mean(be == emin) > 0.8
    assert res.stats.spin_updates == R * 16 * 1000


@pytest.mark.parametrize("kern", ["resident", "per_iteration", "fp32"])
def test_config1_single_replica_reaches_ground_state(gpu_lib, kern):
    """The plain-PHIA case exactly: N = 16 SK, seed 0, one replica, 1000 iterations, FP32 on
    the GPU and FP64 in the oracle with the same seeds; both reach the exhaustive minimum
    (2^16 states) and the GPU's returned energy is Eq. 2 on its returned spins."""
    phia = gpu_lib
    d = ins.sk_pm1(16, 0)
    P = _oinst(d)
    emin, _, _ = o.brute_force(P)
    if kern == "fp32":
        h = phia.Annealer(d.k, d.kh, path=phia.PATH_FP32)
    else:
        h = phia.Annealer(d.k, d.kh, path=phia.PATH_TC,
                          tc_kernel=phia.KERNEL_RESIDENT if kern == "resident" else phia.KERNEL_PER_STEP)
    with h as A:
        for seed in (1, 2, 3):
            ref = o.anneal(P, 1, 1000, seed, 0, 0.05, 2.0, 0.2, 2.0)
            res = A.anneal(phia.schedule(0.05, 2.0, 0.2, 2.0), 1, 1000, seed=seed)
            assert ref["best_e"][0] == emin == res.energy_k
            assert o.energy_exact(P, res.spins) == res.energy_k
            assert res.stats.spin_updates == 16 * 1000


def test_short_trajectories_follow_the_oracle(gpu_lib):
    """From identical initial states, 12 iterations on the GPU (FP32) and in the oracle
    (FP64) give the same per-replica best energies for nearly every replica; the few
    that may differ are those whose sign was decided within FP32 rounding."""
    phia = gpu_lib
    N, R, T, eps = 200, 64, 12, 0.1
    d = ins.dense_int(N, 7, 7, seed=5)
    P = _oinst(d)
    x, v = _safe_state(R, N, eps, seed=8)
    sched = phia.schedule(0.01, 0.1, eps, 2.0)
    with _handle(phia, d, TC_E4M3) as A:
        xt, vt = torch.from_numpy(x).cuda(), torch.from_numpy(v).cuda()
        phia.run(A.h, sched, R, 0, T, T, 3, xt, vt)
        be, bs, _, _ = phia.replica_results(A.h, R, N)
        xg = xt.cpu().numpy()
    same = 0
    for r in range(R):
        ref = o.anneal_replica(P, T, 3, 0, r, 0.01, 0.1, eps, 2.0,
                               x0=x[r].astype(np.float64), v0=v[r].astype(np.float64))
        if ref["best_e"] == be[r] and ref["best_step"] == bs[r] and np.allclose(xg[r], ref["x"], atol=1e-3):
            same += 1
    assert same >= int(0.9 * R)


def test_resume_is_bit_identical(gpu_lib):
    """Philox counters and beta_t depend on the absolute iteration, so [0,a) then [a,T)
    reproduces [0,T) exactly (state and records)."""
    phia = gpu_lib
    N, R, T, a = 200, 48, 300, 113
    d = ins.dense_int(N, 7, 7, seed=9)
    sched = phia.schedule(0.01, 0.1, 0.1, 2.0, refresh=50)
    with _handle(phia, d, TC_E4M3) as A:
        x1 = torch.empty((R, N), device="cuda"); v1 = torch.empty((R, N), device="cuda")
        phia.init_state(A.h, R, 5, x1, v1)
        x2, v2 = x1.clone(), v1.clone()
        phia.run(A.h, sched, R, 0, T, T, 5, x1, v1, reset_best=True)
        one = phia.replica_results(A.h, R, N)
        phia.run(A.h, sched, R, 0, a, T, 5, x2, v2, reset_best=True)
        phia.run(A.h, sched, R, a, T - a, T, 5, x2, v2, reset_best=False)
        two = phia.replica_results(A.h, R, N)
        torch.cuda.synchronize()
        assert torch.equal(x1, x2) and torch.equal(v1, v2)
        for u, w in zip(one, two):
            assert np.array_equal(u, w)
        # and the one-shot anneal equals init_state + run
        A.anneal(sched, R, T, 5)
        three = phia.replica_results(A.h, R, N)
        for u, w in zip(one, three):
            assert np.array_equal(u, w)


def test_success_statistics_match_oracle(gpu_lib):
    """Success probability on N = 16 SK with a short run (so that P is near 1/2): GPU
    (FP32, 512 replicas) and oracle (FP64, 512 replicas, same seeds) agree within a
    two-proportion 99.9% interval."""
    phia = gpu_lib
    d = ins.sk_pm1(16, 0)
    P = _oinst(d)
    emin, _, _ = o.brute_force(P)
    R, T = 512, 30
    with _handle(phia, d, TC_E4M3) as A:
        A.anneal(phia.schedule(0.05, 2.0, 0.2, 2.0), R, T, seed=2)
        be, _, _, _ = phia.replica_results(A.h, R, 16)
    ref = o.anneal(P, R, T, 2, 0, 0.05, 2.0, 0.2, 2.0)
    p1, p2 = np.mean(be == emin), np.mean(ref["best_e"] == emin)
    pp = (p1 + p2) / 2
    z = abs(p1 - p2) / math.sqrt(max(pp * (1 - pp) * 2 / R, 1e-12))
    assert 0.05 < p2 < 0.95, f"oracle success rate {p2} not informative"
    assert z < 3.3, f"GPU P={p1:.3f} vs oracle P={p2:.3f}"


def test_stop_at_target(gpu_lib):
    phia = gpu_lib
    d = ins.sk_pm1(16, 0)
    P = _oinst(d)
    emin, _, _ = o.brute_force(P)
    R, T = 64, 1000
    sched = phia.schedule(0.05, 2.0, 0.2, 2.0, target=emin, stop_at_target=True)
    with _handle(phia, d, TC_E4M3) as A:
        res = A.anneal(sched, R, T, seed=4)
        full = phia.schedule(0.05, 2.0, 0.2, 2.0, target=emin)
        res_full = A.anneal(full, R, T, seed=4)
        _, _, hs_full, _ = phia.replica_results(A.h, R, 16)
    assert res.energy_k <= emin and o.energy_exact(P, res.spins) == res.energy_k
    assert res.stats.hit_step == hs_full[hs_full >= 0].min()
    assert res.stats.spin_updates < res_full.stats.spin_updates


@pytest.mark.parametrize("N,op", [(200, 1), (333, 1), (100, 2)])
def test_tile_variants_bit_identical(gpu_lib, N, op):
    """Replicas per CTA (4, 8, 16) and where J is kept (shared or tensor memory) change
    only the work split and the operand source: every replica's arithmetic is the same,
    so per-replica records and final states must be bit-identical."""
    phia = gpu_lib
    R, T = 50, 150
    kmax = 7 if op == 1 else 100
    d = ins.dense_int(N, kmax, 7, seed=N)
    sched = phia.schedule(0.01, 0.2, 0.1, 2.0, refresh=40)
    outs = []
    variants = [dict(tile_replicas=t, coupling_mem=m) for t, m in ((4, 1), (8, 1), (16, 1), (4, 2), (8, 2), (16, 2))]
    if N <= 256:
        variants += [dict(tile_replicas=8, tc_kernel=3), dict(tile_replicas=16, tc_kernel=3)]
    for kw in variants:
        with phia.Annealer(d.k, d.kh, path=phia.PATH_TC, operand=op, **kw) as A:
            x = torch.empty((R, N), device="cuda"); v = torch.empty((R, N), device="cuda")
            phia.init_state(A.h, R, 17, x, v)
            phia.run(A.h, sched, R, 0, T, T, 17, x, v)
            outs.append((phia.replica_results(A.h, R, N), x.cpu().numpy(), v.cpu().numpy()))
    for rec, x, v in outs[1:]:
        for u, w in zip(outs[0][0], rec):
            assert np.array_equal(u, w)
        assert np.array_equal(outs[0][1], x) and np.array_equal(outs[0][2], v)
