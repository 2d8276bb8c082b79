"""Pins for the FP64 oracle against what the paper and mathematics fix (no GPU).

Each test pins one function of oracle/ to something other than itself:
published known-answer vectors, closed forms, a hand-worked example, exact
discrete invariants, symmetries and exhaustive enumeration.
"""
import math
import os

import numpy as np
import pytest

import oracle as o
from paper_2407_10205_gb300 import instances as ins
from conftest import GOLDEN, read_golden


def _dense(k, kh, f=0):
    return o.Instance(np.asarray(kh, dtype=np.int32), k=np.asarray(k, dtype=np.int8), frac_bits=f)


# ------------------------------------------------------------------ Philox

def test_philox_known_answers():
    """Philox4x32-10 against the Random123 known-answer vectors (Salmon et al., SC'11)."""
    n = 0
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(t, 16) for t in line.split()]
            assert o.philox4x32_10(w[0:4], w[4:6]) == w[6:10]
            n += 1
    assert n == 3


def test_uniform_and_box_muller_closed_forms():
    # u in (0,1] on 24 bits: all-ones maps to exactly 1, zero to 2^-24
    assert o.u01_open(0xFFFFFFFF) == 1.0
    assert o.u01_open(0) == 2.0 ** -24
    assert o.u01_half(0) == 0.0
    assert o.u01_half(0x80000000) == 0.5
    # u1 = 1 -> radius 0
    assert o.box_muller(0xFFFFFFFF, 12345) == 0.0
    # u1 = 2^-24, u2 = 0 -> sqrt(-2 ln 2^-24) = sqrt(48 ln 2)
    assert o.box_muller(0, 0) == pytest.approx(math.sqrt(48 * math.log(2)), rel=1e-15)
    # u2 = 1/2 -> cos(pi) = -1
    assert o.box_muller(0, 0x80000000) == pytest.approx(-math.sqrt(48 * math.log(2)), rel=1e-15)
    # u2 = 1/4 -> cos(pi/2) = 0
    assert abs(o.box_muller(0, 0x40000000)) < 1e-14


def test_draws_are_standard_normal():
    from scipy import stats
    X, V = o.draw_grid(seed=7, inst=3, R=40, n=250, d=0)
    for a in (X.ravel(), V.ravel()):
        assert abs(a.mean()) < 0.03
        assert abs(a.var() - 1) < 0.04
        assert stats.kstest(a, "norm").pvalue > 1e-3
    # position and momentum draws are different words of the same block
    assert np.corrcoef(X.ravel(), V.ravel())[0, 1] < 0.05
    # the counter separates replicas, spins, draw indices and instances
    a = o.draw(7, 3, 0, 0, 0)
    assert a != o.draw(7, 3, 1, 0, 0) and a != o.draw(7, 3, 0, 1, 0)
    assert a != o.draw(7, 3, 0, 0, 1) and a != o.draw(7, 4, 0, 0, 0) and a != o.draw(8, 3, 0, 0, 0)


# ------------------------------------------------------------------ energy

def test_three_spin_energy_table():
    g = read_golden("three_spin_step.txt")
    k = np.array(g["J"].split(), dtype=np.int8).reshape(3, 3)
    kh = np.array(g["h"].split(), dtype=np.int32)
    P = _dense(k, kh)
    for item in g["energies_by_state"].split():
        st, e = item.split(":")
        s = np.array([1 if c == "+" else -1 for c in st], dtype=np.int8)
        assert o.energy_exact(P, s) == int(e)
    emin, cnt, arg = o.brute_force(P)
    assert emin == int(g["ground_energy"])
    assert cnt == int(g["ground_count"])
    assert list(arg) == [int(t) for t in g["ground_state"].split()]


@pytest.mark.parametrize("n", [2, 5, 9, 12])
def test_ferromagnet_closed_form(n):
    """All J_ij = +1, h = 0: ground energy -n(n-1)/2, reached only by the two aligned states."""
    k = np.ones((n, n), dtype=np.int8) - np.eye(n, dtype=np.int8)
    P = _dense(k, np.zeros(n))
    emin, cnt, _ = o.brute_force(P)
    assert emin == -n * (n - 1) // 2 and cnt == 2
    assert o.energy_exact(P, np.ones(n)) == -n * (n - 1) // 2


def test_antiferromagnetic_triangle():
    """J = -1 on a triangle: frustrated, ground energy -1 with six ground states."""
    k = -(np.ones((3, 3), dtype=np.int8) - np.eye(3, dtype=np.int8))
    emin, cnt, _ = o.brute_force(_dense(k, np.zeros(3)))
    assert (emin, cnt) == (-1, 6)


@pytest.mark.parametrize("n", [4, 10, 15])
def test_open_chain(n):
    k = np.zeros((n, n), dtype=np.int8)
    for i in range(n - 1):
        k[i, i + 1] = k[i + 1, i] = 1
    emin, cnt, _ = o.brute_force(_dense(k, np.zeros(n)))
    assert (emin, cnt) == (-(n - 1), 2)


def test_independent_spins():
    """J = 0: the ground state is s = sgn h with E = -sum |h|, unique when no h is 0."""
    g = np.random.default_rng(1)
    kh = g.integers(1, 50, size=11) * np.where(g.random(11) < 0.5, -1, 1)
    P = _dense(np.zeros((11, 11)), kh)
    emin, cnt, arg = o.brute_force(P)
    assert emin == -np.abs(kh).sum() and cnt == 1
    assert np.array_equal(arg, np.sign(kh))


def test_field_is_minus_energy_gradient():
    """Eq. 6 as a discrete derivative of Eq. 2: flipping spin k changes E by 2 s_k I_k."""
    d = ins.dense_int(23, 9, 20, seed=5)
    P = _dense(d.k, d.kh)
    s = ins.random_spins(1, 23, seed=6)[0]
    I = o.field(P, s)
    e0 = o.energy_exact(P, s)
    for kidx in range(23):
        t = s.copy(); t[kidx] = -t[kidx]
        assert o.energy_exact(P, t) - e0 == 2 * int(s[kidx]) * int(I[kidx])


def test_energy_identity_and_csr_agree():
    """E = -1/2 sum s (I + h) equals Eq. 2; the CSR and dense forms agree."""
    c = ins.erdos_renyi(120, 0.08, 127, 31, 4, seed=2)
    dd = c.to_dense()
    Pc = o.Instance(c.kh, row_ptr=c.row_ptr, col=c.col, val=c.val, frac_bits=4)
    Pd = o.Instance(dd.kh, k=dd.k, frac_bits=4)
    S = ins.random_spins(20, 120, seed=3)
    for s in S:
        Ic, Id = o.field(Pc, s), o.field(Pd, s)
        assert np.array_equal(Ic, Id)
        e = o.energy_exact(Pd, s)
        assert o.energy_exact(Pc, s) == e
        assert o.energy_from_field(Pd, s, Id) == e


def test_flip_symmetry_without_field():
    d = ins.sk_pm1(40, seed=4)
    P = _dense(d.k, d.kh)
    for s in ins.random_spins(10, 40, seed=5):
        assert o.energy_exact(P, s) == o.energy_exact(P, -s)


# ------------------------------------------------------------------ update

def test_three_spin_step_matches_hand_derivation():
    g = read_golden("three_spin_step.txt")
    k = np.array(g["J"].split(), dtype=np.int8).reshape(3, 3)
    kh = np.array(g["h"].split(), dtype=np.int32)
    P = _dense(k, kh)
    f = lambda key: np.array(g[key].split(), dtype=np.float64)
    x, v, s, I, e = o.step(P, f("x"), f("v"), float(g["beta"]), float(g["eps"]), float(g["gamma"]))
    assert np.allclose(x, f("x_new"), rtol=0, atol=1e-15)
    assert list(s) == [int(t) for t in g["s"].split()]
    assert list(I) == [int(t) for t in g["I"].split()]
    assert e == int(g["E"])
    assert np.allclose(v, f("v_new"), rtol=1e-14, atol=0)


def test_quadratic_derivative_factor():
    """The quadratic stand-in for the derivative factor of Eq. 8 (deriv = 1; the paper's
    FPGA uses a quadratic fit whose coefficients it does not print, these are chosen
    here): 1 at y = 0, 0 from |y| = 1.5 on, even, never above 1, and its integral over
    the real line is 2, the integral of the exact factor sech^2 (tanh(+inf) -
    tanh(-inf)), both checked by the midpoint rule."""
    assert o.dfactor(0.0, 1) == 1.0 and o.dfactor(0.0, 0) == 1.0
    for y in (1.5, -1.5, 1.6, -7.0, 40.0):
        assert o.dfactor(y, 1) == 0.0
    ys = np.linspace(-2.0, 2.0, 401)
    q = np.array([o.dfactor(y, 1) for y in ys])
    qm = np.array([o.dfactor(-y, 1) for y in ys])
    assert np.all(q <= 1.0) and np.array_equal(q, qm)
    h = 1e-4
    mid = np.arange(-1.5 + h / 2, 1.5, h)
    assert abs(sum(o.dfactor(y, 1) for y in mid) * h - 2.0) < 1e-6
    mid = np.arange(-12.0 + h / 2, 12.0, h)
    assert abs(sum(o.dfactor(y, 0) for y in mid) * h - 2.0) < 1e-6


def test_quadratic_derivative_step():
    """deriv = 1 changes only the derivative factor: where every |gamma x'| >= 1.5 the
    field term vanishes (v' = v - eps x' exactly); where every x' = 0 both factors are 1
    and the update equals the exact one; elsewhere the two differ."""
    g = read_golden("three_spin_step.txt")
    k = np.array(g["J"].split(), dtype=np.int8).reshape(3, 3)
    kh = np.array(g["h"].split(), dtype=np.int32)
    P = _dense(k, kh)
    eps, gamma, beta = 0.1, 2.0, 1.3
    x, v = np.array([1.0, -1.0, 2.0]), np.array([0.5, -0.5, 0.1])
    xn, vn, *_ = o.step(P, x, v, beta, eps, gamma, deriv=1)
    assert np.all(np.abs(gamma * xn) >= 1.5)
    assert np.array_equal(vn, v - eps * xn)
    v0 = np.array([0.3, -0.7, 1.1])
    x0 = -(eps * v0)
    a = o.step(P, x0, v0, beta, eps, gamma, deriv=1)
    b = o.step(P, x0, v0, beta, eps, gamma, deriv=0)
    assert np.array_equal(a[0], np.zeros(3)) and np.array_equal(a[1], b[1])
    c = o.step(P, f64(g["x"]), f64(g["v"]), beta, eps, gamma, deriv=1)
    d = o.step(P, f64(g["x"]), f64(g["v"]), beta, eps, gamma, deriv=0)
    assert not np.allclose(c[1], d[1])


def f64(text):
    return np.array(text.split(), dtype=np.float64)


def test_beta_zero_discrete_invariant():
    """With beta = 0 the update is symplectic Euler on a unit oscillator per spin;
    x^2 + v^2 + eps x v is then exactly conserved (up to FP64 rounding)."""
    d = ins.dense_int(8, 5, 5, seed=9)
    P = _dense(d.k, d.kh)
    g = np.random.default_rng(0)
    x, v, eps = g.standard_normal(8), g.standard_normal(8), 0.3
    inv0 = x * x + v * v + eps * x * v
    for _ in range(10000):
        x, v, *_ = o.step(P, x, v, 0.0, eps, 2.0)
    assert np.allclose(x * x + v * v + eps * x * v, inv0, rtol=1e-11)


def test_mirror_symmetry_without_field():
    """h = 0: the dynamics are odd, (x, v) -> (-x, -v) maps a step onto its mirror."""
    d = ins.sk_pm1(30, seed=10)
    P = _dense(d.k, d.kh)
    x, v = ins.random_state(1, 30, seed=11, min_abs=0.05)
    x = x[0].astype(np.float64); v = v[0].astype(np.float64) * 0.1
    a = o.step(P, x, v, 0.7, 0.1, 3.0)
    b = o.step(P, -x, -v, 0.7, 0.1, 3.0)
    assert np.array_equal(a[0], -b[0]) and np.array_equal(a[1], -b[1])
    assert np.array_equal(a[2], -b[2]) and a[4] == b[4]


def test_fixed_point_scale_invariance():
    """J = k 2^-f: doubling k and h while adding one fractional bit leaves the step unchanged."""
    d = ins.dense_int(25, 30, 30, seed=12)
    P1 = _dense(d.k, d.kh, f=3)
    P2 = _dense(d.k.astype(np.int16) * 2, d.kh * 2, f=4)
    x, v = ins.random_state(1, 25, seed=13, min_abs=0.05)
    x = x[0].astype(np.float64); v = v[0].astype(np.float64)
    a = o.step(P1, x, v, 0.4, 0.1, 2.0)
    b = o.step(P2, x, v, 0.4, 0.1, 2.0)
    assert np.array_equal(a[0], b[0]) and np.allclose(a[1], b[1], rtol=1e-15)
    assert np.array_equal(a[2], b[2]) and np.array_equal(2 * a[3], b[3]) and 2 * a[4] == b[4]


def test_permutation_equivariance():
    d = ins.dense_int(17, 7, 7, seed=14)
    perm = np.random.default_rng(15).permutation(17)
    P = _dense(d.k, d.kh)
    Pp = _dense(d.k[np.ix_(perm, perm)], d.kh[perm])
    x, v = ins.random_state(1, 17, seed=16, min_abs=0.05)
    x = x[0].astype(np.float64); v = v[0].astype(np.float64)
    a = o.step(P, x, v, 0.3, 0.1, 2.0)
    b = o.step(Pp, x[perm], v[perm], 0.3, 0.1, 2.0)
    assert np.array_equal(a[0][perm], b[0]) and np.array_equal(a[1][perm], b[1])
    assert np.array_equal(a[3][perm], b[3]) and a[4] == b[4]


def test_sign_of_zero_is_plus():
    P = _dense(np.zeros((2, 2)), [0, 0])
    _, _, s, _, _ = o.step(P, [0.0, -0.0], [0.0, 0.0], 1.0, 0.1, 1.0)
    assert list(s) == [1, 1]


# ------------------------------------------------------------------ schedule and runs

def test_linear_beta_schedule():
    assert o.beta_at(0, 100, 0.1, 2.0) == 0.1
    assert o.beta_at(99, 100, 0.1, 2.0) == 2.0
    assert o.beta_at(33, 67, 0.0, 1.0) == pytest.approx(0.5)
    assert o.beta_at(0, 1, 0.3, 9.0) == 0.3


def test_run_is_composition_of_draws_and_steps():
    """A run is: draw (x, v) with d = 0, then steps, with the momentum redrawn (d = t)
    at every t % refresh == 0, t > 0."""
    d = ins.dense_int(12, 4, 4, seed=20)
    P = _dense(d.k, d.kh)
    T, seed, inst, r, refresh = 7, 99, 5, 3, 3
    res = o.anneal_replica(P, T, seed, inst, r, 0.1, 0.9, 0.2, 2.0, refresh=refresh, trace=True)
    x = np.array([o.draw(seed, inst, r, j, 0)[0] for j in range(12)])
    v = np.array([o.draw(seed, inst, r, j, 0)[1] for j in range(12)])
    es = []
    for t in range(T):
        if t > 0 and t % refresh == 0:
            v = np.array([o.draw(seed, inst, r, j, t)[1] for j in range(12)])
        x, v, s, I, e = o.step(P, x, v, o.beta_at(t, T, 0.1, 0.9), 0.2, 2.0)
        es.append(e)
    assert list(res["trace"]) == es
    assert np.array_equal(res["x"], x) and np.array_equal(res["v"], v)


def test_best_state_is_consistent():
    d = ins.dense_int(30, 7, 7, seed=21)
    P = _dense(d.k, d.kh)
    for r in range(4):
        res = o.anneal_replica(P, 300, 5, 0, r, 0.01, 1.0, 0.1, 2.0, refresh=20, trace=True)
        tr = res["trace"]
        assert res["best_e"] == tr.min()
        assert res["best_step"] == int(np.argmin(tr))      # first occurrence: strict improvement
        assert o.energy_exact(P, res["best_s"]) == res["best_e"]


def test_small_sk_reaches_brute_force_ground_state():
    """N = 16 SK (J in {-1,+1}, h = 0, seed 0): the best energy found never goes below
    the exhaustive minimum, and the defaults reach it in most runs."""
    d = ins.sk_pm1(16, 0)
    P = _dense(d.k, d.kh)
    emin, cnt, _ = o.brute_force(P)
    res = o.anneal(P, 64, 1000, 1, 0, 0.05, 2.0, 0.2, 2.0)
    assert (res["best_e"] >= emin).all()
    assert np.mean(res["best_e"] == emin) > 0.8
    for r in range(64):
        assert o.energy_exact(P, res["best_s"][r]) == res["best_e"][r]


def test_stop_at_target_freezes_the_result():
    d = ins.sk_pm1(16, 0)
    P = _dense(d.k, d.kh)
    emin, _, _ = o.brute_force(P)
    full = o.anneal(P, 32, 1000, 1, 0, 0.05, 2.0, 0.2, 2.0, target=emin)
    stop = o.anneal(P, 32, 1000, 1, 0, 0.05, 2.0, 0.2, 2.0, target=emin, stop_at_target=True)
    hit = full["hit_step"] >= 0
    assert np.array_equal(full["hit_step"], stop["hit_step"])
    assert np.array_equal(stop["steps_run"][hit], stop["hit_step"][hit] + 1)
    assert (stop["best_e"][hit] <= emin).all()


def test_tts_definition():
    """Eq. 9 with the brackets read as grouping."""
    assert o.tts(2.0, 0.9) == pytest.approx(4.0)
    assert o.tts(2.0, 0.99) == 2.0 and o.tts(2.0, 1.0) == 2.0
    assert o.tts(1.0, 0.5) == pytest.approx(math.log(0.01) / math.log(0.5))
    assert o.tts(1.0, 0.0) == math.inf


# ------------------------------------------------------------------ acceptance test (Table 3, state 4)

def test_metropolis_two_spin_hand_case():
    """Hamiltonian (Eq. 4 / A6) and the Metropolis decision on the hand-worked 2-spin case
    of tests/golden/metropolis_two_spin.txt: one proposal always accepted (dH < 0), the
    reverse one accepted only below exp(-dH); fixed point scales E, not H."""
    g = read_golden("metropolis_two_spin.txt")
    k = np.array(g["k"].split(), dtype=np.int8).reshape(2, 2)
    P = _dense(k, [0, 0])
    beta = float(g["beta"])
    xA, vA, xB, vB = f64(g["xA"]), f64(g["vA"]), f64(g["xB"]), f64(g["vB"])
    sA, sB = np.sign(xA).astype(np.int8), np.sign(xB).astype(np.int8)
    assert o.energy_exact(P, sA) == int(g["EA"]) and o.energy_exact(P, sB) == int(g["EB"])
    HA = o.hamiltonian(beta, 1.0, int(g["EA"]), xA, vA)
    HB = o.hamiltonian(beta, 1.0, int(g["EB"]), xB, vB)
    assert HA == float(g["HA"]) and HB == float(g["HB"])
    # fixed point: k = 2 with q = 1/2 is the same physical instance
    P2 = o.Instance(np.zeros(2, dtype=np.int32), k=(2 * k).astype(np.int8), frac_bits=1)
    eA2 = o.energy_exact(P2, sA)
    assert eA2 == 2 * int(g["EA"]) and o.hamiltonian(beta, P2.q, eA2, xA, vA) == HA
    thr = float(g["exp_minus_dH"])
    for u in (1.0, 0.5, 0.0143, 0.0142, 2.0 ** -24):
        assert o.metropolis(HA, HB, u)                      # dH < 0: always
    assert not o.metropolis(HB, HA, 0.5)
    assert o.metropolis(HB, HA, 0.0142) and not o.metropolis(HB, HA, 0.0143)
    assert abs(math.exp(-(HA - HB)) - thr) < 1e-15
    assert o.metropolis(HA, HA, 1.0)                          # dH = 0: accepted even at u = 1


def test_accept_uniform_is_philox_word0_on_the_24_bit_grid():
    """The test's uniform: Philox4x32-10 word 0 of counter (0xFFFFFFFF, r, t, inst), mapped
    like every other uniform onto {1, ..., 2^24} / 2^24."""
    seed, inst, r, t = 0x0123456789ABCDEF, 7, 3, 50
    w = o.philox4x32_10([0xFFFFFFFF, r, t, inst], [seed & 0xFFFFFFFF, seed >> 32])[0]
    u = o.accept_uniform(seed, inst, r, t)
    assert u == ((w >> 8) + 1) / 2.0 ** 24 and 0.0 < u <= 1.0


def _metropolis_run_by_composition(P, T, seed, inst, r, b0, b1, eps, gamma, refresh):
    """The run with the acceptance test spelled out from the oracle's single steps and
    draws: a test at every momentum draw t (t % refresh == 0, t > 0) except the first, of
    the trajectory [t - refresh, t) under beta_{t-1}, with the uniform of draw t; a
    rejection puts x back to the trajectory's start."""
    n = P.n
    x = np.array([o.draw(seed, inst, r, j, 0)[0] for j in range(n)])
    v = np.array([o.draw(seed, inst, r, j, 0)[1] for j in range(n)])
    es, xs, vs, e_start, have, prop, acc = [], None, None, None, False, 0, 0
    e = None
    for t in range(T):
        if t > 0 and t % refresh == 0:
            if have:
                be = o.beta_at(t - 1, T, b0, b1)
                prop += 1
                if o.accept_uniform(seed, inst, r, t) <= math.exp(-(o.hamiltonian(be, P.q, e, x, v)
                                                                       - o.hamiltonian(be, P.q, e_start, xs, vs))):
                    acc += 1
                    e_start = e
                else:
                    x = xs.copy()
            else:
                e_start, have = e, True
            v = np.array([o.draw(seed, inst, r, j, t)[1] for j in range(n)])
            xs, vs = x.copy(), v.copy()
        x, v, s, I, e = o.step(P, x, v, o.beta_at(t, T, b0, b1), eps, gamma)
        es.append(e)
    return es, x, v, prop, acc


def test_metropolis_run_is_composition_of_steps_and_tests():
    d = ins.dense_int(10, 5, 5, seed=31)
    P = _dense(d.k, d.kh)
    T, seed, inst, refresh = 23, 17, 2, 4
    b0, b1, eps, gamma = 0.2, 1.5, 0.35, 2.0
    total_rej = 0
    for r in range(6):
        res = o.anneal_replica(P, T, seed, inst, r, b0, b1, eps, gamma, refresh=refresh, trace=True, accept_test=1)
        es, x, v, prop, acc = _metropolis_run_by_composition(P, T, seed, inst, r, b0, b1, eps, gamma, refresh)
        assert list(res["trace"]) == es
        assert np.array_equal(res["x"], x) and np.array_equal(res["v"], v)
        assert res["proposed"] == prop == 4 and res["accepted"] == acc      # tests at t = 8, 12, 16, 20
        total_rej += prop - acc
    assert total_rej > 0, "choose a case with rejections"


def test_metropolis_without_trajectories_changes_nothing():
    """With refresh = 0 the run is one trajectory and no test happens."""
    d = ins.dense_int(9, 5, 5, seed=3)
    P = _dense(d.k, d.kh)
    a = o.anneal_replica(P, 40, 1, 0, 0, 0.1, 1.0, 0.3, 2.0, refresh=0, trace=True, accept_test=1)
    b = o.anneal_replica(P, 40, 1, 0, 0, 0.1, 1.0, 0.3, 2.0, refresh=0, trace=True, accept_test=0)
    assert np.array_equal(a["trace"], b["trace"]) and a["proposed"] == 0


def test_metropolis_beta_zero_acceptance_tends_to_one():
    """beta = 0: per spin the map is symplectic Euler on a unit oscillator, which keeps
    x^2 + v^2 + eps x v, so dH = (eps / 2) sum_i (x_i v_i |start - x_i v_i |end) -> 0 with
    eps: the acceptance rate goes to 1 (App. A: exact dynamics accept everything), and
    falls below 1 when eps is large."""
    d = ins.dense_int(8, 5, 5, seed=4)
    P = _dense(d.k, d.kh)
    rates = {}
    for eps in (0.001, 0.8):
        res = o.anneal(P, 32, 201, 5, 0, 0.0, 0.0, eps, 2.0, refresh=4, accept_test=1)
        rates[eps] = res["accepted"].sum() / res["proposed"].sum()
    assert rates[0.001] >= 0.99 and rates[0.8] < rates[0.001]


# ------------------------------------------------------------------ vanilla GAHMC (exact zero crossings)

def test_gahmc_two_spin_hand_case():
    g = read_golden("gahmc_two_spin.txt")
    k = np.array(g["k"].split(), dtype=np.int8).reshape(2, 2)
    P = _dense(k, [0, 0])
    x0, v0 = f64(g["x0"]), f64(g["v0"])
    tc = f64(g["t_cross"])
    assert abs(o.gahmc_cross_time(x0[0], v0[0], 1) - tc[0]) < 1e-9
    assert abs(o.gahmc_cross_time(x0[1], v0[1], -1) - tc[1]) < 1e-9
    b = float(g["beta"])
    res = o.gahmc_replica(P, 1, 0, 0, 0, b, b, float(g["travel"]), x0=x0, v0=v0, events_cap=8)
    assert list(res["events"]) == [int(t) for t in g["events"].split()]
    assert np.allclose(res["x"], f64(g["x_end"]), atol=2e-9) and np.allclose(res["v"], f64(g["v_end"]), atol=2e-9)
    assert list(res["s"]) == [int(t) for t in g["s_end"].split()]
    assert res["best_e"] == int(g["best_e"]) and res["best_traj"] == 0
    assert res["crossings"] == 1 and res["reflections"] == 1


def test_gahmc_one_spin_threshold():
    """One spin in a field h = 1 (E = -s): leaving s = +1 costs dE = 2, so the wall is
    crossed exactly when A^2 / 2 > 2 beta (A = speed at the wall, here 1)."""
    P = o.Instance(np.array([1], dtype=np.int32), k=np.zeros((1, 1), dtype=np.int8))
    for beta, crosses in ((0.2, True), (0.24, True), (0.26, False), (1.0, False)):
        res = o.gahmc_replica(P, 1, 0, 0, 0, beta, beta, 3.0, x0=[1.0], v0=[0.0], events_cap=2)
        assert list(res["events"]) == ([0] if crosses else [-1])
        w = -math.sqrt(1.0 - 4 * beta) if crosses else 1.0          # outgoing velocity
        u = 3.0 - math.pi / 2
        assert abs(res["x"][0] - w * math.sin(u)) < 1e-12 and abs(res["v"][0] - w * math.cos(u)) < 1e-12


def test_gahmc_beta_zero_is_free_rotation():
    """beta = 0: no potential step, every wall is crossed at unchanged speed, so each
    coordinate rotates freely: x(T) = x cos T + v sin T, v(T) = -x sin T + v cos T, and
    the spins end as sgn x(T)."""
    d = ins.dense_int(12, 5, 5, seed=6)
    P = _dense(d.k, d.kh)
    g = np.random.default_rng(1)
    x0, v0 = g.standard_normal(12), g.standard_normal(12)
    T = 2.2
    res = o.gahmc_replica(P, 1, 0, 0, 0, 0.0, 0.0, T, x0=x0, v0=v0)
    assert np.allclose(res["x"], x0 * math.cos(T) + v0 * math.sin(T), atol=1e-12)
    assert np.allclose(res["v"], -x0 * math.sin(T) + v0 * math.cos(T), atol=1e-12)
    assert np.array_equal(res["s"], np.where(res["x"] >= 0, 1, -1)) and res["reflections"] == 0


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gahmc_conserves_h_within_a_trajectory(seed):
    """App. A: the exact dynamics conserve H = beta E(sgn x) + x.x/2 + v.v/2 (Eq. 4):
    across one trajectory (fixed beta, no momentum draw) H at the end equals H at the
    start, crossings and reflections included; the tracked energy equals Eq. 2."""
    d = ins.dense_int(20, 7, 7, seed=10 + seed)
    P = _dense(d.k, d.kh, f=2)
    g = np.random.default_rng(seed)
    x0, v0 = g.standard_normal(20), 2.0 * g.standard_normal(20)
    beta = 0.4
    s0 = np.where(x0 >= 0, 1, -1).astype(np.int8)
    h0 = o.hamiltonian(beta, P.q, o.energy_exact(P, s0), x0, v0)
    res = o.gahmc_replica(P, 1, 0, 0, 0, beta, beta, math.pi, x0=x0, v0=v0)
    assert res["crossings"] > 0 and res["reflections"] > 0
    e_end = o.energy_exact(P, res["s"])
    assert abs(o.hamiltonian(beta, P.q, e_end, res["x"], res["v"]) - h0) < 1e-10
    assert o.energy_exact(P, res["best_s"]) == res["best_e"] <= o.energy_exact(P, s0)


def test_gahmc_run_reaches_ground_state_and_keeps_consistent_records():
    d = ins.sk_pm1(16, 0)
    P = _dense(d.k, d.kh)
    emin, _, _ = o.brute_force(P)
    hits = 0
    for r in range(16):
        res = o.gahmc_replica(P, 200, 3, 0, r, 0.05, 1.5, math.pi / 2, target=emin)
        assert res["best_e"] >= emin and o.energy_exact(P, res["best_s"]) == res["best_e"]
        hits += res["best_e"] == emin
        assert (res["hit_traj"] >= 0) == (res["best_e"] == emin)
    assert hits >= 8
