"""Seeded synthetic Ising instances and states shaped like the paper's workloads.

This module only draws random inputs; it holds none of PHIA's arithmetic, so both
the CUDA path and the oracle may be fed from it.  Families follow the paper's
benchmark table (Table 2): sk_ising (J in {-1,+1}, h = 0) and spin_model-like
fixed-point couplings.  The paper's benchmark instance files are not used; all
inputs are generated here from a numpy PCG64 stream with an explicit seed.

Couplings are returned in fixed point: J = k * 2^-f, h = kh * 2^-f, with int8 k
(symmetric, zero diagonal) and int32 kh.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def _rng(seed):
    return np.random.Generator(np.random.PCG64(int(seed)))


@dataclass
class Dense:
    k: np.ndarray          # int8 [n][n], symmetric, zero diagonal
    kh: np.ndarray         # int32 [n]
    frac_bits: int = 0

    @property
    def n(self) -> int:
        return int(self.kh.shape[0])


@dataclass
class Csr:
    row_ptr: np.ndarray    # int32 [n+1]
    col: np.ndarray        # int32 [nnz], sorted within each row
    val: np.ndarray        # int8 [nnz]
    kh: np.ndarray         # int32 [n]
    frac_bits: int = 0

    @property
    def n(self) -> int:
        return int(self.kh.shape[0])

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    def to_dense(self) -> Dense:
        n = self.n
        k = np.zeros((n, n), dtype=np.int8)
        rows = np.repeat(np.arange(n), np.diff(self.row_ptr))
        k[rows, self.col] = self.val
        return Dense(k, self.kh.copy(), self.frac_bits)


def _symmetric_from_upper(n, upper_vals):
    k = np.zeros((n, n), dtype=np.int8)
    iu = np.triu_indices(n, 1)
    k[iu] = upper_vals
    return k + k.T


def sk_pm1(n: int, seed: int) -> Dense:
    """Fully connected SK instance: J_ij uniform in {-1,+1}, h = 0 (Table 2, sk_ising)."""
    g = _rng(seed)
    m = n * (n - 1) // 2
    up = np.where(g.random(m) < 0.5, -1, 1).astype(np.int8)
    return Dense(_symmetric_from_upper(n, up), np.zeros(n, dtype=np.int32), 0)


# ------------------------------------------------------------------ Table 2 families
#
# The paper's benchmark instances (from its reference [Hamerly 2019]) are not available;
# these generators draw instances of the same families and coefficient types (Table 2).
# Readings: Table 2 lists the problems' own weights w; a graph problem whose weights are
# non-negative with h = 0 would, taken as Ising couplings with the sign of Eq. 2, be a
# ferromagnet whose ground state is all spins aligned, so for maxcut_dense, maxcut_d3,
# sk_bool and sk_uniform the couplings are J = -w (minimising Eq. 2 then maximises the
# weighted cut).  Fractional coefficients are fixed point with 7 fractional bits
# (k = round(127 u)).

def maxcut_dense(n: int, seed: int, p: float = 0.5) -> Dense:
    """Max-cut of an unweighted G(n, p) graph (p = 1/2): J_ij = -1 on edges, h = 0."""
    g = _rng(seed)
    m = n * (n - 1) // 2
    up = np.where(g.random(m) < p, -1, 0).astype(np.int8)
    return Dense(_symmetric_from_upper(n, up), np.zeros(n, dtype=np.int32), 0)


def maxcut_d3(n: int, seed: int) -> Dense:
    """Max-cut of a random 3-regular simple graph (n even; configuration model, redrawn
    until it has no loop or repeated edge): J_ij = -1 on edges, h = 0."""
    if n % 2 or n < 4:
        raise ValueError("a 3-regular graph needs an even n >= 4")
    g = _rng(seed)
    for _ in range(10000):
        stubs = g.permutation(np.repeat(np.arange(n), 3))
        a, b = stubs[0::2], stubs[1::2]
        if np.any(a == b):
            continue
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        if np.unique(lo * n + hi).size != lo.size:
            continue
        k = np.zeros((n, n), dtype=np.int8)
        k[lo, hi] = -1
        k[hi, lo] = -1
        return Dense(k, np.zeros(n, dtype=np.int32), 0)
    raise RuntimeError("no simple 3-regular graph drawn")


def sk_bool(n: int, seed: int) -> Dense:
    """SK model with weights w_ij uniform in {0, 1}: J_ij = -w_ij, h = 0."""
    g = _rng(seed)
    m = n * (n - 1) // 2
    up = -(g.random(m) < 0.5).astype(np.int8)
    return Dense(_symmetric_from_upper(n, up), np.zeros(n, dtype=np.int32), 0)


def sk_uniform(n: int, seed: int) -> Dense:
    """SK model with weights 0 or U(0, 1) (each with probability 1/2), fixed point
    k = round(127 u) with 7 fractional bits: J_ij = -k_ij 2^-7, h = 0."""
    g = _rng(seed)
    m = n * (n - 1) // 2
    on = g.random(m) < 0.5
    u = g.random(m)
    up = -np.where(on, np.rint(127.0 * u), 0.0).astype(np.int8)
    return Dense(_symmetric_from_upper(n, up), np.zeros(n, dtype=np.int32), 7)


def spin_model(n: int, seed: int) -> Dense:
    """Ising model with J_ij and h_i uniform in (-1, 1), fixed point k = round(127 u)
    with 7 fractional bits."""
    g = _rng(seed)
    m = n * (n - 1) // 2
    up = np.rint(127.0 * g.uniform(-1.0, 1.0, size=m)).astype(np.int8)
    kh = np.rint(127.0 * g.uniform(-1.0, 1.0, size=n)).astype(np.int32)
    return Dense(_symmetric_from_upper(n, up), kh, 7)


@dataclass
class Planted(Dense):
    """An instance with a known optimum energy (units of q)."""
    optimum_k: int = 0


def nae_3_sat(n: int, seed: int, alpha: float = 2.1) -> Planted:
    """Planted not-all-equal 3-SAT with m = round(alpha n) clauses as an Ising model.  A
    clause on variables (a, b, c) with literal signs (sa, sb, sc) is satisfied when the
    three y = s sigma are not all equal; y_a y_b + y_a y_c + y_b y_c is then -1, else 3.
    Summed over clauses this is Eq. 2 with J_ab = -sum over clauses of sa sb (integer
    couplings), h = 0, and every energy is >= -m.  Each clause draws its variables and
    signs so that a hidden random assignment satisfies it, so the optimum is exactly -m."""
    g = _rng(seed)
    z = np.where(g.random(n) < 0.5, -1, 1)
    m = int(round(alpha * n))
    rows, cols, vals = [], [], []
    for _ in range(m):
        v = g.choice(n, size=3, replace=False)
        while True:
            sg = np.where(g.random(3) < 0.5, -1, 1)
            y = sg * z[v]
            if not (y[0] == y[1] == y[2]):
                break
        for a, b in ((0, 1), (0, 2), (1, 2)):
            rows.append(v[a]); cols.append(v[b]); vals.append(-int(sg[a] * sg[b]))
    k = np.zeros((n, n), dtype=np.int32)
    np.add.at(k, (np.array(rows), np.array(cols)), np.array(vals))
    k = k + k.T
    if np.abs(k).max() > 127:
        raise ValueError("coupling outside int8")
    return Planted(k.astype(np.int8), np.zeros(n, dtype=np.int32), 0, -m)


FAMILIES = {"maxcut_dense": maxcut_dense, "maxcut_d3": maxcut_d3, "sk_bool": sk_bool, "sk_ising": None,
            "sk_uniform": sk_uniform, "nae_3_sat": nae_3_sat, "spin_model": spin_model}


def tts_seed(family: str, n: int, k: int, base_seed: int = 9) -> int:
    """Seed of instance k of a family at size n in the time-to-solution study."""
    return base_seed * 100_003 + sorted(FAMILIES).index(family) * 10_000_019 + n * 1000 + k


def family_instance(name: str, n: int, seed: int) -> Dense:
    """An instance of one of the Table 2 families."""
    if name == "sk_ising":
        return sk_pm1(n, seed)
    return FAMILIES[name](n, seed)


def dense_int(n: int, kmax: int, hmax: int, seed: int, frac_bits: int = 0) -> Dense:
    """Dense integer couplings: k_ij uniform in [-kmax, kmax], kh_i uniform in [-hmax, hmax]."""
    g = _rng(seed)
    m = n * (n - 1) // 2
    up = g.integers(-kmax, kmax + 1, size=m).astype(np.int8)
    kh = g.integers(-hmax, hmax + 1, size=n).astype(np.int32)
    return Dense(_symmetric_from_upper(n, up), kh, frac_bits)


def erdos_renyi(n: int, density: float, kmax: int, hmax: int, frac_bits: int, seed: int) -> Csr:
    """Erdos-Renyi graph G(n, p): each pair i<j is an edge with probability p, drawn as a
    Binomial number of distinct pair indices; an edge carries k uniform in [-kmax, kmax]
    (a drawn k = 0 is kept as a stored zero)."""
    g = _rng(seed)
    M = n * (n - 1) // 2
    m = int(g.binomial(M, density)) if M > 0 else 0
    lin = np.sort(g.choice(M, size=m, replace=False)) if m > 0 else np.zeros(0, dtype=np.int64)
    # linear index l -> (i, j), pairs in row-major upper-triangle order; row i starts at
    # off(i) = i (2n - i - 1) / 2
    lin = lin.astype(np.int64)
    i = np.floor(((2 * n - 1) - np.sqrt((2.0 * n - 1) ** 2 - 8.0 * lin)) / 2).astype(np.int64)
    off = lambda r: r * (2 * n - r - 1) // 2
    i = np.where(off(i + 1) <= lin, i + 1, i)
    i = np.where(off(i) > lin, i - 1, i)
    j = lin - off(i) + i + 1
    iu, ju = i, j
    w = g.integers(-kmax, kmax + 1, size=iu.shape[0]).astype(np.int8)
    kh = g.integers(-hmax, hmax + 1, size=n).astype(np.int32)
    rows = np.concatenate([iu, ju])
    cols = np.concatenate([ju, iu])
    vals = np.concatenate([w, w])
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr).astype(np.int32)
    return Csr(row_ptr, cols.astype(np.int32), vals, kh, frac_bits)


def batched_er(count: int, seed: int, n_lo: int = 100, n_hi: int = 3000,
               d_lo: float = 0.006, d_hi: float = 0.06) -> list[Csr]:
    """Ragged batch: N uniform in [n_lo, n_hi], density uniform in [d_lo, d_hi],
    J = k/16 with k uniform in [-127, 127], h = k/16 with k uniform in [-31, 31]."""
    g = _rng(seed)
    out = []
    for b in range(count):
        n = int(g.integers(n_lo, n_hi + 1))
        d = float(g.uniform(d_lo, d_hi))
        out.append(erdos_renyi(n, d, 127, 31, 4, seed * 1_000_003 + b + 1))
    return out


@dataclass
class Request:
    arrival_s: float
    instance: object       # Dense or Csr
    kind: str              # "dense" or "sparse"


def serving_stream(count: int, seed: int, rate_hz: float = 200.0, n_lo: int = 64,
                   n_hi: int = 8192) -> list[Request]:
    """Poisson arrivals at rate_hz; N log-uniform in [n_lo, n_hi]; alternately dense
    {-1,+1} couplings and sparse fixed-point couplings (8 fractional bits, density 0.01,
    k and kh uniform in [-127, 127])."""
    g = _rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += float(g.exponential(1.0 / rate_hz))
        n = int(round(math.exp(g.uniform(math.log(n_lo), math.log(n_hi)))))
        if i % 2 == 0:
            inst = sk_pm1(n, seed * 7919 + i + 1)
            out.append(Request(t, inst, "dense"))
        else:
            inst = erdos_renyi(n, 0.01, 127, 127, 8, seed * 7919 + i + 1)
            out.append(Request(t, inst, "sparse"))
    return out


def serving_pool(count: int, seed: int, n_lo: int = 64, n_hi: int = 8192) -> list:
    """Pool of serving instances: N log-uniform in [n_lo, n_hi]; even entries dense
    {-1,+1} with h = 0, odd entries sparse fixed point (8 fractional bits, density 0.01,
    k and kh uniform in [-127, 127])."""
    g = _rng(seed)
    out = []
    for i in range(count):
        n = int(round(math.exp(g.uniform(math.log(n_lo), math.log(n_hi)))))
        if i % 2 == 0:
            out.append(sk_pm1(n, seed * 7919 + i + 1))
        else:
            out.append(erdos_renyi(n, 0.01, 127, 127, 8, seed * 7919 + i + 1))
    return out


def serving_arrivals(count: int, seed: int, pool_size: int, rate_hz: float = 200.0):
    """Poisson arrival times (s) at rate_hz, each with a pool index and a run seed."""
    g = _rng(seed)
    t = np.cumsum(g.exponential(1.0 / rate_hz, size=count))
    idx = g.integers(0, pool_size, size=count)
    seeds = g.integers(1, 2**62, size=count)
    return [(float(t[i]), int(idx[i]), int(seeds[i])) for i in range(count)]


def random_spins(R: int, n: int, seed: int) -> np.ndarray:
    """Uniform +-1 states, int8 [R][n]."""
    g = _rng(seed)
    return np.where(g.random((R, n)) < 0.5, -1, 1).astype(np.int8)


def random_state(R: int, n: int, seed: int, min_abs: float = 0.0):
    """Continuous HMC state (x, v), float32 [R][n], standard normal.  With min_abs > 0,
    positions closer to 0 than min_abs are pushed out to +-min_abs (so the sign of x is
    not decided by rounding)."""
    g = _rng(seed)
    x = g.standard_normal((R, n)).astype(np.float32)
    v = g.standard_normal((R, n)).astype(np.float32)
    if min_abs > 0:
        small = np.abs(x) < min_abs
        x[small] = np.where(x[small] >= 0, min_abs, -min_abs).astype(np.float32)
    return x, v
