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
