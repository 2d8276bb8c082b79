"""FP64 CPU oracle for PHIA (arXiv 2407.10205) -- test infrastructure only.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports it and shares no code with it.

The arithmetic lives in ``phia_oracle.c`` (plain C, FP64, int64 energies);
this module compiles it with gcc, loads it with ctypes and exposes numpy-level
wrappers.  Passages followed (see the C file for the per-function mapping):
Eq. 2 (energy), Eq. 6 (field), Eqs. 4, 5, 7, 8 (Hamiltonian and its tanh
gradient), Eqs. A7-A8 (the position-then-momentum update), Table 3 state 4
(the optional Metropolis test on H at trajectory ends) and state 5 (best-state
keeping), Sec. 2.1 / 3.2 (vanilla GAHMC: the exact dynamics by zero crossings)
and Eq. 9 (time to solution).

Parity status: every function here is pinned by the ``-m "not gpu"`` tests
(published Philox known-answer vectors, brute force, closed forms, hand-worked
3-spin step, 2-spin Metropolis and 2-spin GAHMC cases, the beta = 0 discrete
invariant and free rotation, exact H conservation of GAHMC).  The default
hyper-parameters (eps, gamma, beta schedule, GAHMC travel time) have no value in
the paper and are therefore unpinned as *values*; the updates they feed are
pinned.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "phia_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-o", tmp, _SRC,
           "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Inst(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32),
                ("k", ctypes.c_void_p),
                ("row_ptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p),
                ("val", ctypes.c_void_p),
                ("kh", ctypes.c_void_p)]


class _Sched(ctypes.Structure):
    _fields_ = [("beta0", ctypes.c_double), ("beta1", ctypes.c_double),
                ("eps", ctypes.c_double), ("gamma", ctypes.c_double),
                ("refresh", ctypes.c_int64),
                ("has_target", ctypes.c_int32), ("stop_at_target", ctypes.c_int32),
                ("target", ctypes.c_int64), ("deriv", ctypes.c_int32), ("accept_test", ctypes.c_int32)]


class _GahmcSched(ctypes.Structure):
    _fields_ = [("beta0", ctypes.c_double), ("beta1", ctypes.c_double), ("travel", ctypes.c_double),
                ("trajectories", ctypes.c_int64), ("has_target", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("target", ctypes.c_int64)]


class _GahmcOut(ctypes.Structure):
    _fields_ = [("best_e", ctypes.c_int64), ("best_traj", ctypes.c_int64), ("crossings", ctypes.c_int64),
                ("reflections", ctypes.c_int64), ("hit_traj", ctypes.c_int64)]


class _RepOut(ctypes.Structure):
    _fields_ = [("best_e", ctypes.c_int64), ("best_step", ctypes.c_int64),
                ("hit_step", ctypes.c_int64), ("steps_run", ctypes.c_int64),
                ("proposed", ctypes.c_int64), ("accepted", ctypes.c_int64)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            lib.orc_philox4x32_10.argtypes = [P(ctypes.c_uint32), P(ctypes.c_uint32), P(ctypes.c_uint32)]
            lib.orc_box_muller.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
            lib.orc_box_muller.restype = ctypes.c_double
            lib.orc_u01_open.argtypes = [ctypes.c_uint32]
            lib.orc_u01_open.restype = ctypes.c_double
            lib.orc_u01_half.argtypes = [ctypes.c_uint32]
            lib.orc_u01_half.restype = ctypes.c_double
            lib.orc_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                     ctypes.c_uint32, P(ctypes.c_double), P(ctypes.c_double)]
            lib.orc_energy_exact.argtypes = [P(_Inst), ctypes.c_void_p]
            lib.orc_energy_exact.restype = ctypes.c_int64
            lib.orc_field.argtypes = [P(_Inst), ctypes.c_void_p, ctypes.c_void_p]
            lib.orc_energy_from_field.argtypes = [P(_Inst), ctypes.c_void_p, ctypes.c_void_p]
            lib.orc_energy_from_field.restype = ctypes.c_int64
            lib.orc_brute_force.argtypes = [P(_Inst), P(ctypes.c_int64), ctypes.c_void_p]
            lib.orc_brute_force.restype = ctypes.c_int64
            lib.orc_step.argtypes = [P(_Inst), ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p]
            lib.orc_step.restype = ctypes.c_int64
            lib.orc_step_mode.argtypes = [P(_Inst), ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p]
            lib.orc_step_mode.restype = ctypes.c_int64
            lib.orc_dfactor.argtypes = [ctypes.c_double, ctypes.c_int32]
            lib.orc_dfactor.restype = ctypes.c_double
            lib.orc_hamiltonian.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int64, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_int]
            lib.orc_hamiltonian.restype = ctypes.c_double
            lib.orc_metropolis.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
            lib.orc_metropolis.restype = ctypes.c_int
            lib.orc_accept_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32]
            lib.orc_accept_uniform.restype = ctypes.c_double
            lib.orc_gahmc_cross_time.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int8]
            lib.orc_gahmc_cross_time.restype = ctypes.c_double
            lib.orc_gahmc_replica.argtypes = [P(_Inst), ctypes.c_int32, P(_GahmcSched), ctypes.c_uint64,
                                              ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p,
                                              P(_GahmcOut), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]
            lib.orc_beta_at.argtypes = [P(_Sched), ctypes.c_int64, ctypes.c_int64]
            lib.orc_beta_at.restype = ctypes.c_double
            lib.orc_anneal_replica.argtypes = [P(_Inst), ctypes.c_int32, P(_Sched), ctypes.c_int64,
                                               ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                               ctypes.c_void_p, ctypes.c_void_p, P(_RepOut),
                                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_void_p]
            lib.orc_anneal_replicas.argtypes = [P(_Inst), ctypes.c_int32, P(_Sched), ctypes.c_int64,
                                                ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32,
                                                ctypes.c_int32, ctypes.c_int32, P(_RepOut),
                                                ctypes.c_void_p]
            _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


class Instance:
    """An Ising instance in fixed point: J = k * 2^-f, h = kh * 2^-f.

    Dense (``k`` an int8 n x n symmetric matrix with zero diagonal) or CSR
    (``row_ptr``, ``col``, ``val``).  Holds numpy arrays alive for ctypes.
    """

    def __init__(self, kh, k=None, row_ptr=None, col=None, val=None, frac_bits=0):
        self.kh = np.ascontiguousarray(kh, dtype=np.int32)
        self.n = int(self.kh.shape[0])
        self.frac_bits = int(frac_bits)
        self.k = None if k is None else np.ascontiguousarray(k, dtype=np.int8)
        self.row_ptr = None if row_ptr is None else np.ascontiguousarray(row_ptr, dtype=np.int32)
        self.col = None if col is None else np.ascontiguousarray(col, dtype=np.int32)
        self.val = None if val is None else np.ascontiguousarray(val, dtype=np.int8)
        if self.k is None and self.row_ptr is None:
            raise ValueError("need a dense k or a CSR triple")
        self._c = _Inst(self.n, _ptr(self.k), _ptr(self.row_ptr), _ptr(self.col), _ptr(self.val),
                        _ptr(self.kh))

    @property
    def q(self) -> float:
        return math.ldexp(1.0, -self.frac_bits)


def _sched(beta0, beta1, eps, gamma, refresh=0, target=None, stop_at_target=False, deriv=0, accept_test=0):
    return _Sched(float(beta0), float(beta1), float(eps), float(gamma), int(refresh),
                  0 if target is None else 1, 1 if stop_at_target else 0,
                  0 if target is None else int(target), int(deriv), int(accept_test))


# ----------------------------------------------------------------- wrappers

def philox4x32_10(ctr, key):
    """Philox4x32-10 block (Salmon et al., SC'11): 4 counter words, 2 key words -> 4 words."""
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib.orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def box_muller(a: int, b: int) -> float:
    return _load().orc_box_muller(a & 0xFFFFFFFF, b & 0xFFFFFFFF)


def u01_open(a: int) -> float:
    return _load().orc_u01_open(a & 0xFFFFFFFF)


def u01_half(a: int) -> float:
    return _load().orc_u01_half(a & 0xFFFFFFFF)


def draw(seed: int, inst: int, r: int, j: int, d: int):
    """(position normal, momentum normal) for spin j of replica r, draw index d."""
    nx, nv = ctypes.c_double(), ctypes.c_double()
    _load().orc_draw(seed & (2**64 - 1), inst, r, j, d, ctypes.byref(nx), ctypes.byref(nv))
    return nx.value, nv.value


def draw_grid(seed, inst, R, n, d):
    """Normals for all (replica, spin): arrays [R][n] of positions and momenta."""
    X = np.empty((R, n)); V = np.empty((R, n))
    for r in range(R):
        for j in range(n):
            X[r, j], V[r, j] = draw(seed, inst, r, j, d)
    return X, V


def energy_exact(P: Instance, s) -> int:
    s = np.ascontiguousarray(s, dtype=np.int8)
    return int(_load().orc_energy_exact(ctypes.byref(P._c), _ptr(s)))


def field(P: Instance, s) -> np.ndarray:
    s = np.ascontiguousarray(s, dtype=np.int8)
    I = np.empty(P.n, dtype=np.int64)
    _load().orc_field(ctypes.byref(P._c), _ptr(s), _ptr(I))
    return I


def energy_from_field(P: Instance, s, I) -> int:
    s = np.ascontiguousarray(s, dtype=np.int8)
    I = np.ascontiguousarray(I, dtype=np.int64)
    return int(_load().orc_energy_from_field(ctypes.byref(P._c), _ptr(s), _ptr(I)))


def field_batch(P: Instance, S) -> tuple[np.ndarray, np.ndarray]:
    """Field (Eq. 6) and energy (Eq. 2) for each row of S ([R][n] of +-1)."""
    S = np.ascontiguousarray(S, dtype=np.int8)
    I = np.empty(S.shape, dtype=np.int64)
    E = np.empty(S.shape[0], dtype=np.int64)
    for r in range(S.shape[0]):
        I[r] = field(P, S[r])
        E[r] = energy_from_field(P, S[r], I[r])
    return I, E


def brute_force(P: Instance):
    """(minimum energy, number of minimisers, lowest-index minimiser) over all 2^n states."""
    if P.n > 24:
        raise ValueError("brute force is limited to n <= 24")
    cnt = ctypes.c_int64()
    arg = np.empty(P.n, dtype=np.int8)
    e = _load().orc_brute_force(ctypes.byref(P._c), ctypes.byref(cnt), _ptr(arg))
    return int(e), int(cnt.value), arg


def step(P: Instance, x, v, beta, eps, gamma, deriv=0):
    """One Eq. A7 iteration in FP64 (deriv: 0 exact derivative factor of Eq. 8, 1 the
    quadratic stand-in of `dfactor`).  Returns (x', v', s, I, E)."""
    x = np.array(x, dtype=np.float64, copy=True)
    v = np.array(v, dtype=np.float64, copy=True)
    s = np.empty(P.n, dtype=np.int8)
    I = np.empty(P.n, dtype=np.int64)
    e = _load().orc_step_mode(ctypes.byref(P._c), P.q, float(beta), float(eps), float(gamma), int(deriv),
                              _ptr(x), _ptr(v), _ptr(s), _ptr(I))
    return x, v, s, I, int(e)


def hamiltonian(beta, q, e, x, v):
    """Eq. 4 / Eq. A6: beta q e + x.x/2 + v.v/2 (e = E(sgn x) in units of q)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    return float(_load().orc_hamiltonian(float(beta), float(q), int(e), _ptr(x), _ptr(v), int(x.shape[0])))


def metropolis(h_start, h_end, u) -> bool:
    """Table 3 state 4 as a Metropolis test: accept when u <= exp(-(h_end - h_start))."""
    return bool(_load().orc_metropolis(float(h_start), float(h_end), float(u)))


def accept_uniform(seed, inst, r, t) -> float:
    """The test's uniform before the momentum draw d = t: Philox (0xFFFFFFFF, r, t, inst)
    word 0 on the 24-bit grid of (0, 1]."""
    return float(_load().orc_accept_uniform(seed & (2**64 - 1), inst, r, t))


def dfactor(y, deriv=0):
    """The derivative factor of Eq. 8 at y = gamma x: 1 - tanh^2(y), or (deriv = 1) the
    quadratic stand-in max(0, 1 - (y / 1.5)^2) (coefficients chosen here: the paper
    prints none)."""
    return float(_load().orc_dfactor(float(y), int(deriv)))


def beta_at(t, T, beta0, beta1):
    return _load().orc_beta_at(ctypes.byref(_sched(beta0, beta1, 0.0, 0.0)), int(t), int(T))


def anneal_replica(P: Instance, T, seed, inst_id, r, beta0, beta1, eps, gamma, refresh=0,
                   target=None, stop_at_target=False, x0=None, v0=None, trace=False, deriv=0, accept_test=0):
    """One replica of a PHIA run in FP64.  Returns a dict with best_e, best_step,
    hit_step, steps_run, proposed, accepted (trajectories put to / passing the acceptance
    test of accept_test = 1), best_s, x, v and (optionally) the per-iteration energies."""
    S = _sched(beta0, beta1, eps, gamma, refresh, target, stop_at_target, deriv, accept_test)
    out = _RepOut()
    best_s = np.zeros(P.n, dtype=np.int8)
    xo = np.empty(P.n); vo = np.empty(P.n)
    tr = np.empty(T, dtype=np.int64) if trace else None
    x0a = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float64)
    v0a = None if v0 is None else np.ascontiguousarray(v0, dtype=np.float64)
    _load().orc_anneal_replica(ctypes.byref(P._c), P.frac_bits, ctypes.byref(S), int(T),
                               seed & (2**64 - 1), inst_id, r, _ptr(x0a), _ptr(v0a),
                               ctypes.byref(out), _ptr(best_s), _ptr(xo), _ptr(vo), _ptr(tr))
    res = dict(best_e=out.best_e, best_step=out.best_step, hit_step=out.hit_step,
               steps_run=out.steps_run, proposed=out.proposed, accepted=out.accepted, best_s=best_s, x=xo, v=vo)
    if trace:
        res["trace"] = tr
    return res


def anneal(P: Instance, R, T, seed, inst_id, beta0, beta1, eps, gamma, refresh=0,
           target=None, stop_at_target=False, threads=None, r0=0, want_spins=True, deriv=0, accept_test=0):
    """R replicas (indices r0..r0+R-1) on `threads` host threads.
    Returns arrays best_e[R], best_step[R], hit_step[R], steps_run[R], proposed[R],
    accepted[R], best_s[R][n]."""
    S = _sched(beta0, beta1, eps, gamma, refresh, target, stop_at_target, deriv, accept_test)
    outs = (_RepOut * R)()
    best_s = np.zeros((R, P.n), dtype=np.int8) if want_spins else None
    th = threads or os.cpu_count() or 1
    _load().orc_anneal_replicas(ctypes.byref(P._c), P.frac_bits, ctypes.byref(S), int(T),
                                seed & (2**64 - 1), inst_id, int(r0), int(R), int(th), outs,
                                _ptr(best_s))
    return dict(best_e=np.array([o.best_e for o in outs], dtype=np.int64),
                best_step=np.array([o.best_step for o in outs], dtype=np.int64),
                hit_step=np.array([o.hit_step for o in outs], dtype=np.int64),
                steps_run=np.array([o.steps_run for o in outs], dtype=np.int64),
                proposed=np.array([o.proposed for o in outs], dtype=np.int64),
                accepted=np.array([o.accepted for o in outs], dtype=np.int64),
                best_s=best_s)


def gahmc_cross_time(x0, v0, s) -> float:
    """Time in [0, pi] at which x0 cos t + v0 sin t leaves the orthant of sign s."""
    return float(_load().orc_gahmc_cross_time(float(x0), float(v0), int(s)))


def gahmc_replica(P: Instance, K, seed, inst_id, r, beta0, beta1, travel, target=None, x0=None, v0=None,
                  events_cap=0):
    """One replica of vanilla GAHMC (exact zero crossings, Sec. 2.1 / 3.2) in FP64: K
    trajectories of time `travel`.  Returns best_e, best_traj, crossings, reflections,
    hit_traj, best_s, x, v, s and (events_cap > 0) the first events: j for a crossing of
    spin j, -(j + 1) for a reflection."""
    S = _GahmcSched(float(beta0), float(beta1), float(travel), int(K), 0 if target is None else 1, 0,
                    0 if target is None else int(target))
    out = _GahmcOut()
    n = P.n
    best_s = np.zeros(n, dtype=np.int8)
    s = np.zeros(n, dtype=np.int8)
    xo, vo = np.empty(n), np.empty(n)
    ev = np.full(max(events_cap, 1), np.iinfo(np.int32).min, dtype=np.int32)
    x0a = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float64)
    v0a = None if v0 is None else np.ascontiguousarray(v0, dtype=np.float64)
    _load().orc_gahmc_replica(ctypes.byref(P._c), P.frac_bits, ctypes.byref(S), seed & (2**64 - 1), inst_id, r,
                              _ptr(x0a), _ptr(v0a), ctypes.byref(out), _ptr(best_s), _ptr(xo), _ptr(vo), _ptr(s),
                              _ptr(ev) if events_cap > 0 else None, int(events_cap))
    nev = out.crossings + out.reflections
    return dict(best_e=out.best_e, best_traj=out.best_traj, crossings=out.crossings, reflections=out.reflections,
                hit_traj=out.hit_traj, best_s=best_s, x=xo, v=vo, s=s,
                events=ev[:min(events_cap, nev)] if events_cap > 0 else None)


def tts(t1: float, p: float, target_conf: float = 0.99) -> float:
    """Eq. 9: TTS = T1 * lg(1 - 0.99) / lg(1 - P).  The brackets are read as plain
    grouping; P >= 0.99 gives T1 (one run suffices); P = 0 gives infinity."""
    if p <= 0.0:
        return math.inf
    if p >= target_conf:
        return t1
    return t1 * math.log10(1.0 - target_conf) / math.log10(1.0 - p)
