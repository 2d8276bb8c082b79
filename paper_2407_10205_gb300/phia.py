"""Thin Python binding of the PHIA C ABI (include/phia.h).

Argument marshalling only: every step of the hot path runs in the CUDA library
``_build/libphia.so``.  Functions keep the C names without the ``phia_`` prefix
where it would be redundant in Python (``phia.create`` is ``phia_create``).
Device buffers are torch CUDA tensors (PyTorch provides memory and streams);
host buffers are numpy arrays.  Errors raise ``PhiaError`` carrying the C code and
``phia_last_error()``.  There is no fallback: if the library is missing the calls
raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libphia.so")

OK, EINVAL, ERANGE, ENOMEM, ETIMEOUT, ECUDA, ESTATE, ENOTSUP = 0, -1, -2, -3, -4, -5, -6, -7
PATH_AUTO, PATH_TC, PATH_FP32, PATH_CSR = 0, 1, 2, 3
OP_AUTO, OP_E4M3, OP_BF16 = 0, 1, 2
PEAK_S8_MMA_SYNC = 3   # phia_mma_peak only: warp-level int8 mma.sync
_CODES = {EINVAL: "EINVAL", ERANGE: "ERANGE", ENOMEM: "ENOMEM", ETIMEOUT: "ETIMEOUT",
          ECUDA: "ECUDA", ESTATE: "ESTATE", ENOTSUP: "ENOTSUP"}


class PhiaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"PHIA_{_CODES.get(code, code)}: {msg}")
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int32), ("operand", ctypes.c_int32), ("device", ctypes.c_int32),
                ("instance_id", ctypes.c_uint32), ("stream", ctypes.c_void_p),
                ("tile_replicas", ctypes.c_int32), ("coupling_mem", ctypes.c_int32),
                ("tc_kernel", ctypes.c_int32), ("large_variant", ctypes.c_int32)]


class Schedule(ctypes.Structure):
    _fields_ = [("beta0", ctypes.c_float), ("beta1", ctypes.c_float), ("eps", ctypes.c_float),
                ("gamma", ctypes.c_float), ("refresh", ctypes.c_int32), ("has_target", ctypes.c_int32),
                ("stop_at_target", ctypes.c_int32), ("deriv", ctypes.c_int32),
                ("target_k", ctypes.c_int64), ("accept_test", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("replicas", ctypes.c_int64), ("steps", ctypes.c_int64), ("spin_updates", ctypes.c_int64),
                ("best_energy_k", ctypes.c_int64), ("best_replica", ctypes.c_int64),
                ("best_step", ctypes.c_int64), ("hit_step", ctypes.c_int64), ("hit_replica", ctypes.c_int64),
                ("device_ms", ctypes.c_float), ("path", ctypes.c_int32), ("operand", ctypes.c_int32),
                ("kernel_launches", ctypes.c_int32), ("tc_kernel", ctypes.c_int32),
                ("reserved0", ctypes.c_int32), ("hit_ns", ctypes.c_int64)]


class InstanceDesc(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("frac_bits", ctypes.c_int32), ("J_k", ctypes.c_void_p),
                ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("val_k", ctypes.c_void_p),
                ("h_k", ctypes.c_void_p), ("instance_id", ctypes.c_uint32), ("has_target", ctypes.c_int32),
                ("target_k", ctypes.c_int64)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("max_inflight", ctypes.c_int32), ("hbm_budget_bytes", ctypes.c_int64),
                ("chunk_iters", ctypes.c_int32), ("path", ctypes.c_int32)]


class RequestStatus(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("hit", ctypes.c_int32), ("energy_k", ctypes.c_int64),
                ("hit_step", ctypes.c_int64), ("steps_run", ctypes.c_int64), ("t_submit_s", ctypes.c_double),
                ("t_admit_s", ctypes.c_double), ("t_done_s", ctypes.c_double), ("path", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("hits", ctypes.c_int64), ("spin_updates", ctypes.c_int64),
                ("ttt_p50_s", ctypes.c_double), ("ttt_p99_s", ctypes.c_double), ("ttt_admit_p50_s", ctypes.c_double),
                ("ttt_admit_p99_s", ctypes.c_double), ("elapsed_s", ctypes.c_double), ("used_bytes", ctypes.c_int64)]


class GahmcSchedule(ctypes.Structure):
    _fields_ = [("beta0", ctypes.c_float), ("beta1", ctypes.c_float), ("travel", ctypes.c_float),
                ("has_target", ctypes.c_int32), ("target_k", ctypes.c_int64)]


def gahmc_schedule(beta0, beta1, travel=1.5707963267948966, target=None) -> GahmcSchedule:
    return GahmcSchedule(float(beta0), float(beta1), float(travel), 0 if target is None else 1,
                         0 if target is None else int(target))


class TuneResult(ctypes.Structure):
    _fields_ = [("tc_kernel", ctypes.c_int32), ("tile_replicas", ctypes.c_int32), ("coupling_mem", ctypes.c_int32),
                ("candidates", ctypes.c_int32), ("best_us_per_iter", ctypes.c_float),
                ("worst_us_per_iter", ctypes.c_float), ("large_variant", ctypes.c_int32), ("reserved", ctypes.c_int32)]


# name -> (restype, argtypes); every symbol include/phia.h declares
_P = ctypes.c_void_p
SIGNATURES = {
    "phia_create": (ctypes.c_int, [ctypes.POINTER(_P), _P, _P, ctypes.c_int32, ctypes.c_int32, _P]),
    "phia_create_from_device": (ctypes.c_int, [ctypes.POINTER(_P), _P, _P, ctypes.c_int32, ctypes.c_int32, _P]),
    "phia_create_csr": (ctypes.c_int, [ctypes.POINTER(_P), _P, _P, _P, _P, ctypes.c_int32, ctypes.c_int32, _P]),
    "phia_anneal": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64]),
    "phia_best": (ctypes.c_int, [_P, _P, _P]),
    "phia_autotune": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_int32, _P]),
    "phia_stats_get": (ctypes.c_int, [_P, _P]),
    "phia_replica_results": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _P, _P]),
    "phia_acceptance": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P]),
    "phia_gahmc": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, _P, _P, _P, _P,
                                  ctypes.c_int32]),
    "phia_run": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                ctypes.c_uint64, _P, _P, ctypes.c_int32]),
    "phia_init_state": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_uint64, _P, _P]),
    "phia_field": (ctypes.c_int, [_P, _P, ctypes.c_int32, _P, _P]),
    "phia_philox_draws": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int32,
                                         ctypes.c_int32, _P, _P, _P, _P]),
    "phia_run_noalloc": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_int32,
                                        ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64,
                                        ctypes.c_uint32, _P, _P, _P, _P, _P, _P, ctypes.c_int32, _P]),
    "phia_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int32, _P, _P]),
    "phia_batch_anneal": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64]),
    "phia_batch_best": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P]),
    "phia_batch_replica_results": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, _P, _P, _P, _P]),
    "phia_batch_stats_get": (ctypes.c_int, [_P, _P]),
    "phia_batch_autotune": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_int32, _P]),
    "phia_batch_sync": (ctypes.c_int, [_P]),
    "phia_batch_destroy": (None, [_P]),
    "phia_server_create": (ctypes.c_int, [ctypes.POINTER(_P), _P]),
    "phia_server_submit": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, _P]),
    "phia_server_poll": (ctypes.c_int, [_P, ctypes.c_int64, _P, _P]),
    "phia_server_wait_all": (ctypes.c_int, [_P, ctypes.c_int64]),
    "phia_server_stats_get": (ctypes.c_int, [_P, _P]),
    "phia_server_destroy": (None, [_P]),
    "phia_debug_wait": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int32]),
    "phia_mma_peak": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, _P, _P, _P]),
    "phia_sync": (ctypes.c_int, [_P]),
    "phia_destroy": (None, [_P]),
    "phia_last_error": (ctypes.c_char_p, []),
}

_lib = None


def load(path: str | None = None):
    """Load libphia.so (built by ``paper_2407_10205_gb300.build``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"PHIA CUDA library not built ({p}); run paper_2407_10205_gb300.build.build()")
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def last_error() -> str:
    return load().phia_last_error().decode()


def _check(rc):
    if rc != OK:
        raise PhiaError(rc, last_error())


def _np_ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _dev_ptr(t):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("device buffers must be contiguous CUDA tensors")
    return ctypes.c_void_p(t.data_ptr())


DERIV_EXACT, DERIV_QUADRATIC = 0, 1


ACCEPT_ALL, ACCEPT_METROPOLIS = 0, 1


def schedule(beta0, beta1, eps, gamma, refresh=0, target=None, stop_at_target=False,
             deriv=DERIV_EXACT, accept_test=ACCEPT_ALL) -> Schedule:
    return Schedule(float(beta0), float(beta1), float(eps), float(gamma), int(refresh),
                    0 if target is None else 1, 1 if stop_at_target else 0, int(deriv),
                    0 if target is None else int(target), int(accept_test), 0)


MEM_AUTO, MEM_SHARED, MEM_TENSOR = 0, 1, 2
KERNEL_AUTO, KERNEL_RESIDENT, KERNEL_PER_STEP, KERNEL_IMMA, KERNEL_INCREMENTAL = 0, 1, 2, 3, 4


def opts(path=PATH_AUTO, operand=OP_AUTO, device=0, instance_id=0, stream=None, tile_replicas=0,
         coupling_mem=MEM_AUTO, tc_kernel=KERNEL_AUTO, large_variant=0) -> Opts:
    s = 0 if stream is None else int(stream)
    return Opts(int(path), int(operand), int(device), int(instance_id) & 0xFFFFFFFF, ctypes.c_void_p(s or None),
                int(tile_replicas), int(coupling_mem), int(tc_kernel), int(large_variant))


def create(J_k, h_k, frac_bits=0, o: Opts | None = None):
    J_k = np.ascontiguousarray(J_k, dtype=np.int8)
    h_k = np.ascontiguousarray(h_k, dtype=np.int32)
    n = h_k.shape[0]
    if J_k.shape != (n, n):
        raise ValueError("J_k must be N x N")
    h = ctypes.c_void_p()
    _check(load().phia_create(ctypes.byref(h), _np_ptr(J_k), _np_ptr(h_k), n, int(frac_bits),
                              ctypes.byref(o) if o is not None else None))
    return h


def create_from_device(J_k, h_k, frac_bits=0, o: Opts | None = None):
    """J_k: contiguous int8 [N, N] and h_k: contiguous int32 [N] device tensors (anything
    with data_ptr(), shape, dtype and is_contiguous())."""
    n = int(h_k.shape[0])
    if tuple(J_k.shape) != (n, n):
        raise ValueError("J_k must be N x N")
    if str(J_k.dtype) != "torch.int8" or str(h_k.dtype) != "torch.int32":
        raise TypeError("J_k must be int8 and h_k int32")
    if not (J_k.is_contiguous() and h_k.is_contiguous()):
        raise ValueError("J_k and h_k must be contiguous")
    h = ctypes.c_void_p()
    _check(load().phia_create_from_device(ctypes.byref(h), ctypes.c_void_p(J_k.data_ptr()),
                                          ctypes.c_void_p(h_k.data_ptr()), n, int(frac_bits),
                                          ctypes.byref(o) if o is not None else None))
    return h


def create_csr(row_ptr, col, val_k, h_k, frac_bits=0, o: Opts | None = None):
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val_k = np.ascontiguousarray(val_k, dtype=np.int8)
    h_k = np.ascontiguousarray(h_k, dtype=np.int32)
    h = ctypes.c_void_p()
    _check(load().phia_create_csr(ctypes.byref(h), _np_ptr(row_ptr), _np_ptr(col), _np_ptr(val_k),
                                  _np_ptr(h_k), h_k.shape[0], int(frac_bits),
                                  ctypes.byref(o) if o is not None else None))
    return h


def anneal(h, sched: Schedule, replicas: int, steps: int, seed: int):
    _check(load().phia_anneal(h, ctypes.byref(sched), int(replicas), int(steps), int(seed) & (2**64 - 1)))


def autotune(h, sched: Schedule, replicas: int, probe_iters: int = 200) -> TuneResult:
    r = TuneResult()
    _check(load().phia_autotune(h, ctypes.byref(sched), int(replicas), int(probe_iters), ctypes.byref(r)))
    return r


def best(h, n: int):
    e = ctypes.c_int64()
    spins = np.empty(n, dtype=np.int8)
    _check(load().phia_best(h, ctypes.byref(e), _np_ptr(spins)))
    return int(e.value), spins


def stats_get(h) -> Stats:
    s = Stats()
    _check(load().phia_stats_get(h, ctypes.byref(s)))
    return s


def replica_results(h, replicas: int, n: int):
    W = (n + 31) // 32
    be = np.empty(replicas, dtype=np.int64)
    bs = np.empty(replicas, dtype=np.int64)
    hs = np.empty(replicas, dtype=np.int64)
    bits = np.empty((replicas, W), dtype=np.uint32)
    _check(load().phia_replica_results(h, int(replicas), _np_ptr(be), _np_ptr(bs), _np_ptr(hs), _np_ptr(bits)))
    return be, bs, hs, bits


def gahmc(h, sched: GahmcSchedule, replicas, trajectories, seed, x=None, v=None, counts=None, events=None):
    """phia_gahmc: vanilla GAHMC (exact zero crossings) on a dense handle.  x, v, counts,
    events: optional device tensors ([R][N] float32, [R][2] int64, [R][cap] int32)."""
    cap = int(events.shape[1]) if events is not None else 0
    _check(load().phia_gahmc(h, ctypes.byref(sched), int(replicas), int(trajectories), int(seed) & (2**64 - 1),
                             _dev_ptr(x), _dev_ptr(v), _dev_ptr(counts), _dev_ptr(events), cap))


def acceptance(h, replicas: int):
    """(proposed, accepted) per replica of the last run (phia_acceptance)."""
    prop = np.empty(replicas, dtype=np.int64)
    acc = np.empty(replicas, dtype=np.int64)
    _check(load().phia_acceptance(h, int(replicas), _np_ptr(prop), _np_ptr(acc)))
    return prop, acc


def unpack_bits(bits, n: int) -> np.ndarray:
    """Bit-packed spins ([R][W] uint32, bit i%32 of word i/32 = (s_i == +1)) -> int8 [R][n]."""
    b = np.asarray(bits, dtype=np.uint32)
    idx = np.arange(n)
    on = (b[:, idx >> 5] >> (idx & 31).astype(np.uint32)) & 1
    return np.where(on == 1, 1, -1).astype(np.int8)


def run(h, sched: Schedule, replicas, t0, steps, total_steps, seed, x, v, reset_best=True):
    _check(load().phia_run(h, ctypes.byref(sched), int(replicas), int(t0), int(steps), int(total_steps),
                           int(seed) & (2**64 - 1), _dev_ptr(x), _dev_ptr(v), 1 if reset_best else 0))


def init_state(h, replicas, seed, x, v):
    _check(load().phia_init_state(h, int(replicas), int(seed) & (2**64 - 1), _dev_ptr(x), _dev_ptr(v)))


def field(h, spins, field_k=None, energy_k=None):
    _check(load().phia_field(h, _dev_ptr(spins), spins.shape[0], _dev_ptr(field_k), _dev_ptr(energy_k)))


def philox_draws(seed, instance_id, d, replicas, n, raw=None, x=None, v=None, stream=None):
    _check(load().phia_philox_draws(int(seed) & (2**64 - 1), int(instance_id) & 0xFFFFFFFF, int(d),
                                    int(replicas), int(n), _dev_ptr(raw), _dev_ptr(x), _dev_ptr(v),
                                    ctypes.c_void_p(int(stream) if stream else None)))


def run_noalloc(J_k, h_k, frac_bits, operand, sched: Schedule, replicas, t0, steps, total_steps, seed, instance_id,
                x, v, best_energy_k, best_step, hit_step, best_bits, reset_best=True, stream=None):
    """phia_run_noalloc: every argument a device tensor the caller owns; no allocation."""
    n = int(h_k.shape[0])
    _check(load().phia_run_noalloc(_dev_ptr(J_k), _dev_ptr(h_k), n, int(frac_bits), int(operand), ctypes.byref(sched),
                                   int(replicas), int(t0), int(steps), int(total_steps), int(seed) & (2**64 - 1),
                                   int(instance_id) & 0xFFFFFFFF, _dev_ptr(x), _dev_ptr(v), _dev_ptr(best_energy_k),
                                   _dev_ptr(best_step), _dev_ptr(hit_step), _dev_ptr(best_bits),
                                   1 if reset_best else 0, ctypes.c_void_p(int(stream) if stream else None)))


def mma_peak(operand, n=256, rounds=20000, stream=None):
    """(device ms, TFLOP/s or TOP/s) of the throughput probe (phia_mma_peak): tcgen05 with
    OP_E4M3 / OP_BF16, warp-level int8 mma.sync with PEAK_S8_MMA_SYNC."""
    ms, tf = ctypes.c_float(), ctypes.c_double()
    _check(load().phia_mma_peak(int(operand), int(n), int(rounds), ctypes.c_void_p(int(stream) if stream else None),
                                ctypes.byref(ms), ctypes.byref(tf)))
    return float(ms.value), float(tf.value)


def debug_wait(h, wait_budget_ns, stall_producer=False):
    _check(load().phia_debug_wait(h, int(wait_budget_ns), 1 if stall_producer else 0))


def sync(h):
    _check(load().phia_sync(h))


def destroy(h):
    if h:
        load().phia_destroy(h)


@dataclass
class Result:
    energy_k: int
    spins: np.ndarray
    stats: Stats


class Annealer:
    """One Ising instance on the device; ``anneal`` runs PHIA and returns the best state."""

    def __init__(self, J_k=None, h_k=None, frac_bits=0, csr=None, path=PATH_AUTO, operand=OP_AUTO,
                 device=0, instance_id=0, stream=None, tile_replicas=0, coupling_mem=MEM_AUTO,
                 tc_kernel=KERNEL_AUTO, large_variant=0):
        o = opts(path, operand, device, instance_id, stream, tile_replicas, coupling_mem, tc_kernel, large_variant)
        if csr is not None:
            row_ptr, col, val = csr
            self.n = len(row_ptr) - 1
            self.h = create_csr(row_ptr, col, val, h_k, frac_bits, o)
        elif hasattr(J_k, "data_ptr") and getattr(J_k, "is_cuda", False):
            self.n = int(h_k.shape[0])
            self.h = create_from_device(J_k, h_k, frac_bits, o)   # device tensors: no host copy
        else:
            self.n = int(np.asarray(h_k).shape[0])
            self.h = create(J_k, h_k, frac_bits, o)

    def anneal(self, sched: Schedule, replicas: int, steps: int, seed: int) -> Result:
        anneal(self.h, sched, replicas, steps, seed)
        e, s = best(self.h, self.n)
        return Result(e, s, stats_get(self.h))

    def close(self):
        destroy(self.h)
        self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            if getattr(self, "h", None):
                self.close()
        except Exception:
            pass


class Batch:
    """Many instances annealed together on the sparse path (phia_batch_*).

    ``instances``: objects with ``kh``, ``frac_bits`` and either ``k`` (dense) or
    ``row_ptr``/``col``/``val`` (CSR), e.g. from ``instances.py``.  ``targets``: optional
    per-instance target energies (units of q) or None entries."""

    def __init__(self, instances, instance_ids=None, targets=None, device=0, stream=None, csr_mode=0):
        self._keep = []
        descs = (InstanceDesc * len(instances))()
        self.n = []
        for k, inst in enumerate(instances):
            kh = np.ascontiguousarray(inst.kh, dtype=np.int32)
            self._keep.append(kh)
            d = descs[k]
            d.N = kh.shape[0]
            d.frac_bits = int(getattr(inst, "frac_bits", 0))
            d.h_k = kh.ctypes.data
            if getattr(inst, "k", None) is not None:
                J = np.ascontiguousarray(inst.k, dtype=np.int8)
                self._keep.append(J)
                d.J_k = J.ctypes.data
            else:
                rp = np.ascontiguousarray(inst.row_ptr, dtype=np.int32)
                col = np.ascontiguousarray(inst.col, dtype=np.int32)
                val = np.ascontiguousarray(inst.val, dtype=np.int8)
                self._keep += [rp, col, val]
                d.row_ptr, d.col, d.val_k = rp.ctypes.data, col.ctypes.data, val.ctypes.data
            d.instance_id = k if instance_ids is None else int(instance_ids[k])
            tg = None if targets is None else targets[k]
            d.has_target = 0 if tg is None else 1
            d.target_k = 0 if tg is None else int(tg)
            self.n.append(int(d.N))
        o = opts(path=PATH_AUTO, device=device, stream=stream, tc_kernel=csr_mode)
        self.h = ctypes.c_void_p()
        _check(load().phia_batch_create(ctypes.byref(self.h), len(instances), descs, ctypes.byref(o)))
        self._keep = None

    def anneal(self, sched: Schedule, replicas: int, steps: int, seed: int):
        _check(load().phia_batch_anneal(self.h, ctypes.byref(sched), int(replicas), int(steps),
                                        int(seed) & (2**64 - 1)))

    def autotune(self, sched: Schedule, replicas: int, probe_iters: int = 50) -> TuneResult:
        r = TuneResult()
        _check(load().phia_batch_autotune(self.h, ctypes.byref(sched), int(replicas), int(probe_iters), ctypes.byref(r)))
        return r

    def best(self, k: int):
        e = ctypes.c_int64()
        spins = np.empty(self.n[k], dtype=np.int8)
        _check(load().phia_batch_best(self.h, int(k), ctypes.byref(e), _np_ptr(spins)))
        return int(e.value), spins

    def replica_results(self, k: int, replicas: int):
        W = (self.n[k] + 31) // 32
        be = np.empty(replicas, dtype=np.int64)
        bs = np.empty(replicas, dtype=np.int64)
        hs = np.empty(replicas, dtype=np.int64)
        bits = np.empty((replicas, W), dtype=np.uint32)
        _check(load().phia_batch_replica_results(self.h, int(k), int(replicas), _np_ptr(be), _np_ptr(bs),
                                                 _np_ptr(hs), _np_ptr(bits)))
        return be, bs, hs, bits

    def stats(self) -> Stats:
        st = Stats()
        _check(load().phia_batch_stats_get(self.h, ctypes.byref(st)))
        return st

    def sync(self):
        _check(load().phia_batch_sync(self.h))

    def close(self):
        if self.h:
            load().phia_batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def _desc_of(inst, instance_id=0, target=None):
    """InstanceDesc for a Dense/Csr instance; returns (desc, arrays kept alive)."""
    keep = []
    d = InstanceDesc()
    kh = np.ascontiguousarray(inst.kh, dtype=np.int32)
    keep.append(kh)
    d.N = kh.shape[0]
    d.frac_bits = int(getattr(inst, "frac_bits", 0))
    d.h_k = kh.ctypes.data
    if getattr(inst, "k", None) is not None:
        J = np.ascontiguousarray(inst.k, dtype=np.int8)
        keep.append(J)
        d.J_k = J.ctypes.data
    else:
        rp = np.ascontiguousarray(inst.row_ptr, dtype=np.int32)
        col = np.ascontiguousarray(inst.col, dtype=np.int32)
        val = np.ascontiguousarray(inst.val, dtype=np.int8)
        keep += [rp, col, val]
        d.row_ptr, d.col, d.val_k = rp.ctypes.data, col.ctypes.data, val.ctypes.data
    d.instance_id = int(instance_id) & 0xFFFFFFFF
    d.has_target = 0 if target is None else 1
    d.target_k = 0 if target is None else int(target)
    return d, keep


class Server:
    """The continuous-batching request loop (phia_server_*)."""

    def __init__(self, max_inflight=8, hbm_budget_bytes=8 << 30, chunk_iters=100, device=0, path=PATH_AUTO):
        o = ServerOpts(int(device), int(max_inflight), int(hbm_budget_bytes), int(chunk_iters), int(path))
        self.h = ctypes.c_void_p()
        _check(load().phia_server_create(ctypes.byref(self.h), ctypes.byref(o)))
        self.n = {}

    def submit(self, inst, sched: Schedule, replicas, step_cap, seed, instance_id=0, target=None) -> int:
        d, keep = _desc_of(inst, instance_id, target)
        rid = ctypes.c_int64()
        _check(load().phia_server_submit(self.h, ctypes.byref(d), ctypes.byref(sched), int(replicas), int(step_cap),
                                         int(seed) & (2**64 - 1), ctypes.byref(rid)))
        self.n[rid.value] = int(d.N)
        return int(rid.value)

    def poll(self, rid: int, want_spins=False):
        st = RequestStatus()
        spins = np.empty(self.n[rid], dtype=np.int8) if want_spins else None
        _check(load().phia_server_poll(self.h, int(rid), ctypes.byref(st), _np_ptr(spins)))
        return st, spins

    def wait_all(self, timeout_ms=600_000):
        _check(load().phia_server_wait_all(self.h, int(timeout_ms)))

    def stats(self) -> ServerStats:
        st = ServerStats()
        _check(load().phia_server_stats_get(self.h, ctypes.byref(st)))
        return st

    def close(self):
        if self.h:
            load().phia_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
