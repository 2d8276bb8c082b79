"""Benchmark of the PHIA hot path on GB300.

Workload (one bench step = one whole PHIA run, i.e. every row of the hot path over one
batch): the N = 2000 complete graph, J_ij uniform in {-1,+1}, h = 0 (seed 3), 4096
replicas x 5000 iterations, beta linear 0.005 -> 0.134, eps 0.1, gamma 2, momentum
refreshed every 50 iterations, run on the kernel the autotuner picks among the thirteen
per-iteration tcgen05 variants (at this size the overlapped kernel, one cooperative launch
per run).  Metric: spin updates per second = replicas * N * iterations
/ time.

  value        device time of phia_anneal with the instance resident in HBM (CUDA events
               on the handle's stream), whole job over all ranks (weak scaling: every
               rank anneals its own replicas, no collective on the data path).
  e2e          same metric through the public C ABI from host buffers: phia_create
               (host -> device copy of J, h) + phia_anneal + phia_best (device -> host
               copy of the result) per step, wall clock.
  roofline     dominant kernel: the dense field (Eq. 6) is 2 N flops per spin update;
               achieved = 2 R N^2 per launch / the kernel's mean launch time, against the
               e4m3 tensor peak (the measured bf16 peak x 2, the nominal e4m3 : bf16 ratio);
               the HBM fraction of the algorithmic bytes beside it, and the e4m3 / bf16
               rates this library's own tcgen05 probe (phia_mma_peak) measures on the box.
  cpu_baseline the FP64 oracle on the host cores over a bounded sample of the workload
               (rank 0, N = 1 only), extrapolated per spin update.
  comparator   the plain FP32 per-instance GPU path on the same instance and seeds.
  clocks       SM clock and throttle reasons sampled by NVML every 5 ms inside the timed
               region (a child process started before the warm-up).
  also         (N = 1 only) the other workloads measured the same way, shorter: N = 200
               dense (1024 x 2000, resident kernel), the 256-instance Erdos-Renyi batch,
               and the serving stream (p50 / p99 time to target).

L2 is flushed (256 MB write) between timed steps.  `--impl reference` times the oracle
(this method has no reference code; the oracle is the reference arm) on a bounded
sample of the workload per step.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # N = 200 dense, k and kh in [-7, 7], 1024 replicas x 2000 iterations
    "dense200": dict(N=200, kind="int", kmax=7, hmax=7, seed=1, replicas=1024, iterations=2000,
                     beta0=0.01, beta1=0.1, eps=0.1, gamma=2.0, refresh=50, run_seed=12345,
                     name="N=200 dense, k and kh uniform int [-7,7]; 1024 replicas x 2000 iterations, "
                          "linear beta 0.01->0.1",
                     cmp_iters=2000, cpu_replicas=1024, cpu_iters=2000),
    # plain PHIA: N = 16 SK instance (seed 0), one replica x 1000 iterations; a latency case
    # (one CTA), reported as time per iteration
    "sk16": dict(N=16, kind="pm1", seed=0, replicas=1, iterations=1000,
                 beta0=0.05, beta1=2.0, eps=0.2, gamma=2.0, refresh=0, run_seed=1,
                 name="N=16 SK instance (J uniform {-1,+1}, h=0, seed 0); 1 replica x 1000 iterations",
                 cmp_iters=1000, cpu_replicas=1, cpu_iters=1000),
    # the default workload: complete graph N = 2000, J in {-1,+1}, h = 0, 4096 replicas x
    # 5000 iterations
    "dense2000": dict(N=2000, kind="pm1", seed=3, replicas=4096, iterations=5000,
                      beta0=0.005, beta1=0.134, eps=0.1, gamma=2.0, refresh=50, run_seed=777,
                      name="N=2000 complete graph, J uniform {-1,+1}, h=0; 4096 replicas x 5000 iterations",
                      cmp_iters=20, cpu_replicas=256, cpu_iters=50),
    # 256 Erdos-Renyi instances of uneven N, fixed point (f = 4), one batch
    "batched_er": dict(kind="batch", count=256, seed=4, replicas=256, iterations=2000,
                       beta0=0.01, beta1=0.18, eps=0.1, gamma=2.0, refresh=50, run_seed=4242,
                       name="256 Erdos-Renyi instances, N ~ U[100,3000], density ~ U[0.006,0.06], J = k/16 "
                            "(k ~ U[-127,127]), h = k/16 (k ~ U[-31,31]); 256 replicas each x 2000 iterations, "
                            "one batch",
                       cmp_instances=8, cmp_iters=20, cpu_instances=4, cpu_iters=50),
    # time-to-solution scaling (Eq. 9) of PHIA on the seven Table 2 families, n = 8..1024,
    # 100 instances per n; vanilla GAHMC on the same sk_ising instances for the Sec. 3.2
    # ablation
    "tts": dict(kind="tts", sizes=(8, 16, 32, 64, 128, 256, 512, 1024), instances=100, replicas=256,
                iterations=1000, ref_replicas=1024, ref_factor=4, streams=8, jump=None,
                # 3-regular max-cut: fields of at most 3 units; a sweep of eps, gamma, the
                # trajectory length and the final jump on 12 instances each at n = 256, 512 and
                # 1024, scored against the best of every setting's longer run, chose these
                family_schedule={"maxcut_d3": dict(eps=0.3, gamma=1.0, refresh=20, jump=12.0)},
                gahmc_family="sk_ising", gahmc_sizes=(8, 16, 32, 64, 128, 256), gahmc_trajectories=200,
                name="TTS99 scaling on the Table 2 families (maxcut_dense, maxcut_d3, sk_bool, sk_ising, "
                     "sk_uniform, nae_3_sat, spin_model), n = 8..1024, 100 instances per n; 256 replicas x "
                     "1000 max(1, n/128) max(1, n/256) iterations; optimum: exhaustive for n <= 16, planted for nae_3_sat, "
                     "else the best of the run and of 1024 replicas x 4 times as many iterations (for maxcut_d3, "
                     "which runs its own schedule, of such a run under each of its schedule and the heuristic's)"),
    # serving stream, Poisson arrivals at 200/s over a pool of seeded instances
    "serving": dict(kind="serving", pool=32, pool_seed=5, requests=2000, arrival_seed=11, rate_hz=200.0,
                    replicas=256, step_cap=5000, max_inflight=64, budget_gb=64, chunk_iters=200,
                    cmp_requests=60, cmp_wall_s=90.0,
                    name="serving: Poisson 200/s, N log-uniform [64,8192], half dense {-1,+1}, half sparse "
                         "f=8 density 0.01; 256 replicas, step cap 5000, target = best of an oracle run of up to "
                         "64 replicas x 5000 iterations (4e11 field multiply-adds per instance)"),
}
WORKLOAD = WORKLOADS["dense2000"]
WORKLOAD_NAME = WORKLOAD["name"]
METRIC = "spin-updates/s"
# dram__bytes_read.sum + dram__bytes_write.sum of one launch of each kernel, from the
# committed ncu summaries under profiles/; absent once a kernel changed after its capture.
KERNEL_TRAFFIC_BYTES = {
    "tc_flow_run": (2_078_996_000 + 4_795_566_000) // 100,   # N = 2000, 4096 replicas: a 100-iteration launch,
                                                             # per iteration (a launch runs all of them)
    "tc_large_step": None,                                   # not re-captured since its last change
    "csr_step": 975_512_832 + 774_093_056,                   # 256 ER instances, 256 replicas (one iteration)
    "tc_small_kernel": 140_544,                              # N = 200, 1024 replicas (a launch is the whole run)
}


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _instance(w=None):
    from paper_2407_10205_gb300 import instances as ins
    w = w or WORKLOAD
    if w["kind"] == "pm1":
        return ins.sk_pm1(w["N"], w["seed"])
    return ins.dense_int(w["N"], w["kmax"], w["hmax"], w["seed"])


# sampler period: 1 ms polling slowed the timed process's host calls (not its device time)
CLOCK_POLL_MS = 5.0
# NVML clock-event reason bits (nvml.h) reported by the sampler
_NVML_REASONS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20,
                 "hw_thermal_slowdown": 0x40}


def _nvml_poll(dev, period_ms):
    """Body of the sampler's child process: print `monotonic_s,sm_mhz,max_sm_mhz,reason_bits`
    for the device (PCI bus id or NVML index) every `period_ms`, reading NVML through ctypes.
    Read-only queries; exits non-zero if NVML or the device is unavailable, zero once its
    parent is gone."""
    import ctypes
    try:
        nv = ctypes.CDLL("libnvidia-ml.so.1")
    except OSError:
        return 1
    if nv.nvmlInit_v2() != 0:
        return 1
    h = ctypes.c_void_p()
    if ":" in dev:
        rc = nv.nvmlDeviceGetHandleByPciBusId_v2(dev.encode(), ctypes.byref(h))
    else:
        rc = nv.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(int(dev)), ctypes.byref(h))
    if rc != 0:
        return 1
    reasons = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
        nv.nvmlDeviceGetCurrentClocksThrottleReasons
    NVML_CLOCK_SM = 1
    mx, clk, bits = ctypes.c_uint(0), ctypes.c_uint(0), ctypes.c_ulonglong(0)
    nv.nvmlDeviceGetMaxClockInfo(h, NVML_CLOCK_SM, ctypes.byref(mx))
    parent = os.getppid()
    try:
        while os.getppid() == parent:             # ends with the timed process
            if nv.nvmlDeviceGetClockInfo(h, NVML_CLOCK_SM, ctypes.byref(clk)) == 0 and \
                    reasons(h, ctypes.byref(bits)) == 0:
                print(f"{time.monotonic():.6f},{clk.value},{mx.value},{bits.value}", flush=True)
            time.sleep(period_ms * 1e-3)
    except (BrokenPipeError, KeyboardInterrupt):
        pass
    return 0


class ClockSampler:
    """SM clock and clock-event (throttle) reasons sampled DURING the timed region: NVML
    polled every CLOCK_POLL_MS by a child process (so short regions still get samples and the
    timed process is not disturbed); only samples stamped inside the `with` block count.
    Falls back to nvidia-smi every 200 ms where NVML cannot be loaded."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.source = None
        self.lines = []

    def _device_key(self):
        try:
            import torch
            p = torch.cuda.get_device_properties(self.gpu)
            return f"{p.pci_domain_id:08X}:{p.pci_bus_id:02X}:{p.pci_device_id:02X}.0"
        except Exception:
            return str(self.gpu)

    def start(self):
        """Start the poller (before warm-up: a new NVML client stalls the process's first
        host calls after it attaches, which must not land in the timed region).  Samples go
        to a temporary file, so a long warm-up cannot fill a pipe and stall the poller."""
        if self.proc is not None:
            return self
        import tempfile
        self.out = tempfile.TemporaryFile(mode="w+b")
        try:
            self.proc = subprocess.Popen(
                [sys.executable, os.path.abspath(__file__), "--clock-poll", self._device_key()],
                stdout=self.out, stderr=subprocess.DEVNULL, text=True)
            deadline = time.monotonic() + 30.0
            while self.proc.poll() is None and os.fstat(self.out.fileno()).st_size == 0 \
                    and time.monotonic() < deadline:
                time.sleep(0.01)                       # the poller is live before timing starts
            if self.proc.poll() is None and os.fstat(self.out.fileno()).st_size > 0:
                self.source = f"nvml, {CLOCK_POLL_MS:g} ms"
            else:
                self._stop()
        except OSError:
            self.proc = None
        if self.proc is None:
            try:
                self.proc = subprocess.Popen(
                    ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                     "--format=csv,noheader,nounits", "-lms", "200"],
                    stdout=self.out, stderr=subprocess.DEVNULL)
                self.source = "nvidia-smi, 200 ms"
            except OSError:
                self.proc = None
        return self

    def _stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.proc.wait()
            self.proc = None

    def __enter__(self):
        self.start()
        self.off0 = os.fstat(self.out.fileno()).st_size     # output written before the region
        self.t0 = time.monotonic()
        return self

    def __exit__(self, *a):
        self.t1 = time.monotonic()
        self._stop()
        self.out.seek(0)
        data = self.out.read()
        self.out.close()
        cut = data.rfind(b"\n", 0, self.off0) + 1             # whole lines from the region on
        self.lines = [l for l in data[cut:].decode(errors="replace").splitlines() if l.strip()]

    def _samples(self):
        """(sm_mhz, max_mhz, set of active reason names) per sample inside the region."""
        out = []
        for l in self.lines:
            f = [t.strip() for t in l.split(",")]
            try:
                if self.source and self.source.startswith("nvml"):
                    if len(f) != 4 or not (self.t0 <= float(f[0]) <= self.t1):
                        continue
                    bits = int(f[3])
                    out.append((float(f[1]), float(f[2]),
                                {n for n, b in _NVML_REASONS.items() if bits & b}))
                elif len(f) >= 9:
                    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
                    out.append((float(f[1]), float(f[2]),
                                {n for n, val in zip(names, f[5:9]) if val.lower().startswith("active")}))
            except ValueError:
                continue
        return out

    def summary(self):
        s = self._samples()
        reasons = set().union(*(r for _, _, r in s)) if s else set()
        mx = s[-1][1] if s else None
        if not s:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0, "source": self.source}
        sm = [c for c, _, _ in s]
        loaded = [c for c in sm if mx is None or c > 0.5 * mx] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm), "sm_mhz_min": min(sm), "source": self.source}


def cpu_baseline(w=None, sample_replicas=None):
    """The FP64 oracle, as it stands, on the host cores: a bounded sample of the workload
    (`sample_replicas` replicas x the workload's sample iterations), its rate extrapolated
    per spin update to the whole workload."""
    import oracle
    w = w or WORKLOAD
    R = sample_replicas or w["cpu_replicas"]
    T = w["cpu_iters"]
    d = _instance(w)
    P = oracle.Instance(d.kh, k=d.k)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    oracle.anneal(P, R, T, w["run_seed"], 0, w["beta0"], w["beta1"], w["eps"],
                  w["gamma"], refresh=w["refresh"], threads=cores, want_spins=False)
    dt = time.perf_counter() - t0
    su = R * w["N"] * T
    whole = R == w["replicas"] and T == w["iterations"]
    # the oracle runs one thread per replica at a time: the threads it actually used
    return {"value": su / dt, "unit": METRIC, "cores": min(cores, R), "kind": "oracle",
            "sample": f"{R} of the {w['replicas']} replicas x {T} of {w['iterations']} iterations ({dt:.1f} s)"
                      + ("" if whole else ", extrapolated per spin update"),
            "seconds": dt}


def run_reference(args):
    """The reference arm: the oracle (this paper has no reference code) on the machine's host
    cores, each step the workload's bounded CPU sample."""
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    per_step, secs = [], []
    cb = None
    for k in range(args.warmup + args.steps):
        r = cpu_baseline()
        if k >= args.warmup:
            per_step.append(r["value"])
            secs.append(r["seconds"])
            cb = r
    val = statistics.median(per_step)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.median(secs) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME, "sample_per_step": cb["sample"].split(" (")[0]},
            "cpu_baseline": {"kind": "oracle", "cores": cb["cores"], "sample": cb["sample"], "value": val,
                             "unit": METRIC},
            "e2e": {"value": val, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return m, "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def mma_probe(phia):
    """Dense rates measured on this GPU by the library's own probe (phia_mma_peak): tcgen05
    M = 128, N = 256 MMAs from shared memory on every SM, e4m3 and bf16 (TFLOP/s); and the
    warp-level int8 mma.sync route of the int8 resident kernel (integer TOP/s)."""
    out = {}
    for name, op in (("e4m3", phia.OP_E4M3), ("bf16", phia.OP_BF16), ("s8_mma_sync", phia.PEAK_S8_MMA_SYNC)):
        try:
            ms, tf = phia.mma_peak(op, 256, 20000)
            out[name + "_tflops"] = tf
        except Exception as e:                      # noqa: BLE001 -- reported, not fatal
            out[name + "_error"] = str(e)
    return out


def _roofline(w, kernel_ms, stats, peaks, src, probe=None, large_variant=0):
    """Roofline of the dominant kernel of a dense workload.  The field (Eq. 6) is a dense
    contraction of 2 N flops per spin update (2 R N^2 per iteration): achieved = those
    flops / device time, against the e4m3 tensor peak taken as the measured bf16 burst
    peak x 2 (the nominal e4m3 : bf16 ratio; the operand here is e4m3 when every |k| <= 16,
    else bf16 at the measured bf16 peak).  Beside it: the same flops against the rates the
    library's own tcgen05 probe measured, and for the per-iteration kernel the fraction of
    HBM bandwidth its algorithmic bytes reach (x and v in and out, 16 B per spin update;
    the next spins, 1 B; the spins read once, 1 B; J once, N^2 B)."""
    N, R, T = w["N"], w["replicas"], w["iterations"]
    su = R * N * T
    e4m3 = stats.operand == 1
    bf16_peak = float(peaks["bf16_tflops"])
    peak = 2.0 * bf16_peak if e4m3 else bf16_peak
    achieved = 2.0 * N * su / (kernel_ms * 1e-3) / 1e12
    kname = {1: "tc_small_kernel", 2: "tc_flow_run" if large_variant >= 7 else "tc_large_step",
             3: "imma_small_kernel", 4: "inc_small_kernel"}.get(stats.tc_kernel, "?")
    out = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
           "traffic": KERNEL_TRAFFIC_BYTES.get(kname), "kernel": kname,
           "flops_per_spin_update": 2 * N,
           "peak_source": (f"{src} bf16 {bf16_peak:g} TFLOP/s x 2 (nominal e4m3 : bf16 ratio)" if e4m3
                           else f"{src} bf16 {bf16_peak:g} TFLOP/s")}
    if probe:
        mp = probe.get("e4m3_tflops" if e4m3 else "bf16_tflops")
        if mp:
            out["probe_peak"] = mp
            out["frac_of_probe_peak"] = achieved / mp
    if stats.tc_kernel == 2:
        # per iteration: one launch of tc_large_step; tc_flow_run runs all T in one launch,
        # so its per-launch figures are T times these over T times the time
        launch_ms = kernel_ms / T
        bytes_per_launch = R * N * 17 + R * N + N * N
        hbm = bytes_per_launch / (launch_ms * 1e-3) / 1e9
        out["launch_ms"] = launch_ms
        out["per"] = "iteration"
        out["hbm"] = {"achieved": hbm, "peak": float(peaks["hbm_gbs"]), "unit": "GB/s",
                      "frac": hbm / float(peaks["hbm_gbs"]), "algorithmic_bytes_per_launch": bytes_per_launch,
                      "peak_source": f"{src} HBM copy bandwidth"}
    return out


def measure_batch(args, w, light=False):
    """The batched workload: one phia_batch over all instances; the comparator is the
    plain FP32 per-instance dense path, timed on a sample of instances and scaled by N^2.
    light: no CPU baseline."""
    import torch
    import oracle
    from paper_2407_10205_gb300 import instances as ins
    from paper_2407_10205_gb300 import phia
    phia.load()
    insts = ins.batched_er(w["count"], w["seed"])
    R, T = w["replicas"], w["iterations"]
    sched = phia.schedule(w["beta0"], w["beta1"], w["eps"], w["gamma"], refresh=w["refresh"])
    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    Ns = np.array([c.n for c in insts])
    nnz = np.array([c.nnz for c in insts])
    su_step = int(R * T * Ns.sum())
    cs = ClockSampler(0).start()
    with phia.Batch(insts, stream=stream.cuda_stream) as B:
        tune = B.autotune(sched, R, probe_iters=40)        # persistent CSR launch or one per iteration
        for _ in range(args.warmup):
            flush.fill_(0.0)                          # the flush kernel is loaded before timing
            B.anneal(sched, R, T, w["run_seed"])
            B.sync()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        torch.cuda.synchronize()
        with cs:
            for k in range(args.steps):
                flush.fill_(float(k))
                torch.cuda.current_stream().synchronize()
                ev[k][0].record(stream)
                B.anneal(sched, R, T, w["run_seed"])
                ev[k][1].record(stream)
            torch.cuda.synchronize()
        st = B.stats()
        ms = [a.elapsed_time(b) for a, b in ev]
        best0 = B.best(0)[0]
    ms_per_step = sum(ms) / len(ms)
    value = su_step / (ms_per_step * 1e-3)
    # e2e: batch creation from host arrays + anneal + every instance's best
    t0 = time.perf_counter()
    with phia.Batch(insts, stream=stream.cuda_stream, csr_mode=tune.tc_kernel) as B2:   # the launch form tuned above
        B2.anneal(sched, R, T, w["run_seed"])
        for k in range(len(insts)):
            B2.best(k)
    e2e_ms = (time.perf_counter() - t0) * 1e3
    h2d = int(sum(4 * (c.n + 1) + 5 * c.nnz + 4 * c.n for c in insts))
    d2h = int(sum(3 * 8 * R + 4 * ((c.n + 31) // 32) + c.n for c in insts))
    # comparator on a sample
    g = np.random.default_rng(0)
    sample = sorted(g.choice(len(insts), size=w["cmp_instances"], replace=False).tolist())
    per_n2 = []
    for k in sample:
        dd = insts[k].to_dense()
        with phia.Annealer(dd.k, dd.kh, frac_bits=dd.frac_bits, path=phia.PATH_FP32, stream=stream.cuda_stream) as C:
            phia.anneal(C.h, sched, R, w["cmp_iters"], w["run_seed"])
            phia.sync(C.h)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            phia.anneal(C.h, sched, R, w["cmp_iters"], w["run_seed"])
            e1.record(stream)
            stream.synchronize()
            per_n2.append(e0.elapsed_time(e1) / w["cmp_iters"] / dd.n ** 2)
    cmp_ms = float(np.mean(per_n2)) * float((Ns.astype(np.float64) ** 2).sum()) * T
    # CPU baseline on a sample
    cores = os.cpu_count() or 1
    tc0 = time.perf_counter()
    su_cpu = 0
    for k in range(0 if light else w["cpu_instances"]):
        c = insts[k]
        P = oracle.Instance(c.kh, row_ptr=c.row_ptr, col=c.col, val=c.val, frac_bits=c.frac_bits)
        oracle.anneal(P, R, w["cpu_iters"], w["run_seed"], k, w["beta0"], w["beta1"], w["eps"], w["gamma"],
                      refresh=w["refresh"], threads=cores, want_spins=False)
        su_cpu += R * c.n * w["cpu_iters"]
    dt_cpu = time.perf_counter() - tc0
    peaks, src = _peaks()
    launch_ms = float(st.device_ms) / T
    bytes_launch = float(R * Ns.sum() * (16 + 1.0 / 8) + 5 * nnz.sum() * max(1, R // 256))
    csr_kernel = "csr_step" if tune.tc_kernel == 2 else "csr_persistent"
    achieved = bytes_launch / (launch_ms * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "fp32", "data": "synthetic",
        "config": {"workload": w["name"], "instances": len(insts), "total_spins": int(Ns.sum()),
                   "nnz": int(nnz.sum()), "replicas": R, "iterations": T, "path": "csr batch",
                   "csr_launch": {1: "one persistent cooperative launch", 2: "one launch per iteration"}.get(
                       tune.tc_kernel), "autotune_us_per_iter": [tune.best_us_per_iter, tune.worst_us_per_iter],
                   "l2": "flushed between timed steps (256 MB write)"},
        "e2e": {"value": su_step / (e2e_ms * 1e-3), "unit": METRIC, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": float(peaks["hbm_gbs"]), "unit": "GB/s",
                     "frac": achieved / float(peaks["hbm_gbs"]), "traffic": KERNEL_TRAFFIC_BYTES.get(csr_kernel),
                     "kernel": csr_kernel, "launch_ms": launch_ms, "algorithmic_bytes_per_launch": bytes_launch,
                     "peak_source": f"{src} HBM copy bandwidth"},
        "gpu_launches": args.steps * st.kernel_launches,
        "clocks": cs.summary(),
        "comparator": {"path": "fp32 per-instance dense, one launch per step", "value": su_step / (cmp_ms * 1e-3),
                       "unit": METRIC, "ms_per_run": cmp_ms,
                       "scaled": f"{w['cmp_instances']} instances x {w['cmp_iters']} iterations, time per N^2"},
        "best_energy_k_instance0": int(best0),
    }
    if not light:
        line["cpu_baseline"] = {"value": su_cpu / dt_cpu, "unit": METRIC, "cores": cores, "kind": "oracle",
                                "sample": f"{w['cpu_instances']} instances x {R} replicas x {w['cpu_iters']} "
                                          f"iterations ({dt_cpu:.1f} s), extrapolated per spin update"}
    return line


def _serve_stream(phia, pool, targets, arrivals, w, path, wall_cap_s=None):
    """Replay an arrival stream against a server; returns per-request statuses and stats."""
    import threading
    from paper_2407_10205_gb300 import schedules
    scheds = []
    for inst in pool:
        b0, b1, eps, gamma, refresh = schedules.suggest_schedule(inst, jump=6.0)
        scheds.append(phia.schedule(b0, b1, eps, gamma, refresh=refresh))
    S = phia.Server(max_inflight=w["max_inflight"], hbm_budget_bytes=int(w["budget_gb"] * (1 << 30)),
                    chunk_iters=w["chunk_iters"], path=path)
    ids = []
    t0 = time.perf_counter()

    def submitter():
        for (ta, k, sd) in arrivals:
            dt = ta - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            ids.append(S.submit(pool[k], scheds[k], w["replicas"], w["step_cap"], sd, instance_id=k,
                                target=targets[k]))

    th = threading.Thread(target=submitter)
    th.start()
    th.join()
    try:
        S.wait_all(timeout_ms=int((wall_cap_s or 3600) * 1000))
        complete = True
    except phia.PhiaError:
        complete = False
    sts = [S.poll(r)[0] for r in ids]
    st = S.stats()
    S.close()
    return sts, st, complete


def measure_serving(args, w):
    """The serving workload: a stream of requests through the continuous-batching server."""
    import torch
    from paper_2407_10205_gb300 import instances as ins
    from paper_2407_10205_gb300 import phia
    phia.load()
    with open(os.path.join(ROOT, "tests", "golden", "serving_targets.json")) as f:
        tdoc = json.load(f)
    pool = ins.serving_pool(w["pool"], w["pool_seed"])
    targets = [e["target_k"] for e in tdoc["entries"]]
    arrivals = ins.serving_arrivals(w["requests"], w["arrival_seed"], len(pool), w["rate_hz"])
    cs = ClockSampler(0).start()
    # warm-up: one request of each pool entry (builds kernels, loads modules)
    _serve_stream(phia, pool, targets, [(0.0, k, 1) for k in range(len(pool))], w, phia.PATH_AUTO)
    with cs:
        sts, st, complete = _serve_stream(phia, pool, targets, arrivals, w, phia.PATH_AUTO)
    done = [s for s in sts if s.state == 2]
    span = max(s.t_done_s for s in done) - min(s.t_submit_s for s in sts)
    value = st.spin_updates / span
    cmp_arr = arrivals[: w["cmp_requests"]]
    if args.no_comparator:
        cst = ours_first = None
        ccomplete = False
    else:
        csts, cst, ccomplete = _serve_stream(phia, pool, targets, cmp_arr, w, phia.PATH_FP32, w["cmp_wall_s"])
        ours_first = _serve_stream(phia, pool, targets, cmp_arr, w, phia.PATH_AUTO)[1]
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": 1, "steps": 1, "warmup": 1,
        "ms_per_step": span * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "fp32", "data": "synthetic",
        "config": {"workload": w["name"], "requests": len(arrivals), "pool": len(pool),
                   "max_inflight": w["max_inflight"], "budget_gb": w["budget_gb"], "chunk_iters": w["chunk_iters"]},
        "serving": {"completed": st.completed, "hits": st.hits, "ttt_p50_s": st.ttt_p50_s, "ttt_p99_s": st.ttt_p99_s,
                    "ttt_admit_p50_s": st.ttt_admit_p50_s, "ttt_admit_p99_s": st.ttt_admit_p99_s,
                    "span_s": span, "spin_updates": st.spin_updates, "all_done": complete},
        "comparator": None if cst is None else {
            "path": "fp32 per-instance (same server, PHIA_PATH_FP32)", "requests": len(cmp_arr),
            "completed": cst.completed, "hits": cst.hits, "ttt_p50_s": cst.ttt_p50_s,
            "ttt_p99_s": cst.ttt_p99_s, "all_done_within_s": w["cmp_wall_s"] if ccomplete else None,
            "ours_on_same_requests": {"ttt_p50_s": ours_first.ttt_p50_s, "ttt_p99_s": ours_first.ttt_p99_s,
                                      "hits": ours_first.hits}},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": None, "d2h_bytes_per_step": None,
                "note": "serving is end to end by construction: host instances in, results out"},
        "clocks": cs.summary(),
    }
    return line


def tts99(t1, p):
    """Eq. 9 at 99% confidence, its brackets read as grouping: T1 log(0.01) / log(1 - P),
    T1 itself once P >= 0.99, infinite when P = 0."""
    if p <= 0.0:
        return math.inf
    if p >= 0.99:
        return t1
    return t1 * math.log(1.0 - 0.99) / math.log(1.0 - p)


def _tts_optima():
    with open(os.path.join(ROOT, "tests", "golden", "tts_optima.json")) as f:
        return json.load(f)["optima"]


def tts_schedule_params(w, args, fam, d, own=True):
    """(beta0, beta1, eps, gamma, refresh) of a run of the time-to-solution study on
    instance d of family fam.  own: the family's entry of w["family_schedule"] where it
    has one, else the schedule heuristic; not own: the heuristic alone (the reference's
    second run for a family with an entry).  A nonzero args.tts_jump sets the final jump
    of either; nonzero args.tts_eps, tts_gamma and tts_refresh override the own schedule's."""
    from paper_2407_10205_gb300 import schedules
    f = w.get("family_schedule", {}).get(fam, {}) if own else {}
    b0, b1, eps, gamma, refresh = schedules.suggest_schedule(d, jump=args.tts_jump or f.get("jump") or w["jump"])
    if not own:
        return b0, b1, eps, gamma, refresh
    return (b0, b1, args.tts_eps or f.get("eps") or eps, args.tts_gamma or f.get("gamma") or gamma,
            args.tts_refresh or f.get("refresh") or refresh)


def run_tts(args, w):
    """Time to solution (Eq. 9, 99% confidence) against n on the Table 2 families.
    Per instance: P = the fraction of the short run's replicas whose best energy reaches
    the optimum (exhaustive for n <= 16 -- computed by the oracle's brute force and stored
    under tests/golden --, planted for nae_3_sat, else the best of the short run and of a
    run with 4x the replicas and 4x the iterations); T1 = device time of the short run,
    timed alone on the first instance of each (family, n), divided by its replicas (the
    replicas run concurrently: the time one run costs at full occupancy).  Instances run
    w["streams"] at a time on their own streams.  Reported per (family, n): the median
    TTS99 over instances (null when P = 0 for at least half of them), the number of
    instances with P > 0 and the mean P.  GAHMC (exact zero crossings, phia_gahmc) runs on
    the same instances of one family for the Sec. 3.2 ablation, with its own T1."""
    import torch
    from paper_2407_10205_gb300 import phia, instances as ins, schedules
    fams = args.tts_families.split(",") if args.tts_families else sorted(ins.FAMILIES)
    sizes = tuple(int(t) for t in args.tts_sizes.split(",")) if args.tts_sizes else w["sizes"]
    n_inst = args.tts_instances or w["instances"]
    jump = args.tts_jump or w["jump"]          # None: schedules.default_jump(n)
    optima = _tts_optima()
    S = w["streams"]
    streams = [torch.cuda.Stream() for _ in range(S)]
    R, Rr = w["replicas"], w["ref_replicas"]
    t_start = time.perf_counter()
    rows = []
    optimum_of = {}

    fam_sched = w.get("family_schedule", {})

    def schedule_of(fam, d, own=True):
        b0, b1, eps, gamma, refresh = tts_schedule_params(w, args, fam, d, own)
        return phia.schedule(b0, b1, eps, gamma, refresh=refresh)

    for fam in fams:
        for n in sizes:
            # runs lengthen faster than n past 256 spins (n = 1024: 32x the n <= 128 length)
            T = (args.tts_iters or w["iterations"]) * max(1, n // 128) * max(1, n // 256)
            insts = [ins.family_instance(fam, n, ins.tts_seed(fam, n, k)) for k in range(n_inst)]
            # T1: the short run alone
            d0 = insts[0]
            with phia.Annealer(d0.k, d0.kh, frac_bits=d0.frac_bits, path=phia.PATH_TC) as A:
                sch = schedule_of(fam, d0)
                phia.anneal(A.h, sch, R, T, 1)
                phia.sync(A.h)
                phia.anneal(A.h, sch, R, T, 1)
                t1 = phia.stats_get(A.h).device_ms * 1e-3 / R
            ps, opt_src = [], set()
            for g0 in range(0, n_inst, S):
                group = list(range(g0, min(n_inst, g0 + S)))
                hs = []
                for j, k in enumerate(group):
                    d = insts[k]
                    A = phia.Annealer(d.k, d.kh, frac_bits=d.frac_bits, path=phia.PATH_TC,
                                      stream=streams[j].cuda_stream)
                    sch = schedule_of(fam, d)
                    known = None
                    if n <= 16:
                        known = optima[f"{fam}/{n}"][k]
                    elif isinstance(d, ins.Planted):
                        known = d.optimum_k
                    phia.anneal(A.h, sch, R, T, 7_777 + k)
                    hs.append((A, sch, known, k))
                res = []
                for A, sch, known, k in hs:
                    be, _, _, _ = phia.replica_results(A.h, R, n)
                    res.append(be)
                # the reference: a longer run under the family's schedule and, for a family
                # with a schedule of its own, one under the heuristic as well
                refs = [None] * len(hs)
                for own in ((True, False) if fam in fam_sched else (True,)):
                    for (A, sch, known, k) in hs:
                        if known is None:
                            rs = sch if own else schedule_of(fam, insts[k], own=False)
                            phia.anneal(A.h, rs, Rr, T * w["ref_factor"], 1 + k)
                    for j, (A, sch, known, k) in enumerate(hs):
                        if known is None:
                            e = int(phia.best(A.h, n)[0])
                            refs[j] = e if refs[j] is None else min(refs[j], e)
                for j, (A, sch, known, k) in enumerate(hs):
                    be = res[j]
                    if known is None:
                        opt = min(refs[j], int(be.min()))
                        opt_src.add("best found")
                    else:
                        opt = int(known)
                        opt_src.add("exhaustive" if n <= 16 else "planted")
                        assert be.min() >= opt, "an energy below the exact optimum"
                    ps.append(float(np.mean(be <= opt)))
                    optimum_of[(fam, n, k)] = opt
                    A.close()
            ttss = [tts99(t1, p) for p in ps]
            med = float(np.median(ttss))
            rows.append({"family": fam, "n": n, "iterations": T, "instances": n_inst,
                         "p_mean": float(np.mean(ps)), "p_median": float(np.median(ps)),
                         "solved_instances": int(np.sum(np.array(ps) > 0)), "t1_s": t1,
                         "tts99_s_median": med if math.isfinite(med) else None,
                         "optimum": "/".join(sorted(opt_src))})
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    # GAHMC ablation (Sec. 3.2) on one family's instances, against the same per-instance
    # optimum as PHIA (lowered where GAHMC finds better; such instances are counted)
    gam = []
    gfam = w["gahmc_family"]
    gsizes = [m for m in w["gahmc_sizes"] if m in sizes] if gfam in fams else []
    for n in gsizes:
        K = w["gahmc_trajectories"] * max(1, n // 32)
        ps, t1, better = [], None, 0
        phia_row = next((r for r in rows if r["family"] == gfam and r["n"] == n), None)
        for k in range(n_inst):
            d = ins.family_instance(gfam, n, ins.tts_seed(gfam, n, k))
            b0, b1, _, _, _ = schedules.suggest_schedule(d, jump=jump)
            gs = phia.gahmc_schedule(b0, b1, math.pi / 2)
            with phia.Annealer(d.k, d.kh, frac_bits=d.frac_bits, path=phia.PATH_TC) as A:
                phia.gahmc(A.h, gs, R, K, 5_555 + k)
                if t1 is None:
                    phia.gahmc(A.h, gs, R, K, 5_555 + k)
                    t1 = phia.stats_get(A.h).device_ms * 1e-3 / R
                be, _, _, _ = phia.replica_results(A.h, R, n)
            opt = optimum_of[(gfam, n, k)]
            if n > 16 and be.min() < opt:
                better += 1
                opt = int(be.min())
            ps.append(float(np.mean(be <= opt)))
        med = float(np.median([tts99(t1, p) for p in ps]))
        row = {"family": gfam, "n": n, "trajectories": K, "travel": "pi/2", "p_mean": float(np.mean(ps)),
               "solved_instances": int(np.sum(np.array(ps) > 0)), "t1_s": t1,
               "tts99_s_median": med if math.isfinite(med) else None,
               "instances_where_gahmc_found_lower": better}
        if phia_row and phia_row["tts99_s_median"] and row["tts99_s_median"]:
            row["tts_ratio_gahmc_over_phia"] = row["tts99_s_median"] / phia_row["tts99_s_median"]
        gam.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)
    line = {"metric": "TTS99 (median over instances; null = not reached)",
            "value": rows[-1]["tts99_s_median"] if rows else None, "unit": "s",
            "n_gpus": 1, "higher_is_better": False, "data": "synthetic", "dtype": "fp32",
            "config": {"workload": w["name"], "replicas": R,
                       "jump": jump if jump else "6 max(1, sqrt(n / 128)) (schedules.default_jump)",
                       "reference": f"best of {Rr} replicas x {w['ref_factor']} times the iterations",
                       "eps": args.tts_eps or "heuristic", "gamma": args.tts_gamma or "heuristic",
                       "refresh": args.tts_refresh or "heuristic", "family_schedule": w.get("family_schedule", {})},
            "table": rows, "gahmc": gam, "wall_s": time.perf_counter() - t_start}
    print(json.dumps(line))
    return 0


def _tuned_opts(tune):
    """Annealer options naming the kernel an autotune result chose."""
    if tune.tc_kernel == 2:
        return {"tc_kernel": 2, "large_variant": tune.large_variant}
    return {"tc_kernel": tune.tc_kernel, "tile_replicas": tune.tile_replicas, "coupling_mem": tune.coupling_mem}


def measure_dense(args, w, rank=0, world=1, local=0, with_cpu=True, dist=None):
    """One dense workload on the tensor-core path: the autotuned kernel timed over
    args.steps whole runs (after args.warmup), e2e through the C ABI, the FP32 comparator
    and (optionally) the oracle's CPU baseline.  Returns the JSON line's fields."""
    import torch
    from paper_2407_10205_gb300 import phia
    d = _instance(w)
    N, R, T = w["N"], w["replicas"], w["iterations"]
    sched = phia.schedule(w["beta0"], w["beta1"], w["eps"], w["gamma"], refresh=w["refresh"])
    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    seed = w["run_seed"] + rank * 1_000_003     # each rank anneals its own replicas

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    with phia.Annealer(d.k, d.kh, path=phia.PATH_TC, stream=stream.cuda_stream) as A:
        tune = phia.autotune(A.h, sched, R, probe_iters=min(T, 200))   # kernel variant for (N, R)
        cs = ClockSampler(local).start()
        for _ in range(args.warmup):
            flush.fill_(0.0)                          # the flush kernel is loaded before timing
            phia.anneal(A.h, sched, R, T, seed)
            phia.sync(A.h)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        barrier()
        with cs:
            t_wall = time.perf_counter()
            for k in range(args.steps):
                flush.fill_(float(k))                     # L2 flush between timed steps
                torch.cuda.current_stream().synchronize()
                ev[k][0].record(stream)
                phia.anneal(A.h, sched, R, T, seed)
                ev[k][1].record(stream)
            barrier()
            t_wall = time.perf_counter() - t_wall
        st = phia.stats_get(A.h)
        launches = args.steps * st.kernel_launches
        ms = [a.elapsed_time(b) for a, b in ev]
        kernel_ms = float(st.device_ms)
        best_e, _ = phia.best(A.h, N)

    ms_per_step = sum(ms) / len(ms)
    if world > 1:
        t = torch.tensor([ms_per_step], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_per_step = float(t.item())
    su_step = R * N * T
    value = world * su_step / (ms_per_step * 1e-3)

    # e2e: public C ABI from host buffers, host<->device copies inside the timed region, on
    # the kernel the autotuner chose (named explicitly: a new automatic handle would not take
    # a cooperative variant)
    e2e_ms = []
    for k in range(max(2, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with phia.Annealer(d.k, d.kh, path=phia.PATH_TC, stream=stream.cuda_stream, **_tuned_opts(tune)) as B:
            phia.anneal(B.h, sched, R, T, seed)
            e, spins = phia.best(B.h, N)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_step = statistics.median(e2e_ms)
    h2d = N * N + 4 * N
    d2h = 3 * 8 * R + 4 + 4 * ((N + 31) // 32) + 8

    # comparator: the plain FP32 per-instance GPU path, same instance and seeds; long runs
    # are timed on their first cmp_iters iterations and scaled (labelled).
    Tc = min(T, w["cmp_iters"])
    with phia.Annealer(d.k, d.kh, path=phia.PATH_FP32, stream=stream.cuda_stream) as C:
        phia.anneal(C.h, sched, R, Tc, seed)
        phia.sync(C.h)
        cmp_ms = []
        for _ in range(2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            phia.anneal(C.h, sched, R, Tc, seed)
            e1.record(stream)
            stream.synchronize()
            cmp_ms.append(e0.elapsed_time(e1))
        cmp_best, _ = phia.best(C.h, N)
    cmp_run_ms = min(cmp_ms) * T / Tc
    cmp_value = su_step / (cmp_run_ms * 1e-3)

    peaks, src = _peaks()
    probe = mma_probe(phia) if with_cpu else None
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "fp32", "data": "synthetic",
        "config": {"workload": w["name"], "N": N, "replicas": R, "iterations": T, "path": "tc",
                   "tc_kernel": {1: "resident tcgen05", 2: "per-iteration tcgen05", 3: "resident int8 mma.sync",
                                 4: "resident incremental field"}.get(st.tc_kernel, str(st.tc_kernel)),
                   "autotune": {"tc_kernel": tune.tc_kernel, "tile_replicas": tune.tile_replicas,
                                "coupling_mem": tune.coupling_mem, "candidates": tune.candidates,
                                "best_us_per_iter": tune.best_us_per_iter,
                                "worst_us_per_iter": tune.worst_us_per_iter, "large_variant": tune.large_variant},
                   "field_operand": ("e4m3" if st.operand == 1 else "bf16")
                   + " (exact re-encoding of int8 k), fp32 accumulation of integer products",
                   "state": "fp32 x, v", "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": f"replicas sharded over {world} GPU(s), no collective"},
        "e2e": {"value": su_step / (e2e_step * 1e-3), "unit": METRIC, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_step},
        "roofline": _roofline(w, kernel_ms, st, peaks, src, probe, tune.large_variant),
        "gpu_launches": launches,
        "clocks": cs.summary(),
        "comparator": {"path": "fp32 per-instance, one launch per step", "value": cmp_value, "unit": METRIC,
                       "ms_per_run": cmp_run_ms,
                       "timed_iterations": Tc, "scaled": Tc != T,
                       "best_energy_k_of_timed_iterations": int(cmp_best)},
        "best_energy_k": int(best_e),
        "us_per_iteration": ms_per_step * 1e3 / T,
        "wall_s_timed": t_wall,
    }
    if probe:
        line["tensor_probe"] = probe
    if with_cpu and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w)
    return line


def _summary(line, keys=("value", "unit", "ms_per_step", "roofline", "e2e", "comparator", "clocks",
                         "gpu_launches", "serving", "config")):
    return {k: line[k] for k in keys if k in line}


def run_ours(args):
    import torch
    import torch.distributed as dist

    rank, world, local = _dist()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2407_10205_gb300 import phia
    phia.load()
    w = WORKLOADS[args.workload]
    if w["kind"] == "batch":
        print(json.dumps(measure_batch(args, w)))
        return 0
    if w["kind"] == "tts":
        return run_tts(args, w)
    if w["kind"] == "serving":
        w = dict(w)
        if args.max_inflight:
            w["max_inflight"] = args.max_inflight
        if args.chunk_iters:
            w["chunk_iters"] = args.chunk_iters
        print(json.dumps(measure_serving(args, w)))
        return 0
    line = measure_dense(args, w, rank, world, local, dist=dist)
    if rank != 0:
        return 0
    if world == 1 and not args.no_extras and args.workload == "dense2000":
        # the other workloads of the benchmark set, one line each under "also"
        also = {}
        for name in ("dense200",):
            also[name] = _summary(measure_dense(args, WORKLOADS[name], with_cpu=False))
        also["batched_er"] = _summary(measure_batch(args, WORKLOADS["batched_er"], light=True))
        sv = dict(WORKLOADS["serving"])
        sv["requests"] = 200
        a2 = argparse.Namespace(**vars(args))
        a2.no_comparator = True
        also["serving"] = _summary(measure_serving(a2, sv))
        line["also"] = also
    print(json.dumps(line))
    return 0


def main():
    if len(sys.argv) == 3 and sys.argv[1] == "--clock-poll":
        return _nvml_poll(sys.argv[2], CLOCK_POLL_MS)
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="dense2000", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tile-replicas", type=int, default=0, help="tensor-core replicas per CTA (0 = auto)")
    ap.add_argument("--coupling-mem", type=int, default=0, help="tensor-core: 1 = J in shared, 2 = in tensor memory")
    ap.add_argument("--tc-kernel", type=int, default=0, help="tensor-core kernel: 1 tcgen05 resident, 2 per-iteration, 3 int8 mma.sync")
    ap.add_argument("--max-inflight", type=int, default=0, help="serving: request slots (0 = the workload's)")
    ap.add_argument("--chunk-iters", type=int, default=0, help="serving: iterations per chunk (0 = the workload's)")
    ap.add_argument("--no-comparator", action="store_true", help="serving: skip the FP32 comparator runs")
    ap.add_argument("--tts-sizes", default="", help="tts: comma-separated sizes (default: the workload's)")
    ap.add_argument("--tts-families", default="", help="tts: comma-separated families (default: all seven)")
    ap.add_argument("--tts-instances", type=int, default=0, help="tts: instances per (family, n)")
    ap.add_argument("--tts-jump", type=float, default=0.0, help="tts: schedule heuristic's final jump")
    ap.add_argument("--tts-iters", type=int, default=0, help="tts: iterations per run at n <= 128 (0 = the workload's)")
    ap.add_argument("--tts-eps", type=float, default=0.0, help="tts: step size eps (0 = the schedule heuristic's)")
    ap.add_argument("--tts-gamma", type=float, default=0.0, help="tts: gamma of Eq. 7 (0 = the heuristic's)")
    ap.add_argument("--tts-refresh", type=int, default=0, help="tts: iterations per trajectory (0 = the heuristic's)")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload: skip the other workloads reported under 'also'")
    ap.add_argument("--profile-only", action="store_true",
                    help="run warmup + steps anneals of the tensor-core path and nothing else (for ncu)")
    ap.add_argument("--large-variant", type=int, default=0, help="per-iteration kernel variant (0 = auto)")
    ap.add_argument("--profile-iters", type=int, default=0, help="profile-only: iterations per run (0 = the workload's)")
    ap.add_argument("--profile-gahmc", action="store_true",
                    help="profile-only: vanilla GAHMC (phia_gahmc) on an n = 256 SK instance, 1024 replicas")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_only:
        return run_profile(args)
    return run_ours(args)


def run_profile(args):
    import torch
    from paper_2407_10205_gb300 import phia
    phia.load()
    w = WORKLOADS[args.workload]
    iters = args.profile_iters or w["iterations"]
    if args.profile_gahmc:
        from paper_2407_10205_gb300 import instances as ins
        d = ins.sk_pm1(256, 3)
        with phia.Annealer(d.k, d.kh, path=phia.PATH_TC) as A:
            for _ in range(args.warmup + args.steps):
                phia.gahmc(A.h, phia.gahmc_schedule(0.02, 0.3, math.pi / 2), 1024, args.profile_iters or 200, 1)
                phia.sync(A.h)
            st = phia.stats_get(A.h)
        print(json.dumps({"profile_only": True, "device_ms_last": st.device_ms, "launches_per_run": st.kernel_launches}))
        return 0
    if w["kind"] == "batch":
        from paper_2407_10205_gb300 import instances as ins
        sched = phia.schedule(w["beta0"], w["beta1"], w["eps"], w["gamma"], refresh=w["refresh"])
        with phia.Batch(ins.batched_er(w["count"], w["seed"]), csr_mode=2) as B:   # one launch per iteration
            for _ in range(args.warmup + args.steps):
                B.anneal(sched, w["replicas"], iters, w["run_seed"])
                B.sync()
            st = B.stats()
        print(json.dumps({"profile_only": True, "device_ms_last": st.device_ms, "launches_per_run": st.kernel_launches}))
        return 0
    d = _instance(w)
    sched = phia.schedule(w["beta0"], w["beta1"], w["eps"], w["gamma"], refresh=w["refresh"])
    with phia.Annealer(d.k, d.kh, path=phia.PATH_TC, tile_replicas=args.tile_replicas,
                       coupling_mem=args.coupling_mem, tc_kernel=args.tc_kernel,
                       large_variant=args.large_variant) as A:
        if args.tile_replicas == 0 and args.tc_kernel == 0:
            phia.autotune(A.h, sched, w["replicas"], probe_iters=min(w["iterations"], 200))   # as bench.py does
        for _ in range(args.warmup + args.steps):
            phia.anneal(A.h, sched, w["replicas"], iters, w["run_seed"])
            phia.sync(A.h)
        st = phia.stats_get(A.h)
    torch.cuda.synchronize()
    print(json.dumps({"profile_only": True, "device_ms_last": st.device_ms, "launches_per_run": st.kernel_launches}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
