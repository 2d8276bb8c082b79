// noalloc.cu -- phia_run_noalloc: the per-iteration tensor-core path with every piece of
// scratch memory taken from one fixed array compiled into the library, for callers that
// cannot allocate device memory (see include/phia.h for who they are and the limits).
#include <cstdio>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/phia.h"
#include "phia_internal.h"

namespace phia {
namespace {

// Scratch of phia_run_noalloc.  Every GPU on which the library's module is loaded holds
// this array until the process exits; all calls share it.
constexpr size_t kScratchBytes = (size_t)64 << 20;
static __device__ __align__(256) uint8_t g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 128;
uint8_t *g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of the scratch array on `dev` (the current device), looked up once per
// device.  The name g_noalloc_scratch is only a host-side handle: kernels must be given
// this address, never the symbol itself.
int scratch_address(int dev, uint8_t **out) {
    if (dev < 0 || dev >= kMaxDevices) return set_last_error(PHIA_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            char msg[256];
            snprintf(msg, sizeof msg, "cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(e));
            return set_last_error(PHIA_ECUDA, msg);
        }
        g_scratch_ptr[dev] = static_cast<uint8_t *>(p);
    }
    *out = g_scratch_ptr[dev];
    return PHIA_OK;
}

__global__ void noalloc_reset_records(int R, int W, int64_t *best_e, int64_t *best_step, int64_t *hit,
                                      uint32_t *bits) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < R) {
        best_e[idx] = INT64_MAX;
        best_step[idx] = -1;
        hit[idx] = -1;
    }
    if (idx < (int64_t)R * W) bits[idx] = 0u;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace
}  // namespace phia

using namespace phia;

extern "C" int phia_run_noalloc(const int8_t *J_k, const int32_t *h_k, int32_t N, int32_t frac_bits,
                                int32_t operand, const phia_schedule *sched, int32_t replicas, int64_t t0,
                                int64_t steps, int64_t total_steps, uint64_t seed, uint32_t instance_id, float *x,
                                float *v, int64_t *best_energy_k, int64_t *best_step, int64_t *hit_step,
                                uint32_t *best_bits, int32_t reset_best, void *stream) {
    if (!J_k || !h_k || !sched || !x || !v || !best_energy_k || !best_step || !hit_step || !best_bits)
        return set_last_error(PHIA_EINVAL, "phia_run_noalloc: a required pointer is NULL");
    if (N < 1 || replicas < 1 || steps < 1 || t0 < 0 || total_steps < t0 + steps)
        return set_last_error(PHIA_EINVAL, "phia_run_noalloc: need N, replicas, steps >= 1 and t0 + steps <= total");
    if (total_steps > ((int64_t)1 << 31)) return set_last_error(PHIA_ERANGE, "phia_run_noalloc: total_steps >= 2^31");
    if (frac_bits < 0 || frac_bits > 30) return set_last_error(PHIA_EINVAL, "phia_run_noalloc: frac_bits not in [0, 30]");
    if (operand != PHIA_OP_E4M3 && operand != PHIA_OP_BF16 && operand != PHIA_OP_AUTO)
        return set_last_error(PHIA_EINVAL, "phia_run_noalloc: unknown operand");
    if (!(sched->eps > 0.0f) || !(sched->gamma > 0.0f) || sched->refresh < 0 || (sched->deriv != 0 && sched->deriv != 1))
        return set_last_error(PHIA_EINVAL, "phia_run_noalloc: invalid schedule");
    const int op = operand == PHIA_OP_E4M3 ? kOpE4M3 : kOpBF16;   // AUTO: bf16, exact for every int8 k

    // Scratch layout: operand J, 4 spin buffers, energy sums, flags, run counters, and the
    // working x, v in the kernel's interleaved layout (the caller's x, v are read at the
    // start and written at the end).
    const int Mpad = round_up(N, 128), Kbytes = large_kbytes(N, op), Rpad = large_rpad(replicas);
    const size_t off_jop = 0;
    const size_t off_s = off_jop + align256((size_t)Mpad * Kbytes);
    const size_t off_e = off_s + align256((size_t)4 * Rpad * Kbytes);
    const size_t off_f = off_e + align256((size_t)2 * Rpad * sizeof(int64_t));
    const size_t off_c = off_f + align256((size_t)2 * Rpad);
    const size_t off_x = off_c + 256;
    const size_t off_v = off_x + align256((size_t)Rpad * Mpad * 4);
    const size_t need = off_v + align256((size_t)Rpad * Mpad * 4);
    if (need > kScratchBytes) {
        char msg[256];
        snprintf(msg, sizeof msg,
                 "phia_run_noalloc: N = %d and %d replicas need %zu bytes of scratch; the fixed scratch holds %zu "
                 "(e.g. N <= 2000 with e4m3 and up to 2048 replicas)",
                 N, replicas, need, kScratchBytes);
        return set_last_error(PHIA_ERANGE, msg);
    }

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return set_last_error(PHIA_ECUDA, "phia_run_noalloc: no current device");
    uint8_t *base = nullptr;
    int rc = scratch_address(dev, &base);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    auto cuda_fail = [&](cudaError_t e) {
        char msg[256];
        snprintf(msg, sizeof msg, "phia_run_noalloc: %s", cudaGetErrorString(e));
        return set_last_error(PHIA_ECUDA, msg);
    };
    // The array keeps the previous call's contents: clear what must start at zero (the
    // spin buffers' padding, the energy sums, the flags and the counters).
    cudaError_t e = cudaMemsetAsync(base + off_s, 0, off_x - off_s, st);
    if (e != cudaSuccess) return cuda_fail(e);
    e = launch_convert_operand(J_k, N, base + off_jop, Mpad, Kbytes, op, st);
    if (e != cudaSuccess) return cuda_fail(e);
    const int W = (N + 31) / 32;
    if (reset_best) {
        const int64_t n = (int64_t)replicas * W > replicas ? (int64_t)replicas * W : replicas;
        noalloc_reset_records<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(replicas, W, best_energy_k, best_step,
                                                                         hit_step, best_bits);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e);
    }
    unsigned long long *counters = reinterpret_cast<unsigned long long *>(base + off_c);
    RunArgs a;
    memset(&a, 0, sizeof a);
    a.N = N;
    a.frac_bits = frac_bits;
    a.Jk = J_k;
    a.hk = h_k;
    a.R = replicas;
    a.t0 = t0; a.nsteps = steps; a.T_total = total_steps;
    a.beta0 = sched->beta0; a.beta1 = sched->beta1; a.eps = sched->eps; a.gamma = sched->gamma;
    a.q = ldexpf(1.0f, -frac_bits);
    a.refresh = sched->refresh;
    a.deriv = sched->deriv;
    a.seed = seed;
    a.inst = instance_id;
    a.x_in = x; a.v_in = v; a.x_out = x; a.v_out = v;
    a.best_e = best_energy_k; a.best_step = best_step; a.hit_step = hit_step; a.best_bits = best_bits; a.W = W;
    a.has_target = sched->has_target; a.stop_at_target = sched->stop_at_target; a.target = sched->target_k;
    a.min_hit = counters;
    a.replica_iters = counters + 1;
    a.err = reinterpret_cast<int32_t *>(counters + 2);
    e = cudaMemsetAsync(counters, 0xFF, 8, st);
    if (e != cudaSuccess) return cuda_fail(e);
    LargeBuffers B;
    B.Jop = base + off_jop;
    B.S = base + off_s;
    B.Epart = reinterpret_cast<int64_t *>(base + off_e);
    B.flags = reinterpret_cast<int8_t *>(base + off_f);
    B.ctl = reinterpret_cast<IterCtl *>(base + off_c + 64);
    B.graphs = nullptr;   // a graph would be an allocation
    B.X = reinterpret_cast<float *>(base + off_x);
    B.V = reinterpret_cast<float *>(base + off_v);
    B.Kbytes = Kbytes; B.Mpad = Mpad; B.Rpad = Rpad;
    int launches = 0;
    e = launch_tc_large(B, a, op, st, &launches);
    if (e != cudaSuccess) return cuda_fail(e);
    // Synchronous: report a bounded device wait that expired.
    int32_t err = 0;
    e = cudaMemcpyAsync(&err, a.err, sizeof err, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e);
    if (err) return set_last_error(PHIA_ETIMEOUT, "phia_run_noalloc: a bounded device wait expired");
    return PHIA_OK;
}
