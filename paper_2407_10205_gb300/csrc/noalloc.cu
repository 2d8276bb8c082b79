// noalloc.cu -- phia_run_noalloc: the per-iteration tensor-core path with every piece of
// scratch memory taken from one fixed array compiled into the library, for callers that
// cannot allocate device memory (see include/phia.h for who they are and the limits).
#include <algorithm>
#include <climits>
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

namespace phia {
namespace {

// Scratch layout for N spins, `replicas` replicas and operand `op`: a 256-byte control
// region (run counters at 0, the iteration control at 64, the instance-check results at
// 128), then the operand J, 4 spin buffers, energy sums, flags, and the working x, v in
// the per-iteration kernel's interleaved layout.
struct NoallocLayout {
    int Mpad, Kbytes, Rpad;
    size_t off_jop, off_s, off_e, off_f, off_x, off_v, need;
};

NoallocLayout noalloc_layout(int N, int replicas, int op) {
    NoallocLayout L;
    L.Mpad = round_up(N, 128);
    L.Kbytes = large_kbytes(N, op);
    L.Rpad = large_rpad(replicas);
    L.off_jop = 256;
    L.off_s = L.off_jop + align256((size_t)L.Mpad * L.Kbytes);
    L.off_e = L.off_s + align256((size_t)4 * L.Rpad * L.Kbytes);
    L.off_f = L.off_e + align256((size_t)2 * L.Rpad * sizeof(int64_t));
    L.off_x = L.off_f + align256((size_t)2 * L.Rpad);
    L.off_v = L.off_x + align256((size_t)L.Rpad * L.Mpad * 4);
    L.need = L.off_v + align256((size_t)L.Rpad * L.Mpad * 4);
    return L;
}

}  // namespace
}  // namespace phia

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
    if (!(sched->eps > 0.0f) || !(sched->gamma > 0.0f) || !(sched->beta0 >= 0.0f) || !(sched->beta1 >= 0.0f) ||
        sched->refresh < 0 || (sched->deriv != 0 && sched->deriv != 1) || sched->reserved != 0)
        return set_last_error(PHIA_EINVAL, "phia_run_noalloc: invalid schedule");
    if (sched->accept_test != 0)
        return set_last_error(PHIA_ENOTSUP, "phia_run_noalloc: schedule.accept_test = 1 is not supported here");
    // A size too large for the scratch whatever the operand is refused before any device work.
    if (noalloc_layout(N, replicas, operand == PHIA_OP_BF16 ? kOpBF16 : kOpE4M3).need > kScratchBytes) {
        char msg[320];
        const int op = operand == PHIA_OP_BF16 ? kOpBF16 : kOpE4M3;
        int rmax = 0;
        while (noalloc_layout(N, rmax + 256, op).need <= kScratchBytes) rmax += 256;
        snprintf(msg, sizeof msg,
                 "phia_run_noalloc: N = %d and %d replicas need %zu bytes of scratch; the fixed scratch holds %zu "
                 "(with this N and the %s operand at most %d replicas fit)",
                 N, replicas, noalloc_layout(N, replicas, op).need, kScratchBytes, op == kOpBF16 ? "bf16" : "e4m3",
                 rmax);
        return set_last_error(PHIA_ERANGE, msg);
    }

    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return set_last_error(PHIA_ECUDA, "phia_run_noalloc: no current device");
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return set_last_error(PHIA_ECUDA, "phia_run_noalloc: device query failed");
    uint8_t *base = nullptr;
    int rc = scratch_address(dev, &base);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    auto cuda_fail = [&](cudaError_t e) {
        char msg[256];
        snprintf(msg, sizeof msg, "phia_run_noalloc: %s", cudaGetErrorString(e));
        return set_last_error(PHIA_ECUDA, msg);
    };

    // The instance checks of phia_create, on the device, into the control region: symmetry,
    // zero diagonal, |h_k| < 2^24 and max |k| (which decides whether e4m3 is exact).
    unsigned long long *res = reinterpret_cast<unsigned long long *>(base + 128);
    cudaError_t e = cudaMemsetAsync(res, 0xFF, 3 * sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(res + 3, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) {
        const int64_t total = (int64_t)N * N;
        const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, (int64_t)sms * 8));
        e = launch_check_dense(J_k, h_k, N, res, blocks, st);
    }
    unsigned long long got[4] = {0, 0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(got, res, sizeof got, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e);
    char msg[256];
    if (got[2] != ULLONG_MAX) {
        snprintf(msg, sizeof msg, "phia_run_noalloc: |h_k[%llu]| >= 2^24", got[2]);
        return set_last_error(PHIA_ERANGE, msg);
    }
    if (got[1] != ULLONG_MAX) {
        snprintf(msg, sizeof msg, "phia_run_noalloc: nonzero diagonal J_k[%llu][%llu]", got[1], got[1]);
        return set_last_error(PHIA_EINVAL, msg);
    }
    if (got[0] != ULLONG_MAX) {
        snprintf(msg, sizeof msg, "phia_run_noalloc: J_k is not symmetric at (%llu, %llu)",
                 got[0] / (unsigned long long)N, got[0] % (unsigned long long)N);
        return set_last_error(PHIA_EINVAL, msg);
    }
    const int max_abs = (int)got[3];
    if (operand == PHIA_OP_E4M3 && max_abs > 16) {
        snprintf(msg, sizeof msg, "phia_run_noalloc: max |k| = %d is not exact in e4m3 (needs <= 16)", max_abs);
        return set_last_error(PHIA_ERANGE, msg);
    }
    // AUTO as in phia_create: e4m3 when every |k| <= 16, else bf16 (exact for every int8 k).
    const int op = operand == PHIA_OP_BF16 || (operand == PHIA_OP_AUTO && max_abs > 16) ? kOpBF16 : kOpE4M3;
    const NoallocLayout Ly = noalloc_layout(N, replicas, op);
    if (Ly.need > kScratchBytes) {
        int rmax = 0;
        while (noalloc_layout(N, rmax + 256, op).need <= kScratchBytes) rmax += 256;
        snprintf(msg, sizeof msg,
                 "phia_run_noalloc: N = %d and %d replicas need %zu bytes of scratch with the bf16 operand; the "
                 "fixed scratch holds %zu (at most %d replicas fit)", N, replicas, Ly.need, kScratchBytes, rmax);
        return set_last_error(PHIA_ERANGE, msg);
    }

    // The array keeps the previous call's contents: clear what must start at zero (the run
    // counters, the spin buffers' padding, the energy sums and the flags).
    e = cudaMemsetAsync(base, 0, 64, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + Ly.off_s, 0, Ly.off_x - Ly.off_s, st);
    if (e == cudaSuccess) e = launch_convert_operand(J_k, N, base + Ly.off_jop, Ly.Mpad, Ly.Kbytes, op, st);
    if (e != cudaSuccess) return cuda_fail(e);
    const int W = (N + 31) / 32;
    if (reset_best) {
        const int64_t n = (int64_t)replicas * W > replicas ? (int64_t)replicas * W : replicas;
        noalloc_reset_records<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(replicas, W, best_energy_k, best_step,
                                                                         hit_step, best_bits);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e);
    }
    unsigned long long *counters = reinterpret_cast<unsigned long long *>(base);
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
    B.Jop = base + Ly.off_jop;
    B.S = base + Ly.off_s;
    B.Epart = reinterpret_cast<int64_t *>(base + Ly.off_e);
    B.flags = reinterpret_cast<int8_t *>(base + Ly.off_f);
    B.ctl = reinterpret_cast<IterCtl *>(base + 64);
    B.graphs = nullptr;   // a graph would be an allocation
    B.ready = nullptr;    // no overlapped variant here
    B.sbits = nullptr;
    B.X = reinterpret_cast<float *>(base + Ly.off_x);
    B.V = reinterpret_cast<float *>(base + Ly.off_v);
    B.Kbytes = Ly.Kbytes; B.Mpad = Ly.Mpad; B.Rpad = Ly.Rpad;
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
