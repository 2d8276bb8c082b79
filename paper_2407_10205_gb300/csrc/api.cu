// api.cu -- the C ABI of include/phia.h and the host runtime behind it: instance
// validation and upload, path and operand selection, per-replica state, run
// launch, records and results.
#include <algorithm>
#include <climits>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/phia.h"
#include "device_common.cuh"
#include "phia_internal.h"

using namespace phia;

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CU(call)                                                                                \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) return fail(PHIA_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

__global__ void reset_records_kernel(int R, int W, int64_t *best_e, int64_t *best_step, int64_t *hit,
                                     uint32_t *bits, uint64_t *hit_ns, uint64_t *start_ns) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < R) {
        best_e[idx] = LLONG_MAX;
        best_step[idx] = -1;
        hit[idx] = -1;
        hit_ns[idx] = 0;
    }
    if (idx < (int64_t)R * W) bits[idx] = 0u;
    if (idx == 0) *start_ns = phia::globaltimer_ns();   // the run's start on the device clock
}

// J = k q in FP32 for the FP32 path, from the device copy of k.
__global__ void k_to_f32_kernel(const int8_t *k, float *jf, int64_t n, float q) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        jf[e] = (float)k[e] * q;
}

}  // namespace

namespace phia {
// Sets the calling thread's phia_last_error() message (for entry points in other files).
int set_last_error(int code, const char *msg) { return fail(code, "%s", msg); }
}  // namespace phia

struct phia_s {
    int device = 0;
    cudaStream_t stream = nullptr;
    int path = PHIA_PATH_TC;
    int op = 0;
    uint32_t inst = 0;
    int tile_rl = 0, coupling_mem = 0;
    phia_batch_s *batch = nullptr;      // CSR instances: a batch of one
    bool large = false;                 // tensor-core path through the per-iteration kernel
    bool imma = false;                  // tensor-core path through the int8 mma.sync resident kernel
    bool inc = false;                   // dense path through the incremental-field resident kernel
    void *d_Jop = nullptr;              // couplings in the operand encoding (per-iteration kernel)
    int Mpad = 0, Kbytes = 0;
    uint8_t *d_S = nullptr;             // [4][Rpad][Kbytes]
    int64_t *d_Epart = nullptr;
    int8_t *d_flags = nullptr;          // [4][Rpad] improved flags
    uint32_t *d_ready = nullptr;        // [2][Rpad/128] tile counters of the overlapped variant
    uint32_t *d_sbits = nullptr;        // [4][Rpad][Mpad/32] packed spins of the overlapped variant
    float *d_X = nullptr, *d_V = nullptr;
    int N = 0, frac_bits = 0, W = 0;
    bool csr = false;
    int64_t nnz = 0;
    int max_abs_k = 0;
    // instance on the device
    int8_t *d_Jk = nullptr;
    float *d_Jf = nullptr;
    int32_t *d_hk = nullptr;
    int32_t *d_rowptr = nullptr, *d_col = nullptr;
    int8_t *d_val = nullptr;
    // per-replica state
    int R_cap = 0, R_last = 0;
    bool cap_large = false;             // replica buffers allocated for the per-iteration kernel
    bool auto_tile = true;              // kernel variant chosen automatically (autotune cache)
    float *d_x = nullptr, *d_v = nullptr;
    int8_t *d_s0 = nullptr, *d_s1 = nullptr;
    int64_t *d_eacc = nullptr;
    int64_t *d_best_e = nullptr, *d_best_step = nullptr, *d_hit = nullptr;
    uint32_t *d_bits = nullptr;
    int64_t *d_prop = nullptr, *d_acc = nullptr;   // acceptance test counts per replica (Table 3, state 4)
    float *d_xstart = nullptr;          // FP32 path with the acceptance test: trajectory start positions
    int64_t *d_elast = nullptr, *d_estart = nullptr;
    float *d_xxs = nullptr, *d_vvs = nullptr;
    int32_t *d_hass = nullptr;
    uint64_t *d_hit_ns = nullptr;       // %globaltimer of each replica's first hit
    uint64_t *d_start_ns = nullptr;     // %globaltimer when the run's records were reset
    // run counters
    unsigned long long *d_min_hit = nullptr, *d_iters = nullptr;
    int32_t *d_err = nullptr;
    IterCtl *d_ctl = nullptr;           // iteration control of the per-iteration kernel
    StepGraphCache *graphs = nullptr;   // its step launches as replayable graphs
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    bool ran = false;
    int64_t last_steps = 0;
    int last_launches = 0;
    int last_stop = 0;
    int large_variant = 0;              // per-iteration kernel variant requested (0 = automatic)
    int tuned_variant = 0;              // the autotuner's choice for it
    bool tuned_coop = false;            // this handle's own autotune chose the cooperative variant
    int64_t wait_ns = 0;                // testing aid (phia_debug_wait): device wait bound, 0 = default
    int stall_producer = 0;             // testing aid: the per-iteration kernel's TMA producer issues nothing
};

namespace {

// A handle's device buffers come from one stream-ordered memory pool per device that
// keeps freed blocks (release threshold at its maximum).  Creating and destroying handles
// in a loop, as a caller with a new instance per request does, then costs neither
// cudaMalloc round trips nor the device-wide synchronisation of cudaFree; the pool keeps
// its peak size reserved for the process.
std::mutex g_pool_mu;
std::map<int, cudaMemPool_t> g_pools;

cudaError_t pool_alloc(void **ptr, size_t bytes, int device, cudaStream_t st) {
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_pool_mu);
        auto it = g_pools.find(device);
        if (it == g_pools.end()) {
            cudaMemPoolProps props;
            memset(&props, 0, sizeof props);
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = device;
            cudaError_t e = cudaMemPoolCreate(&pool, &props);
            if (e != cudaSuccess) return e;
            uint64_t keep = UINT64_MAX;
            e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
            if (e != cudaSuccess) return e;
            g_pools[device] = pool;
        } else {
            pool = it->second;
        }
    }
    return cudaMallocFromPoolAsync(ptr, std::max<size_t>(bytes, 16), pool, st);
}

void pool_free(void *ptr, cudaStream_t st) {
    if (ptr) cudaFreeAsync(ptr, st);
}

void free_replicas(phia_t *p) {
    for (void *b : {(void *)p->d_S, (void *)p->d_Epart, (void *)p->d_flags, (void *)p->d_ready, (void *)p->d_sbits,
                    (void *)p->d_X,
                    (void *)p->d_V,
                    (void *)p->d_x, (void *)p->d_v, (void *)p->d_s0, (void *)p->d_s1, (void *)p->d_eacc,
                    (void *)p->d_best_e, (void *)p->d_best_step, (void *)p->d_hit, (void *)p->d_bits,
                    (void *)p->d_hit_ns, (void *)p->d_prop, (void *)p->d_acc, (void *)p->d_xstart,
                    (void *)p->d_elast, (void *)p->d_estart, (void *)p->d_xxs, (void *)p->d_vvs, (void *)p->d_hass})
        pool_free(b, p->stream);
    p->d_prop = p->d_acc = nullptr; p->d_xstart = nullptr; p->d_elast = p->d_estart = nullptr;
    p->d_xxs = p->d_vvs = nullptr; p->d_hass = nullptr;
    p->d_S = nullptr; p->d_Epart = nullptr; p->d_flags = nullptr; p->d_ready = nullptr; p->d_sbits = nullptr;
    p->d_X = p->d_V = nullptr;
    p->d_x = p->d_v = nullptr; p->d_s0 = p->d_s1 = nullptr; p->d_eacc = nullptr;
    p->d_best_e = p->d_best_step = p->d_hit = nullptr; p->d_bits = nullptr; p->d_hit_ns = nullptr;
    p->R_cap = 0;
}

int ensure_replicas(phia_t *p, int R) {
    if (R <= p->R_cap && p->cap_large == p->large) return PHIA_OK;
    CU(cudaStreamSynchronize(p->stream));
    free_replicas(p);
    const size_t RN = (size_t)R * p->N;
    bool ok = true;
    auto al = [&](void **ptr, size_t bytes) {
        if (ok && pool_alloc(ptr, bytes, p->device, p->stream) != cudaSuccess) ok = false;
    };
    if (p->path == PHIA_PATH_FP32) {
        al((void **)&p->d_x, RN * 4); al((void **)&p->d_v, RN * 4);
        al((void **)&p->d_s0, RN); al((void **)&p->d_s1, RN);
        al((void **)&p->d_xstart, RN * 4);
        al((void **)&p->d_elast, (size_t)R * 8); al((void **)&p->d_estart, (size_t)R * 8);
        al((void **)&p->d_xxs, (size_t)R * 4); al((void **)&p->d_vvs, (size_t)R * 4);
        al((void **)&p->d_hass, (size_t)R * 4);
    }
    al((void **)&p->d_prop, (size_t)R * 8);
    al((void **)&p->d_acc, (size_t)R * 8);
    if (p->large) {
        const size_t Rp = (size_t)large_rpad_handle(R);
        al((void **)&p->d_S, 4 * Rp * p->Kbytes);
        al((void **)&p->d_Epart, 2 * Rp * 8);
        al((void **)&p->d_flags, 4 * Rp);
        al((void **)&p->d_ready, 2 * (Rp / 128) * sizeof(uint32_t));
        const size_t Mp = (size_t)round_up(p->N, 128);   // x, v in the interleaved [Rp/4][Mp][4] layout
        al((void **)&p->d_sbits, 4 * Rp * (Mp / 32) * sizeof(uint32_t));
        al((void **)&p->d_X, Rp * Mp * 4); al((void **)&p->d_V, Rp * Mp * 4);
    }
    al((void **)&p->d_eacc, (size_t)R * 8);
    al((void **)&p->d_best_e, (size_t)R * 8);
    al((void **)&p->d_best_step, (size_t)R * 8);
    al((void **)&p->d_hit, (size_t)R * 8);
    al((void **)&p->d_hit_ns, (size_t)R * 8);
    al((void **)&p->d_bits, (size_t)R * p->W * 4);
    if (!ok) {
        cudaGetLastError();
        free_replicas(p);
        return fail(PHIA_ENOMEM, "device allocation for %d replicas failed", R);
    }
    p->cap_large = p->large;
    CU(cudaMemsetAsync(p->d_eacc, 0, (size_t)R * 8, p->stream));
    if (p->large) {
        const size_t Rp = (size_t)large_rpad_handle(R);
        CU(cudaMemsetAsync(p->d_S, 0, 4 * Rp * p->Kbytes, p->stream));   // K and replica padding stay 0
        CU(cudaMemsetAsync(p->d_flags, 0, 4 * Rp, p->stream));
        CU(cudaMemsetAsync(p->d_Epart, 0, 2 * Rp * 8, p->stream));
    }
    p->R_cap = R;
    return PHIA_OK;
}

int reset_records(phia_t *p, int R) {
    const int64_t n = std::max<int64_t>(R, (int64_t)R * p->W);
    reset_records_kernel<<<(unsigned)((n + 255) / 256), 256, 0, p->stream>>>(R, p->W, p->d_best_e, p->d_best_step,
                                                                             p->d_hit, p->d_bits, p->d_hit_ns,
                                                                             p->d_start_ns);
    CU(cudaGetLastError());
    return PHIA_OK;
}

int check_sched(const phia_schedule *s) {
    if (!s) return fail(PHIA_EINVAL, "schedule is NULL");
    if (!(s->eps > 0.0f) || !(s->gamma > 0.0f)) return fail(PHIA_EINVAL, "eps and gamma must be > 0");
    if (!(s->beta0 >= 0.0f) || !(s->beta1 >= 0.0f)) return fail(PHIA_EINVAL, "beta0 and beta1 must be >= 0");
    if (s->refresh < 0) return fail(PHIA_EINVAL, "refresh must be >= 0");
    if (s->deriv != 0 && s->deriv != 1) return fail(PHIA_EINVAL, "schedule.deriv must be 0 or 1");
    if (s->accept_test != 0 && s->accept_test != 1) return fail(PHIA_EINVAL, "schedule.accept_test must be 0 or 1");
    if (s->reserved != 0) return fail(PHIA_EINVAL, "schedule.reserved must be 0");
    return PHIA_OK;
}

RunArgs base_args(phia_t *p, int R) {
    RunArgs a;
    memset(&a, 0, sizeof a);
    a.N = p->N;
    a.frac_bits = p->frac_bits;
    a.Jk = p->d_Jk;
    a.Jf = p->d_Jf;
    a.hk = p->d_hk;
    a.row_ptr = p->d_rowptr; a.col = p->d_col; a.val = p->d_val;
    a.R = R;
    a.q = ldexpf(1.0f, -p->frac_bits);
    a.inst = p->inst;
    a.best_e = p->d_best_e; a.best_step = p->d_best_step; a.hit_step = p->d_hit;
    a.hit_ns = p->d_hit_ns;
    a.best_bits = p->d_bits; a.W = p->W;
    a.min_hit = p->d_min_hit; a.replica_iters = p->d_iters; a.err = p->d_err;
    a.tile_rl = p->tile_rl;
    a.coupling_mem = p->coupling_mem;
    a.wait_ns = p->wait_ns;
    a.stall_producer = p->stall_producer;
    a.large_variant = p->large_variant ? p->large_variant : p->tuned_variant;
    return a;
}

// Autotune cache: (N, replicas, operand) -> kernel variant, process-wide.
struct TuneKey {
    int N, R, op;
    bool operator<(const TuneKey &o) const {
        return N != o.N ? N < o.N : (R != o.R ? R < o.R : op < o.op);
    }
};
struct TuneChoice {
    bool large;
    int tile_rl, coupling_mem;
    bool imma;
    bool inc;
    int lvar;        // per-iteration kernel variant (large only)
    int lvar_alt;    // when lvar is a cooperative variant (7..13): the fastest of 1..6, which
                     // other handles with the same key take (they may run concurrently)
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneChoice> g_tune;

int ensure_operand(phia_t *p) {
    if (p->d_Jop) return PHIA_OK;
    p->Mpad = round_up(p->N, 128);
    p->Kbytes = large_kbytes(p->N, p->op);
    if (pool_alloc(&p->d_Jop, (size_t)p->Mpad * p->Kbytes, p->device, p->stream) != cudaSuccess)
        return fail(PHIA_ENOMEM, "J operand allocation failed");
    CU(launch_convert_operand(p->d_Jk, p->N, p->d_Jop, p->Mpad, p->Kbytes, p->op, p->stream));
    return PHIA_OK;
}

// A handle whose kernel variant is automatic takes the cached autotune choice for its
// (N, replicas, operand), if any.
int apply_tuned(phia_t *p, int R) {
    if (!p->auto_tile || p->path != PHIA_PATH_TC) return PHIA_OK;
    TuneChoice c;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune.find(TuneKey{p->N, R, p->op});
        if (it == g_tune.end()) return PHIA_OK;
        c = it->second;
    }
    if (c.large) {
        int rc = ensure_operand(p);
        if (rc) return rc;
    }
    p->large = c.large;
    p->imma = c.imma;
    p->inc = c.inc;
    p->tile_rl = c.tile_rl;
    p->coupling_mem = c.coupling_mem;
    p->tuned_variant = c.large ? (c.lvar >= 7 && !p->tuned_coop ? c.lvar_alt : c.lvar) : 0;
    return PHIA_OK;
}

cudaError_t launch_path(phia_t *p, const RunArgs &a, int *launches) {
    if (p->path == PHIA_PATH_TC && p->large) {
        LargeBuffers B;
        B.Jop = p->d_Jop; B.S = p->d_S; B.Epart = p->d_Epart; B.flags = p->d_flags; B.ready = p->d_ready;
        B.sbits = p->d_sbits;
        B.X = p->d_X; B.V = p->d_V; B.Kbytes = p->Kbytes; B.Mpad = p->Mpad; B.Rpad = large_rpad_handle(a.R);
        B.ctl = p->d_ctl; B.graphs = p->graphs;
        return launch_tc_large(B, a, p->op, p->stream, launches);
    }
    if (p->path == PHIA_PATH_TC && p->imma) return launch_imma_small(a, p->stream, launches);
    // The incremental kernel has no field-only mode: the resident tensor-core kernel
    // covers the same sizes.
    if (p->path == PHIA_PATH_TC && p->inc && !a.field_mode) return launch_inc_small(a, p->stream, launches);
    if (p->path == PHIA_PATH_TC) return launch_tc_small(a, p->op, p->stream, launches);
    if (p->path == PHIA_PATH_FP32) {
        Fp32Metro m{p->d_xstart, p->d_elast, p->d_estart, p->d_xxs, p->d_vvs, p->d_hass};
        return launch_fp32_run(a, p->d_x, p->d_v, p->d_s0, p->d_s1, p->d_eacc, m, p->stream, launches);
    }
    return cudaErrorNotSupported;
}

int common_create(phia_t **out, int32_t N, int32_t frac_bits, const phia_opts *opts, const int32_t *h_k,
                  bool host_h = true) {
    if (!out) return fail(PHIA_EINVAL, "out is NULL");
    *out = nullptr;
    if (N < 1) return fail(PHIA_EINVAL, "N must be >= 1 (got %d)", N);
    if (N > (1 << 20)) return fail(PHIA_ERANGE, "N = %d exceeds 2^20", N);
    if (frac_bits < 0 || frac_bits > 30) return fail(PHIA_EINVAL, "frac_bits must be in [0, 30]");
    if (!h_k) return fail(PHIA_EINVAL, "h_k is NULL");
    for (int i = 0; host_h && i < N; ++i)
        if (h_k[i] >= (1 << 24) || h_k[i] <= -(1 << 24)) return fail(PHIA_ERANGE, "|h_k[%d]| >= 2^24", i);
    return PHIA_OK;
}

int finish_create(phia_t *p, const int32_t *h_k, const phia_opts *opts,
                  cudaMemcpyKind h_kind = cudaMemcpyHostToDevice) {
    CU(pool_alloc((void **)&p->d_hk, (size_t)p->N * 4, p->device, p->stream));
    CU(cudaMemcpyAsync(p->d_hk, h_k, (size_t)p->N * 4, h_kind, p->stream));
    CU(pool_alloc((void **)&p->d_min_hit, 8, p->device, p->stream));
    CU(pool_alloc((void **)&p->d_start_ns, 8, p->device, p->stream));
    CU(cudaMemsetAsync(p->d_start_ns, 0, 8, p->stream));
    CU(pool_alloc((void **)&p->d_iters, 8, p->device, p->stream));
    CU(pool_alloc((void **)&p->d_err, 4, p->device, p->stream));
    CU(cudaMemsetAsync(p->d_err, 0, 4, p->stream));
    CU(pool_alloc((void **)&p->d_ctl, sizeof(IterCtl), p->device, p->stream));
    p->graphs = step_graphs_new();
    CU(cudaEventCreate(&p->ev0));
    CU(cudaEventCreate(&p->ev1));
    CU(cudaStreamSynchronize(p->stream));
    (void)opts;
    return PHIA_OK;
}

}  // namespace

extern "C" {

const char *phia_last_error(void) { return g_err.c_str(); }

}  // extern "C"

namespace {

// The checks of phia_create on device-resident J and h, on opts.device and opts.stream.
int check_dense_on_device(const int8_t *J_k, const int32_t *h_k, int N, const phia_opts &o, int *max_abs) {
    int dev_count = 0;
    if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count == 0)
        return fail(PHIA_ECUDA, "no CUDA device available");
    if (o.device < 0 || o.device >= dev_count) return fail(PHIA_EINVAL, "device %d out of range", o.device);
    CU(cudaSetDevice(o.device));
    const void *ptrs[2] = {J_k, h_k};
    for (const void *ptr : ptrs) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess ||
            (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)) {
            cudaGetLastError();
            return fail(PHIA_EINVAL, "J_k and h_k must be device memory (phia_create takes host arrays)");
        }
        if (at.type == cudaMemoryTypeDevice && at.device != o.device)
            return fail(PHIA_EINVAL, "J_k / h_k are on device %d, opts.device is %d", at.device, o.device);
    }
    int sms = 0;
    CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, o.device));
    cudaStream_t st = (cudaStream_t)o.stream;
    unsigned long long *res = nullptr;
    CU(cudaMalloc((void **)&res, 4 * sizeof(unsigned long long)));
    const unsigned long long init[4] = {ULLONG_MAX, ULLONG_MAX, ULLONG_MAX, 0ull};
    unsigned long long got[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(res, init, sizeof init, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        const int64_t total = (int64_t)N * N;
        const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, (int64_t)sms * 8));
        e = launch_check_dense(J_k, h_k, N, res, blocks, st);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(got, res, sizeof got, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(res);
    if (e != cudaSuccess) return fail(PHIA_ECUDA, "device instance check failed: %s", cudaGetErrorString(e));
    if (got[2] != ULLONG_MAX) return fail(PHIA_ERANGE, "|h_k[%llu]| >= 2^24", got[2]);
    if (got[1] != ULLONG_MAX) return fail(PHIA_EINVAL, "nonzero diagonal J_k[%llu][%llu]", got[1], got[1]);
    if (got[0] != ULLONG_MAX)
        return fail(PHIA_EINVAL, "J_k is not symmetric at (%llu, %llu)", got[0] / (unsigned long long)N,
                    got[0] % (unsigned long long)N);
    *max_abs = (int)got[3];
    return PHIA_OK;
}

// phia_create (host J, h) and phia_create_from_device (device J, h): same checks, options
// and buffers; the checks run where the data lives and the copies are host-to-device or
// device-to-device.
int create_dense(phia_t **out, const int8_t *J_k, const int32_t *h_k, int32_t N, int32_t frac_bits,
                 const phia_opts *opts, bool dev) {
    int rc = common_create(out, N, frac_bits, opts, h_k, !dev);
    if (rc) return rc;
    if (!J_k) return fail(PHIA_EINVAL, "J_k is NULL");
    phia_opts o{};
    if (opts) o = *opts;
    int max_abs = 0;
    if (dev) {
        rc = check_dense_on_device(J_k, h_k, N, o, &max_abs);
        if (rc) return rc;
    } else {
        // Symmetry, zero diagonal and max |k| over the upper triangle, in 64 x 64 tiles so
        // that a tile and its mirror both stay in cache (a row-by-column walk misses on
        // every element of the mirror for large N); bands of tile rows go to the host's
        // cores for large N, and the first mismatch in the serial order is reported.
        constexpr int kTile = 64;
        for (int i = 0; i < N; ++i)
            if (J_k[(size_t)i * N + i] != 0) return fail(PHIA_EINVAL, "nonzero diagonal J_k[%d][%d]", i, i);
        const int bands = (N + kTile - 1) / kTile;
        auto scan = [&](int b0, int b1, int &mx, int64_t &bad) {
            mx = 0;
            bad = -1;
            for (int bi = b0 * kTile; bi < std::min(N, b1 * kTile); bi += kTile) {
                const int ie = std::min(N, bi + kTile);
                for (int bj = bi; bj < N; bj += kTile) {
                    const int je = std::min(N, bj + kTile);
                    for (int i = bi; i < ie; ++i) {
                        const int8_t *row = J_k + (size_t)i * N;
                        for (int j = std::max(bj, i + 1); j < je; ++j) {
                            const int a = row[j], b = J_k[(size_t)j * N + i];
                            if (a != b) {
                                bad = (int64_t)i * N + j;
                                return;
                            }
                            mx = std::max(mx, std::abs(a));
                        }
                    }
                }
            }
        };
        const int nt = N >= 1024 ? std::max(1, std::min<int>(bands, (int)std::thread::hardware_concurrency())) : 1;
        std::vector<int> mx(nt, 0);
        std::vector<int64_t> bad(nt, -1);
        if (nt == 1) {
            scan(0, bands, mx[0], bad[0]);
        } else {
            // the triangle's work shrinks with the band: split it into equal shares of tiles
            std::vector<int> cut(nt + 1, bands);
            cut[0] = 0;
            const int64_t tiles = (int64_t)bands * (bands + 1) / 2;
            int64_t acc = 0;
            for (int b = 0, k = 1; b < bands && k < nt; ++b) {
                acc += bands - b;
                if (acc * nt >= tiles * k) cut[k++] = b + 1;
            }
            std::vector<std::thread> th;
            for (int k = 0; k < nt; ++k) th.emplace_back(scan, cut[k], cut[k + 1], std::ref(mx[k]), std::ref(bad[k]));
            for (auto &x : th) x.join();
        }
        for (int k = 0; k < nt; ++k) {
            if (bad[k] >= 0)
                return fail(PHIA_EINVAL, "J_k is not symmetric at (%d, %d)", (int)(bad[k] / N), (int)(bad[k] % N));
            max_abs = std::max(max_abs, mx[k]);
        }
    }
    if (o.tile_replicas != 0 && o.tile_replicas != 4 && o.tile_replicas != 8 && o.tile_replicas != 16)
        return fail(PHIA_EINVAL, "tile_replicas must be 0, 4, 8 or 16");
    if (o.coupling_mem < 0 || o.coupling_mem > 2) return fail(PHIA_EINVAL, "coupling_mem must be 0, 1 or 2");
    int path = o.path == PHIA_PATH_AUTO ? PHIA_PATH_TC : o.path;
    if (path == PHIA_PATH_CSR) return fail(PHIA_ENOTSUP, "dense instance on the CSR path: use phia_create_csr");
    if (path != PHIA_PATH_TC && path != PHIA_PATH_FP32) return fail(PHIA_EINVAL, "unknown path %d", o.path);
    int op = 0;
    if (path == PHIA_PATH_TC) {
        op = o.operand == PHIA_OP_AUTO ? (max_abs <= 16 ? PHIA_OP_E4M3 : PHIA_OP_BF16) : o.operand;
        if (op != PHIA_OP_E4M3 && op != PHIA_OP_BF16) return fail(PHIA_EINVAL, "unknown operand %d", o.operand);
        if (op == PHIA_OP_E4M3 && max_abs > 16)
            return fail(PHIA_ERANGE, "max |k| = %d is not exact in e4m3 (needs <= 16)", max_abs);
        const int opk = op == PHIA_OP_E4M3 ? kOpE4M3 : kOpBF16;
        if (o.tc_kernel == 1 && N > tc_small_max_n(opk))
            return fail(PHIA_ENOTSUP, "the resident kernel handles N <= %d with this operand (N = %d)",
                        tc_small_max_n(opk), N);
    }
    if (o.tc_kernel < 0 || o.tc_kernel > 4) return fail(PHIA_EINVAL, "tc_kernel must be 0, 1, 2, 3 or 4");
    if (o.tc_kernel == 4 && path == PHIA_PATH_TC) {
        const int nmax = std::min(inc_small_max_n(), tc_small_max_n(op == PHIA_OP_E4M3 ? kOpE4M3 : kOpBF16));
        if (N > nmax)
            return fail(PHIA_ENOTSUP, "the incremental kernel handles N <= %d with this operand (N = %d)", nmax, N);
    }
    if (o.tc_kernel == 3 && N > imma_small_max_n())
        return fail(PHIA_ENOTSUP, "the int8 mma.sync kernel handles N <= %d (N = %d)", imma_small_max_n(), N);
    if (o.large_variant < 0 || o.large_variant > 13) return fail(PHIA_EINVAL, "large_variant must be 0..13");
    int dev_count = 0;
    if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count == 0)
        return fail(PHIA_ECUDA, "no CUDA device available");
    if (o.device < 0 || o.device >= dev_count) return fail(PHIA_EINVAL, "device %d out of range", o.device);
    CU(cudaSetDevice(o.device));
    phia_t *p = new phia_t();
    p->device = o.device;
    p->stream = (cudaStream_t)o.stream;
    p->path = path;
    p->op = op == PHIA_OP_E4M3 ? kOpE4M3 : (op == PHIA_OP_BF16 ? kOpBF16 : 0);
    p->inst = o.instance_id;
    p->tile_rl = o.tile_replicas;
    p->coupling_mem = o.coupling_mem;
    p->auto_tile = o.tile_replicas == 0 && o.coupling_mem == 0 && o.tc_kernel == 0 && o.large_variant == 0;
    p->large_variant = o.large_variant;
    p->N = N;
    p->frac_bits = frac_bits;
    p->W = (N + 31) / 32;
    p->max_abs_k = max_abs;
    if (path == PHIA_PATH_TC) {
        p->large = o.tc_kernel == 2 || (o.tc_kernel == 0 && N > tc_small_max_n(p->op));
        p->imma = o.tc_kernel == 3;
        p->inc = o.tc_kernel == 4;
    }
    const size_t NN = (size_t)N * N;
    auto cleanup = [&](int code) { phia_destroy(p); return code; };
    if (pool_alloc((void **)&p->d_Jk, NN, p->device, p->stream) != cudaSuccess)
        return cleanup(fail(PHIA_ENOMEM, "J allocation failed"));
    if (cudaMemcpyAsync(p->d_Jk, J_k, NN, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, p->stream) !=
        cudaSuccess)
        return cleanup(fail(PHIA_ECUDA, "J upload failed"));
    if (p->large) {
        p->Mpad = round_up(N, 128);
        p->Kbytes = large_kbytes(N, p->op);
        if (pool_alloc(&p->d_Jop, (size_t)p->Mpad * p->Kbytes, p->device, p->stream) != cudaSuccess)
            return cleanup(fail(PHIA_ENOMEM, "J operand allocation failed"));
        if (launch_convert_operand(p->d_Jk, N, p->d_Jop, p->Mpad, p->Kbytes, p->op, p->stream) != cudaSuccess)
            return cleanup(fail(PHIA_ECUDA, "J operand conversion failed"));
    }
    if (path == PHIA_PATH_FP32) {
        const float q = ldexpf(1.0f, -frac_bits);
        if (pool_alloc((void **)&p->d_Jf, NN * 4, p->device, p->stream) != cudaSuccess)
            return cleanup(fail(PHIA_ENOMEM, "J allocation failed"));
        if (dev) {
            k_to_f32_kernel<<<1024, 256, 0, p->stream>>>(p->d_Jk, p->d_Jf, (int64_t)NN, q);
            if (cudaGetLastError() != cudaSuccess) return cleanup(fail(PHIA_ECUDA, "J conversion failed"));
        } else {
            std::vector<float> jf(NN);
            for (size_t e = 0; e < NN; ++e) jf[e] = (float)J_k[e] * q;
            // on the handle's stream, after the pool allocation; a copy from pageable memory
            // returns once jf has been staged
            if (cudaMemcpyAsync(p->d_Jf, jf.data(), NN * 4, cudaMemcpyHostToDevice, p->stream) != cudaSuccess)
                return cleanup(fail(PHIA_ECUDA, "J upload failed"));
        }
    }
    rc = finish_create(p, h_k, &o, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice);
    if (rc) return cleanup(rc);
    *out = p;
    return PHIA_OK;
}

}  // namespace

extern "C" {

int phia_create(phia_t **out, const int8_t *J_k, const int32_t *h_k, int32_t N, int32_t frac_bits,
                const phia_opts *opts) {
    return create_dense(out, J_k, h_k, N, frac_bits, opts, false);
}

int phia_create_from_device(phia_t **out, const int8_t *J_k, const int32_t *h_k, int32_t N, int32_t frac_bits,
                            const phia_opts *opts) {
    return create_dense(out, J_k, h_k, N, frac_bits, opts, true);
}

int phia_create_csr(phia_t **out, const int32_t *row_ptr, const int32_t *col, const int8_t *val_k,
                    const int32_t *h_k, int32_t N, int32_t frac_bits, const phia_opts *opts) {
    int rc = common_create(out, N, frac_bits, opts, h_k);
    if (rc) return rc;
    if (!row_ptr || !col || !val_k) return fail(PHIA_EINVAL, "CSR arrays must not be NULL");
    phia_opts o{};
    if (opts) o = *opts;
    if (o.path != PHIA_PATH_AUTO && o.path != PHIA_PATH_CSR)
        return fail(PHIA_ENOTSUP, "CSR instances run on the CSR path");
    phia_instance_desc d{};
    d.N = N; d.frac_bits = frac_bits; d.row_ptr = row_ptr; d.col = col; d.val_k = val_k; d.h_k = h_k;
    d.instance_id = o.instance_id;
    phia_batch_s *b = nullptr;
    // A single CSR instance runs one launch per iteration (graph-replayed) unless the
    // persistent launch is asked for (tc_kernel = 1): several such handles often run at
    // once on their own streams, and a cooperative launch wants the device to itself.
    phia_opts ob = o;
    ob.tc_kernel = o.tc_kernel == 1 ? 1 : 2;
    rc = batch_create(&b, 1, &d, &ob);
    if (rc) return rc;
    phia_t *p = new phia_t();
    p->device = o.device;
    p->stream = (cudaStream_t)o.stream;
    p->path = PHIA_PATH_CSR;
    p->inst = o.instance_id;
    p->N = N;
    p->frac_bits = frac_bits;
    p->W = (N + 31) / 32;
    p->csr = true;
    p->batch = b;
    *out = p;
    return PHIA_OK;
}

static int run_impl(phia_t *p, const phia_schedule *sched, int32_t R, int64_t t0, int64_t steps, int64_t total,
                    uint64_t seed, const float *x_in, float *x_out, const float *v_in, float *v_out, int reset) {
    if (!p) return fail(PHIA_EINVAL, "handle is NULL");
    int rc = check_sched(sched);
    if (rc) return rc;
    if (p->batch) return batch_run(p->batch, sched, R, t0, steps, total, seed, x_in, x_out, v_in, v_out, reset,
                                   nullptr, nullptr, nullptr);
    if (R < 1) return fail(PHIA_EINVAL, "replicas must be >= 1");
    if (sched->accept_test == 1 && p->path == PHIA_PATH_TC) {
        // The acceptance test runs in the resident tcgen05 kernel with J in shared memory.
        if (p->auto_tile && p->N <= tc_small_max_n(p->op)) {
            p->large = p->imma = p->inc = false;
            p->coupling_mem = 1;
        } else if (p->large || p->imma || p->inc || p->coupling_mem == 2) {
            return fail(PHIA_ENOTSUP, "schedule.accept_test = 1 runs on the resident tcgen05 kernel with J in shared "
                                      "memory (tc_kernel 1, N <= %d with this operand) or the FP32 path",
                        tc_small_max_n(p->op));
        }
    }
    if (steps < 1) return fail(PHIA_EINVAL, "steps must be >= 1");
    if (t0 < 0 || total < t0 + steps) return fail(PHIA_EINVAL, "need 0 <= t0 and t0 + steps <= total_steps");
    if (total > (int64_t)1 << 31) return fail(PHIA_ERANGE, "total_steps must be < 2^31 (Philox counter word)");
    CU(cudaSetDevice(p->device));
    if (!reset && (!p->ran || p->R_last != R))
        return fail(PHIA_ESTATE, "reset_best = 0 needs a previous run with the same replica count");
    if (reset && sched->accept_test == 0) {
        rc = apply_tuned(p, R);
        if (rc) return rc;
    }
    rc = ensure_replicas(p, R);
    if (rc) return rc;
    if (reset) {
        rc = reset_records(p, R);
        if (rc) return rc;
    }
    CU(cudaMemsetAsync(p->d_min_hit, 0xFF, 8, p->stream));
    CU(cudaMemsetAsync(p->d_iters, 0, 8, p->stream));
    CU(cudaMemsetAsync(p->d_err, 0, 4, p->stream));
    CU(cudaMemsetAsync(p->d_prop, 0, (size_t)R * 8, p->stream));
    CU(cudaMemsetAsync(p->d_acc, 0, (size_t)R * 8, p->stream));
    RunArgs a = base_args(p, R);
    a.accept_test = sched->accept_test;
    a.proposed = p->d_prop;
    a.accepted = p->d_acc;
    a.t0 = t0; a.nsteps = steps; a.T_total = total;
    a.beta0 = sched->beta0; a.beta1 = sched->beta1; a.eps = sched->eps; a.gamma = sched->gamma;
    a.refresh = sched->refresh;
    a.deriv = sched->deriv;
    a.seed = seed;
    a.x_in = x_in; a.v_in = v_in; a.x_out = x_out; a.v_out = v_out;
    a.has_target = sched->has_target; a.stop_at_target = sched->stop_at_target; a.target = sched->target_k;
    int launches = reset ? 1 : 0;
    CU(cudaEventRecord(p->ev0, p->stream));
    cudaError_t e = launch_path(p, a, &launches);
    if (e != cudaSuccess) return fail(PHIA_ECUDA, "kernel launch failed: %s", cudaGetErrorString(e));
    CU(cudaEventRecord(p->ev1, p->stream));
    p->ran = true;
    p->R_last = R;
    p->last_steps = steps;
    p->last_launches = launches;
    p->last_stop = sched->stop_at_target;
    return PHIA_OK;
}

int phia_autotune(phia_t *p, const phia_schedule *sched, int32_t replicas, int32_t probe_iters,
                  phia_tune_result *out) {
    if (!p || !sched) return fail(PHIA_EINVAL, "NULL argument");
    if (p->path != PHIA_PATH_TC) return fail(PHIA_ENOTSUP, "the autotuner chooses among tensor-core kernels");
    if (replicas < 1 || probe_iters < 1) return fail(PHIA_EINVAL, "need replicas >= 1 and probe_iters >= 1");
    std::vector<TuneChoice> cands;
    if (p->N <= tc_small_max_n(p->op)) {
        for (int tile : {4, 8, 16})
            for (int mem : {1, 2}) cands.push_back(TuneChoice{false, tile, mem, false, false, 0, 0});
    }
    if (p->N <= imma_small_max_n()) {
        cands.push_back(TuneChoice{false, 8, 0, true, false, 0, 0});
        cands.push_back(TuneChoice{false, 16, 0, true, false, 0, 0});
    }
    if (p->N <= std::min(inc_small_max_n(), tc_small_max_n(p->op))) {
        for (int tile : {4, 8, 16})
            if (inc_small_tile_replicas(p->N, tile) == tile)
                cands.push_back(TuneChoice{false, tile, 0, false, true, 0, 0});
    }
    for (int lv = 1; lv <= 13; ++lv) cands.push_back(TuneChoice{true, 0, 0, false, false, lv, 0});
    const bool saved_auto = p->auto_tile;
    p->auto_tile = false;
    float best_ms = 1e30f, worst_ms = 0.f, alt_ms = 1e30f;
    TuneChoice best = cands[0];
    int best_alt = 1;   // fastest non-cooperative per-iteration variant
    for (const TuneChoice &c : cands) {
        if (c.large) {
            int rc = ensure_operand(p);
            if (rc) { p->auto_tile = saved_auto; return rc; }
        }
        p->large = c.large;
        p->imma = c.imma;
        p->inc = c.inc;
        p->tile_rl = c.tile_rl;
        p->coupling_mem = c.coupling_mem;
        p->tuned_variant = c.lvar;
        float ms = 0.f;
        for (int rep = 0; rep < 2; ++rep) {   // the first run warms up
            int rc = run_impl(p, sched, replicas, 0, probe_iters, probe_iters, 1, nullptr, nullptr, nullptr, nullptr, 1);
            if (rc) { p->auto_tile = saved_auto; return rc; }
            CU(cudaEventSynchronize(p->ev1));
            CU(cudaEventElapsedTime(&ms, p->ev0, p->ev1));
        }
        if (ms < best_ms) { best_ms = ms; best = c; }
        if (c.large && c.lvar < 7 && ms < alt_ms) { alt_ms = ms; best_alt = c.lvar; }
        worst_ms = std::max(worst_ms, ms);
    }
    p->large = best.large;
    p->imma = best.imma;
    p->inc = best.inc;
    p->tile_rl = best.tile_rl;
    p->coupling_mem = best.coupling_mem;
    p->tuned_variant = best.lvar;
    p->tuned_coop = best.large && best.lvar >= 7;
    p->auto_tile = saved_auto;
    best.lvar_alt = best_alt;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune[TuneKey{p->N, replicas, p->op}] = best;
    }
    if (out) {
        memset(out, 0, sizeof *out);
        out->tc_kernel = best.large ? 2 : (best.imma ? 3 : (best.inc ? 4 : 1));
        out->tile_replicas = best.large ? 0
                             : (best.imma || best.inc ? best.tile_rl : tc_small_tile_replicas(replicas, best.tile_rl));
        out->coupling_mem = best.large || best.imma || best.inc ? 0 : best.coupling_mem;
        out->candidates = (int32_t)cands.size();
        out->best_us_per_iter = 1000.f * best_ms / probe_iters;
        out->worst_us_per_iter = 1000.f * worst_ms / probe_iters;
        out->large_variant = best.large ? best.lvar : 0;
    }
    return PHIA_OK;
}

int phia_anneal(phia_t *p, const phia_schedule *sched, int32_t replicas, int64_t steps, uint64_t seed) {
    return run_impl(p, sched, replicas, 0, steps, steps, seed, nullptr, nullptr, nullptr, nullptr, 1);
}

int phia_run(phia_t *p, const phia_schedule *sched, int32_t replicas, int64_t t0, int64_t steps,
             int64_t total_steps, uint64_t seed, float *x, float *v, int32_t reset_best) {
    if (!x || !v) return fail(PHIA_EINVAL, "x and v must be device arrays");
    return run_impl(p, sched, replicas, t0, steps, total_steps, seed, x, x, v, v, reset_best ? 1 : 0);
}

int phia_init_state(phia_t *p, int32_t replicas, uint64_t seed, float *x, float *v) {
    if (!p) return fail(PHIA_EINVAL, "handle is NULL");
    if (replicas < 1 || !x || !v) return fail(PHIA_EINVAL, "need replicas >= 1 and device x, v");
    CU(cudaSetDevice(p->device));
    CU(launch_init_state(replicas, p->N, seed, p->inst, x, v, p->stream));
    return PHIA_OK;
}

int phia_field(phia_t *p, const int8_t *spins, int32_t R, int32_t *field_k, int64_t *energy_k) {
    if (!p) return fail(PHIA_EINVAL, "handle is NULL");
    if (R < 1 || !spins) return fail(PHIA_EINVAL, "need replicas >= 1 and device spins");
    if (p->batch) return batch_run(p->batch, nullptr, R, 0, 1, 1, 0, nullptr, nullptr, nullptr, nullptr, 1, spins,
                                   field_k, energy_k);
    CU(cudaSetDevice(p->device));
    int rc = ensure_replicas(p, R);
    if (rc) return rc;
    RunArgs a = base_args(p, R);
    a.field_mode = 1;
    a.spins_in = spins;
    a.field_out = field_k;
    a.energy_out = energy_k;
    a.nsteps = 1; a.T_total = 1;
    int launches = 0;
    cudaError_t e = launch_path(p, a, &launches);
    if (e != cudaSuccess) return fail(PHIA_ECUDA, "kernel launch failed: %s", cudaGetErrorString(e));
    return PHIA_OK;
}

int phia_philox_draws(uint64_t seed, uint32_t instance_id, uint32_t d, int32_t R, int32_t N, uint32_t *raw,
                      float *x, float *v, void *stream) {
    if (R < 0 || N < 0) return fail(PHIA_EINVAL, "negative size");
    CU(launch_philox_draws(seed, instance_id, d, R, N, raw, x, v, (cudaStream_t)stream));
    return PHIA_OK;
}

int phia_debug_wait(phia_t *p, int64_t wait_budget_ns, int32_t stall_producer) {
    if (!p) return fail(PHIA_EINVAL, "handle is NULL");
    if (wait_budget_ns < 0 || stall_producer < 0 || stall_producer > 1)
        return fail(PHIA_EINVAL, "need wait_budget_ns >= 0 and stall_producer 0 or 1");
    if (stall_producer && !(p->path == PHIA_PATH_TC && p->large && !p->auto_tile))
        return fail(PHIA_ENOTSUP, "the stall applies to a handle created with tc_kernel = 2 (per-iteration kernel)");
    p->wait_ns = wait_budget_ns;
    p->stall_producer = stall_producer;
    return PHIA_OK;
}

int phia_sync(phia_t *p) {
    if (!p) return fail(PHIA_EINVAL, "handle is NULL");
    CU(cudaSetDevice(p->device));
    CU(cudaStreamSynchronize(p->stream));
    return PHIA_OK;
}

static int fetch_records(phia_t *p, std::vector<int64_t> &be, std::vector<int64_t> &bs, std::vector<int64_t> &hs) {
    if (!p->ran) return fail(PHIA_ESTATE, "no run on this handle yet");
    CU(cudaSetDevice(p->device));
    CU(cudaStreamSynchronize(p->stream));
    int32_t err = 0;
    CU(cudaMemcpy(&err, p->d_err, 4, cudaMemcpyDeviceToHost));
    if (err) return fail(PHIA_ETIMEOUT, "a bounded device wait expired during the run");
    const int R = p->R_last;
    be.resize(R); bs.resize(R); hs.resize(R);
    CU(cudaMemcpy(be.data(), p->d_best_e, (size_t)R * 8, cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(bs.data(), p->d_best_step, (size_t)R * 8, cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(hs.data(), p->d_hit, (size_t)R * 8, cudaMemcpyDeviceToHost));
    return PHIA_OK;
}

// Result replica: with stop-at-target and a hit, the earliest hit (ties: lowest index);
// otherwise the lowest energy (ties: earliest step, then lowest index).
static int pick_result(phia_t *p, const std::vector<int64_t> &be, const std::vector<int64_t> &bs,
                       const std::vector<int64_t> &hs) {
    int best = -1;
    if (p->last_stop) {
        for (int r = 0; r < (int)hs.size(); ++r)
            if (hs[r] >= 0 && (best < 0 || hs[r] < hs[best])) best = r;
        if (best >= 0) return best;
    }
    for (int r = 0; r < (int)be.size(); ++r) {
        if (bs[r] < 0) continue;
        if (best < 0 || be[r] < be[best] || (be[r] == be[best] && bs[r] < bs[best])) best = r;
    }
    return best;
}

int phia_best(phia_t *p, int64_t *energy_k, int8_t *spins) {
    if (!p) return fail(PHIA_EINVAL, "handle is NULL");
    if (p->batch) return batch_best(p->batch, 0, energy_k, spins);
    std::vector<int64_t> be, bs, hs;
    int rc = fetch_records(p, be, bs, hs);
    if (rc) return rc;
    const int r = pick_result(p, be, bs, hs);
    if (r < 0) return fail(PHIA_ESTATE, "no replica recorded a state");
    if (energy_k) *energy_k = be[r];
    if (spins) {
        std::vector<uint32_t> w(p->W);
        CU(cudaMemcpy(w.data(), p->d_bits + (size_t)r * p->W, (size_t)p->W * 4, cudaMemcpyDeviceToHost));
        for (int i = 0; i < p->N; ++i) spins[i] = ((w[i >> 5] >> (i & 31)) & 1u) ? 1 : -1;
    }
    return PHIA_OK;
}

int phia_gahmc(phia_t *p, const phia_gahmc_schedule *sched, int32_t R, int64_t K, uint64_t seed, float *x, float *v,
               int64_t *counts, int32_t *events, int32_t events_cap) {
    if (!p || !sched) return fail(PHIA_EINVAL, "NULL argument");
    if (p->batch) return fail(PHIA_ENOTSUP, "GAHMC runs on dense handles");
    if (p->N > gahmc_max_n()) return fail(PHIA_ENOTSUP, "GAHMC handles N <= %d (N = %d)", gahmc_max_n(), p->N);
    if (R < 1 || K < 1) return fail(PHIA_EINVAL, "need replicas >= 1 and trajectories >= 1");
    if (K > ((int64_t)1 << 31)) return fail(PHIA_ERANGE, "trajectories must be < 2^31 (Philox counter word)");
    if (!(sched->travel > 0.0f) || !(sched->travel <= 3.14159265f))
        return fail(PHIA_EINVAL, "travel must be in (0, pi]");
    if (!(sched->beta0 >= 0.0f) || !(sched->beta1 >= 0.0f)) return fail(PHIA_EINVAL, "beta0 and beta1 must be >= 0");
    if (events && events_cap < 1) return fail(PHIA_EINVAL, "events_cap must be >= 1 with an events array");
    CU(cudaSetDevice(p->device));
    int rc = ensure_replicas(p, R);
    if (rc) return rc;
    rc = reset_records(p, R);
    if (rc) return rc;
    CU(cudaMemsetAsync(p->d_iters, 0, 8, p->stream));
    CU(cudaMemsetAsync(p->d_err, 0, 4, p->stream));
    CU(cudaMemsetAsync(p->d_prop, 0, (size_t)R * 8, p->stream));
    CU(cudaMemsetAsync(p->d_acc, 0, (size_t)R * 8, p->stream));
    RunArgs a = base_args(p, R);
    a.beta0 = sched->beta0; a.beta1 = sched->beta1;
    a.seed = seed;
    a.x_in = x; a.v_in = v; a.x_out = x; a.v_out = v;
    a.has_target = sched->has_target; a.target = sched->target_k;
    CU(cudaEventRecord(p->ev0, p->stream));
    cudaError_t e = launch_gahmc(a, sched->travel, K, counts, events, events_cap, p->stream);
    if (e != cudaSuccess) return fail(PHIA_ECUDA, "kernel launch failed: %s", cudaGetErrorString(e));
    CU(cudaEventRecord(p->ev1, p->stream));
    p->ran = true;
    p->R_last = R;
    p->last_steps = K;
    p->last_launches = 2;
    p->last_stop = 0;
    return PHIA_OK;
}

int phia_acceptance(phia_t *p, int32_t R, int64_t *proposed, int64_t *accepted) {
    if (!p) return fail(PHIA_EINVAL, "handle is NULL");
    if (p->batch) return fail(PHIA_ENOTSUP, "the acceptance test does not run on the CSR path");
    std::vector<int64_t> be, bs, hs;
    int rc = fetch_records(p, be, bs, hs);
    if (rc) return rc;
    if (R != p->R_last) return fail(PHIA_EINVAL, "replicas (%d) differs from the last run (%d)", R, p->R_last);
    if (proposed) CU(cudaMemcpy(proposed, p->d_prop, (size_t)R * 8, cudaMemcpyDeviceToHost));
    if (accepted) CU(cudaMemcpy(accepted, p->d_acc, (size_t)R * 8, cudaMemcpyDeviceToHost));
    return PHIA_OK;
}

int phia_replica_results(phia_t *p, int32_t R, int64_t *best_energy_k, int64_t *best_step, int64_t *hit_step,
                         uint32_t *best_bits) {
    if (!p) return fail(PHIA_EINVAL, "handle is NULL");
    if (p->batch) return batch_replica_results(p->batch, 0, R, best_energy_k, best_step, hit_step, best_bits);
    std::vector<int64_t> be, bs, hs;
    int rc = fetch_records(p, be, bs, hs);
    if (rc) return rc;
    if (R != p->R_last) return fail(PHIA_EINVAL, "replicas (%d) differs from the last run (%d)", R, p->R_last);
    if (best_energy_k) memcpy(best_energy_k, be.data(), (size_t)R * 8);
    if (best_step) memcpy(best_step, bs.data(), (size_t)R * 8);
    if (hit_step) memcpy(hit_step, hs.data(), (size_t)R * 8);
    if (best_bits) CU(cudaMemcpy(best_bits, p->d_bits, (size_t)R * p->W * 4, cudaMemcpyDeviceToHost));
    return PHIA_OK;
}

int phia_stats_get(phia_t *p, phia_stats *out) {
    if (!p || !out) return fail(PHIA_EINVAL, "NULL argument");
    if (p->batch) return batch_stats(p->batch, 0, out);
    std::vector<int64_t> be, bs, hs;
    int rc = fetch_records(p, be, bs, hs);
    if (rc) return rc;
    memset(out, 0, sizeof *out);
    unsigned long long iters = 0;
    CU(cudaMemcpy(&iters, p->d_iters, 8, cudaMemcpyDeviceToHost));
    float ms = 0.f;
    CU(cudaEventElapsedTime(&ms, p->ev0, p->ev1));
    out->replicas = p->R_last;
    out->steps = p->last_steps;
    out->spin_updates = (int64_t)iters * p->N;
    const int r = pick_result(p, be, bs, hs);
    out->best_replica = r;
    out->best_energy_k = r >= 0 ? be[r] : 0;
    out->best_step = r >= 0 ? bs[r] : -1;
    out->hit_step = -1;
    out->hit_replica = -1;
    for (int k = 0; k < (int)hs.size(); ++k)
        if (hs[k] >= 0 && (out->hit_step < 0 || hs[k] < out->hit_step)) { out->hit_step = hs[k]; out->hit_replica = k; }
    out->hit_ns = -1;
    if (out->hit_replica >= 0) {
        uint64_t t_hit = 0, t_start = 0;
        CU(cudaMemcpy(&t_hit, p->d_hit_ns + out->hit_replica, 8, cudaMemcpyDeviceToHost));
        CU(cudaMemcpy(&t_start, p->d_start_ns, 8, cudaMemcpyDeviceToHost));
        if (t_hit >= t_start && t_start != 0) out->hit_ns = (int64_t)(t_hit - t_start);
    }
    out->device_ms = ms;
    out->path = p->path;
    out->operand = p->op == kOpE4M3 ? PHIA_OP_E4M3 : (p->op == kOpBF16 ? PHIA_OP_BF16 : 0);
    out->kernel_launches = p->last_launches;
    out->tc_kernel = p->path == PHIA_PATH_TC ? (p->large ? 2 : (p->imma ? 3 : (p->inc ? 4 : 1))) : 0;
    return PHIA_OK;
}

void phia_destroy(phia_t *p) {
    if (!p) return;
    if (p->batch) phia_batch_destroy(p->batch);
    cudaSetDevice(p->device);
    cudaStreamSynchronize(p->stream);
    free_replicas(p);
    for (void *b : {(void *)p->d_Jk, (void *)p->d_Jf, (void *)p->d_hk, (void *)p->d_Jop, (void *)p->d_min_hit,
                    (void *)p->d_iters, (void *)p->d_err, (void *)p->d_ctl, (void *)p->d_start_ns})
        pool_free(b, p->stream);
    cudaFree(p->d_rowptr); cudaFree(p->d_col); cudaFree(p->d_val);
    step_graphs_free(p->graphs);
    if (p->ev0) cudaEventDestroy(p->ev0);
    if (p->ev1) cudaEventDestroy(p->ev1);
    delete p;
}

}  // extern "C"
