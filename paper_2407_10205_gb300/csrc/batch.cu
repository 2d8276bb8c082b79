// batch.cu -- batched multi-instance runs (phia_batch_* of the C ABI): instance validation
// and packing, per-replica state of every instance.  Small dense instances (N <= 384 with
// every |k| <= 16, N <= 256 otherwise) run on the resident tcgen05 kernel with a table of
// CTAs, all their iterations in one launch per (operand, spin tiles) group; the rest run
// on the CSR path (dense ones converted to CSR): 64-row blocks, one launch per iteration
// or one persistent launch over all iterations.
#include <algorithm>
#include <atomic>
#include <climits>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/phia.h"
#include "device_common.cuh"
#include "phia_internal.h"

using namespace phia;

struct phia_batch_s {
    int device = 0;
    cudaStream_t stream = nullptr;
    int count = 0;                      // instances (public indices 0 .. count-1)
    std::vector<CsrInst> inst;          // CSR members only (offsets for replicas set per run)
    std::vector<int> csr_pub;           // CSR member -> public index
    std::vector<int> N, frac;           // per public instance
    std::vector<uint32_t> inst_id;
    std::vector<int64_t> h_off;         // into d_hk
    // small dense members: resident tcgen05 kernel over a table of CTAs
    std::vector<int> dense_pub;         // public indices
    std::vector<int64_t> dense_joff;    // offset of each member's J in d_dJ
    std::vector<int> dense_op;          // kOpE4M3 / kOpBF16
    int8_t *d_dJ = nullptr;
    SmallCta *d_small = nullptr;
    size_t small_cap = 0;
    std::vector<SmallCta> small_host;
    std::vector<int64_t> bits_pub;      // per public instance: offset of its best states
    std::vector<long long> targets;     // per instance, LLONG_MIN = none
    std::vector<CsrBlock> blocks;
    int64_t total_rows = 0, total_nnz = 0;
    int max_words = 0;
    CsrInst *d_inst = nullptr;
    CsrBlock *d_blocks = nullptr;
    int32_t *d_rowptr = nullptr, *d_col = nullptr, *d_hk = nullptr;
    int8_t *d_val = nullptr;
    long long *d_targets = nullptr;
    bool any_target = false;
    // replica state (R padded to a multiple of 256)
    int Rcap = 0, R = 0, R_real = 0;
    float *d_X = nullptr, *d_V = nullptr;
    uint32_t *d_S = nullptr;
    int64_t *d_Esum = nullptr;
    int8_t *d_flags = nullptr;
    int64_t *d_best_e = nullptr, *d_best_step = nullptr, *d_hit = nullptr;
    uint32_t *d_bits = nullptr;
    unsigned long long *d_min_hit = nullptr, *d_iters = nullptr;
    uint64_t *d_hit_ns = nullptr;       // %globaltimer of each replica's first hit
    uint64_t *d_start_ns = nullptr;     // %globaltimer when the run's records were reset
    int32_t *d_err = nullptr;
    IterCtl *d_ctl = nullptr;               // iteration control of the step kernel
    unsigned *d_sync = nullptr;             // barrier and work counters of the persistent launch
    int csr_mode = 1;                       // 1 persistent CSR launch, 2 one launch per iteration
    StepGraphCache *graphs = nullptr;       // its step launches as replayable graphs
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    bool ran = false;
    int64_t last_steps = 0;
    int last_launches = 0;
    int last_stop = 0;
};

namespace {

int bfail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return set_last_error(code, buf);
}

#define BCU(call)                                                                                   \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) return bfail(PHIA_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));   \
    } while (0)

__global__ void batch_reset_records(int64_t n, int64_t nbits, int64_t *best_e, int64_t *best_step, int64_t *hit,
                                    uint32_t *bits, uint64_t *hit_ns, uint64_t *start_ns) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < n) {
        best_e[idx] = LLONG_MAX;
        best_step[idx] = -1;
        hit[idx] = -1;
        hit_ns[idx] = 0;
    }
    if (idx < nbits) bits[idx] = 0u;
    if (idx == 0) *start_ns = globaltimer_ns();   // the run's start on the device clock
}

void free_state(phia_batch_s *b) {
    cudaFree(b->d_X); cudaFree(b->d_V); cudaFree(b->d_S); cudaFree(b->d_Esum); cudaFree(b->d_flags);
    cudaFree(b->d_best_e); cudaFree(b->d_best_step); cudaFree(b->d_hit); cudaFree(b->d_bits);
    cudaFree(b->d_hit_ns);
    b->d_X = b->d_V = nullptr; b->d_S = nullptr; b->d_Esum = nullptr; b->d_flags = nullptr;
    b->d_best_e = b->d_best_step = b->d_hit = nullptr; b->d_bits = nullptr; b->d_hit_ns = nullptr;
    b->Rcap = 0;
}

int64_t words_of(int n) { return (n + 31) / 32; }

// Per-replica offsets for R replicas per instance: records and best states by public
// index (instance k's records start at k R), CSR state over the CSR members only.
void layout(phia_batch_s *b, int R) {
    b->bits_pub.assign((size_t)b->count, 0);
    int64_t bits = 0;
    for (int k = 0; k < b->count; ++k) {
        b->bits_pub[(size_t)k] = bits;
        bits += (int64_t)R * words_of(b->N[(size_t)k]);
    }
    int64_t x = 0, xin = 0, s = 0;
    for (size_t c = 0; c < b->inst.size(); ++c) {
        CsrInst &in = b->inst[c];
        const int k = b->csr_pub[c];
        in.x_off = x; in.xin_off = xin; in.s_off = s;
        in.rec_off = (int64_t)k * R;
        in.bits_off = b->bits_pub[(size_t)k];
        x += (int64_t)in.N * R;
        xin += (int64_t)in.N * b->R_real;
        s += (int64_t)in.N * (R / 32);
    }
}

int ensure_state(phia_batch_s *b, int R) {
    if (R <= b->Rcap) return PHIA_OK;
    BCU(cudaStreamSynchronize(b->stream));
    free_state(b);
    const int64_t rows = b->total_rows;
    int64_t bits = 0;
    for (int k = 0; k < b->count; ++k) bits += (int64_t)R * words_of(b->N[k]);
    const int64_t reps = (int64_t)R * b->count;
    bool ok = true;
    auto al = [&](void **p, size_t n) {
        if (ok && cudaMalloc(p, std::max<size_t>(n, 16)) != cudaSuccess) ok = false;
    };
    al((void **)&b->d_X, (size_t)rows * R * 4);
    al((void **)&b->d_V, (size_t)rows * R * 4);
    al((void **)&b->d_S, (size_t)4 * rows * (R / 32) * 4);
    al((void **)&b->d_Esum, (size_t)2 * reps * 8);
    al((void **)&b->d_flags, (size_t)2 * reps);
    al((void **)&b->d_best_e, (size_t)reps * 8);
    al((void **)&b->d_best_step, (size_t)reps * 8);
    al((void **)&b->d_hit, (size_t)reps * 8);
    al((void **)&b->d_hit_ns, (size_t)reps * 8);
    al((void **)&b->d_bits, (size_t)bits * 4);
    if (!ok) {
        cudaGetLastError();
        free_state(b);
        return bfail(PHIA_ENOMEM, "device allocation for %d replicas per instance failed", R);
    }
    BCU(cudaMemsetAsync(b->d_flags, 0, (size_t)2 * reps, b->stream));
    b->Rcap = R;
    return PHIA_OK;
}

}  // namespace

namespace phia {

// One instance of a batch, checked and converted to padded CSR (row offsets relative to
// the instance), before concatenation; code/msg hold its first error.
struct PackedInst {
    int code = PHIA_OK;
    std::string msg;
    std::vector<int32_t> rp, col;
    std::vector<int8_t> val;
    int64_t nnz_real = 0;
    int small_op = 0;       // small dense member: its tensor-core operand (no CSR built)
};

void pack_error(PackedInst &out, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    out.code = code;
    out.msg = buf;
}

void pack_instance(const phia_instance_desc &x, int k, PackedInst &out) {
    const int n = x.N;
    if (n < 1) return pack_error(out, PHIA_EINVAL, "instance %d: N must be >= 1", k);
    if (x.frac_bits < 0 || x.frac_bits > 30) return pack_error(out, PHIA_EINVAL, "instance %d: bad frac_bits", k);
    if (!x.h_k) return pack_error(out, PHIA_EINVAL, "instance %d: h_k is NULL", k);
    for (int i = 0; i < n; ++i)
        if (x.h_k[i] >= (1 << 24) || x.h_k[i] <= -(1 << 24))
            return pack_error(out, PHIA_ERANGE, "instance %d: |h_k[%d]| >= 2^24", k, i);
    std::vector<int32_t> &col = out.col;
    std::vector<int8_t> &val = out.val;
    // Every row is padded to a multiple of 8 entries with k = 0 (column 0): rows start
    // 32-byte aligned in col and 8-byte aligned in val (instances are concatenated in
    // whole padded rows), so the step kernel reads a row's entries 8 at a time with
    // aligned vector loads and no tail.
    auto pad_row = [&]() {
        while (col.size() % 8) {
            col.push_back(0);
            val.push_back(0);
        }
    };
    std::vector<int32_t> &rp = out.rp;
    rp.assign((size_t)n + 1, 0);
    if (x.J_k) {
        // Small enough for the resident tensor-core kernel: checked here, kept dense.
        int maxk = 0;
        for (int i = 0; i < n; ++i) {
            if (x.J_k[(size_t)i * n + i] != 0) return pack_error(out, PHIA_EINVAL, "instance %d: nonzero diagonal", k);
            for (int j = i + 1; j < n; ++j) {
                const int a = x.J_k[(size_t)i * n + j];
                if (a != x.J_k[(size_t)j * n + i])
                    return pack_error(out, PHIA_EINVAL, "instance %d: J_k is not symmetric at (%d, %d)", k, i, j);
                maxk = std::max(maxk, std::abs(a));
            }
        }
        const int op = maxk <= 16 ? kOpE4M3 : kOpBF16;
        if (n <= tc_small_max_n(op)) {
            out.small_op = op;
            return;
        }
        for (int i = 0; i < n; ++i) {
            if (x.J_k[(size_t)i * n + i] != 0) return pack_error(out, PHIA_EINVAL, "instance %d: nonzero diagonal", k);
            for (int j = 0; j < n; ++j) {
                if (x.J_k[(size_t)i * n + j] != x.J_k[(size_t)j * n + i])
                    return pack_error(out, PHIA_EINVAL, "instance %d: J_k is not symmetric at (%d, %d)", k, i, j);
                if (x.J_k[(size_t)i * n + j] != 0) {
                    col.push_back(j);
                    val.push_back(x.J_k[(size_t)i * n + j]);
                    ++out.nnz_real;
                }
            }
            pad_row();
            rp[i + 1] = (int32_t)col.size();
        }
        return;
    }
    if (!x.row_ptr || !x.col || !x.val_k) return pack_error(out, PHIA_EINVAL, "instance %d: CSR arrays missing", k);
    if (x.row_ptr[0] != 0) return pack_error(out, PHIA_EINVAL, "instance %d: row_ptr[0] != 0", k);
    for (int i = 0; i < n; ++i)
        if (x.row_ptr[i + 1] < x.row_ptr[i]) return pack_error(out, PHIA_EINVAL, "instance %d: row_ptr decreases", k);
    // Rows with ascending columns are searched by bisection in the symmetry check.
    std::vector<uint8_t> row_sorted(n);
    for (int i = 0; i < n; ++i) row_sorted[i] = std::is_sorted(x.col + x.row_ptr[i], x.col + x.row_ptr[i + 1]);
    col.reserve((size_t)x.row_ptr[n] + 8 * (size_t)n);
    val.reserve((size_t)x.row_ptr[n] + 8 * (size_t)n);
    for (int i = 0; i < n; ++i) {
        for (int32_t p = x.row_ptr[i]; p < x.row_ptr[i + 1]; ++p) {
            const int j = x.col[p];
            if (j < 0 || j >= n) return pack_error(out, PHIA_EINVAL, "instance %d: col out of range", k);
            if (j == i) return pack_error(out, PHIA_EINVAL, "instance %d: self loop at %d", k, i);
            // symmetry: (j, i) must exist with the same value
            const int32_t *cb = x.col + x.row_ptr[j], *ce = x.col + x.row_ptr[j + 1];
            const int32_t *f = row_sorted[j] ? std::lower_bound(cb, ce, i) : std::find(cb, ce, i);
            if (f != ce && *f != i) f = ce;
            if (f == ce || x.val_k[x.row_ptr[j] + (f - cb)] != x.val_k[p])
                return pack_error(out, PHIA_EINVAL, "instance %d: CSR is not symmetric at (%d, %d)", k, i, j);
            col.push_back(j);
            val.push_back(x.val_k[p]);
            ++out.nnz_real;
        }
        pad_row();
        rp[i + 1] = (int32_t)col.size();
    }
}

int batch_create(phia_batch_s **out, int32_t count, const phia_instance_desc *d, const phia_opts *opts) {
    if (!out) return bfail(PHIA_EINVAL, "out is NULL");
    *out = nullptr;
    if (count < 1 || !d) return bfail(PHIA_EINVAL, "need count >= 1 and descriptors");
    phia_opts o{};
    if (opts) o = *opts;
    if (o.path != PHIA_PATH_AUTO && o.path != PHIA_PATH_CSR)
        return bfail(PHIA_ENOTSUP, "batches run on the CSR path");
    if (o.tc_kernel < 0 || o.tc_kernel > 2) return bfail(PHIA_EINVAL, "batches: tc_kernel must be 0, 1 or 2");
    phia_batch_s *b = new phia_batch_s();
    b->csr_mode = o.tc_kernel == 2 ? 2 : 1;
    auto cleanup = [&](int code) { phia_batch_destroy(b); return code; };
    b->count = count;
    // Instances are checked and converted independently, on every host core (a batch of
    // 256 instances with 2.8e7 couplings took 1.3 s on one core); the first failing
    // instance in order is reported, as a sequential pass would.
    std::vector<PackedInst> packed((size_t)count);
    {
        std::atomic<int> next{0};
        auto work = [&]() {
            for (int k; (k = next.fetch_add(1)) < count;) pack_instance(d[k], k, packed[(size_t)k]);
        };
        const int nthreads = std::max(1, std::min<int>(count, (int)std::thread::hardware_concurrency()));
        std::vector<std::thread> workers;
        for (int t = 1; t < nthreads; ++t) workers.emplace_back(work);
        work();
        for (std::thread &t : workers) t.join();
    }
    size_t tot_rp = 0, tot_nz = 0, tot_h = 0, tot_dj = 0;
    for (int k = 0; k < count; ++k) {
        if (packed[(size_t)k].code != PHIA_OK)
            return cleanup(bfail(packed[(size_t)k].code, "%s", packed[(size_t)k].msg.c_str()));
        tot_rp += packed[(size_t)k].rp.size();
        tot_nz += packed[(size_t)k].col.size();
        tot_h += (size_t)d[k].N;
        if (packed[(size_t)k].small_op) tot_dj += (size_t)d[k].N * d[k].N;
    }
    std::vector<int32_t> rowptr, col, hk;
    std::vector<int8_t> val, dj;
    rowptr.reserve(tot_rp); col.reserve(tot_nz); val.reserve(tot_nz); hk.reserve(tot_h); dj.reserve(tot_dj);
    int64_t row_base = 0, nnz_real = 0;
    for (int k = 0; k < count; ++k) {
        const phia_instance_desc &x = d[k];
        PackedInst &pk = packed[(size_t)k];
        const int n = x.N;
        b->N.push_back(n);
        b->frac.push_back(x.frac_bits);
        b->inst_id.push_back(x.instance_id);
        b->h_off.push_back((int64_t)hk.size());
        b->targets.push_back(x.has_target ? (long long)x.target_k : LLONG_MIN);
        b->any_target |= x.has_target != 0;
        b->max_words = std::max<int>(b->max_words, (int)words_of(n));
        if (pk.small_op) {
            b->dense_pub.push_back(k);
            b->dense_joff.push_back((int64_t)dj.size());
            b->dense_op.push_back(pk.small_op);
            dj.insert(dj.end(), x.J_k, x.J_k + (size_t)n * n);
            hk.insert(hk.end(), x.h_k, x.h_k + n);
            continue;
        }
        b->csr_pub.push_back(k);
        CsrInst in{};
        in.N = n;
        in.inst_id = x.instance_id;
        in.q = ldexpf(1.0f, -x.frac_bits);
        in.rp_off = (int64_t)rowptr.size();
        in.nz_off = (int64_t)col.size();
        in.h_off = (int64_t)hk.size();
        in.row_base = row_base;
        rowptr.insert(rowptr.end(), pk.rp.begin(), pk.rp.end());
        col.insert(col.end(), pk.col.begin(), pk.col.end());
        val.insert(val.end(), pk.val.begin(), pk.val.end());
        nnz_real += pk.nnz_real;
        std::vector<int32_t>().swap(pk.rp);
        std::vector<int32_t>().swap(pk.col);
        std::vector<int8_t>().swap(pk.val);
        hk.insert(hk.end(), x.h_k, x.h_k + n);
        b->inst.push_back(in);
        for (int i0 = 0; i0 < n; i0 += 64) b->blocks.push_back(CsrBlock{(int32_t)(b->inst.size() - 1), i0});
        row_base += n;
    }
    b->total_rows = row_base;
    b->total_nnz = nnz_real;
    int dev_count = 0;
    if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count == 0)
        return cleanup(bfail(PHIA_ECUDA, "no CUDA device available"));
    if (o.device < 0 || o.device >= dev_count) return cleanup(bfail(PHIA_EINVAL, "device %d out of range", o.device));
    if (cudaSetDevice(o.device) != cudaSuccess) return cleanup(bfail(PHIA_ECUDA, "cudaSetDevice failed"));
    b->device = o.device;
    b->stream = (cudaStream_t)o.stream;
    bool ok = true;
    auto up = [&](void **dst, const void *src, size_t bytes) {
        if (!ok) return;
        if (cudaMalloc(dst, std::max<size_t>(bytes, 16)) != cudaSuccess) { ok = false; return; }
        if (bytes && cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) ok = false;
    };
    up((void **)&b->d_rowptr, rowptr.data(), rowptr.size() * 4);
    up((void **)&b->d_col, col.data(), col.size() * 4);
    up((void **)&b->d_val, val.data(), val.size());
    up((void **)&b->d_hk, hk.data(), hk.size() * 4);
    up((void **)&b->d_blocks, b->blocks.data(), b->blocks.size() * sizeof(CsrBlock));
    up((void **)&b->d_targets, b->targets.data(), b->targets.size() * sizeof(long long));
    up((void **)&b->d_dJ, dj.data(), dj.size());
    if (ok && cudaMalloc((void **)&b->d_inst, sizeof(CsrInst) * std::max<size_t>(b->inst.size(), 1)) != cudaSuccess)
        ok = false;
    if (ok && cudaMalloc((void **)&b->d_min_hit, 8) != cudaSuccess) ok = false;
    if (ok && cudaMalloc((void **)&b->d_start_ns, 8) != cudaSuccess) ok = false;
    if (ok && cudaMemset(b->d_start_ns, 0, 8) != cudaSuccess) ok = false;
    if (ok && cudaMalloc((void **)&b->d_iters, 8) != cudaSuccess) ok = false;
    if (ok && cudaMalloc((void **)&b->d_err, 4) != cudaSuccess) ok = false;
    if (ok && cudaMalloc((void **)&b->d_ctl, sizeof(IterCtl)) != cudaSuccess) ok = false;
    if (ok && cudaMalloc((void **)&b->d_sync, 4 * sizeof(unsigned)) != cudaSuccess) ok = false;
    if (ok) b->graphs = step_graphs_new();
    if (ok && (cudaEventCreate(&b->ev0) != cudaSuccess || cudaEventCreate(&b->ev1) != cudaSuccess)) ok = false;
    if (!ok) {
        cudaGetLastError();
        return cleanup(bfail(PHIA_ENOMEM, "device allocation or upload failed"));
    }
    *out = b;
    return PHIA_OK;
}

int batch_run(phia_batch_s *b, const phia_schedule *sched, int32_t R_real, int64_t t0, int64_t steps, int64_t total,
              uint64_t seed, const float *x_in, float *x_out, const float *v_in, float *v_out, int reset,
              const int8_t *spins_in, int32_t *field_out, int64_t *energy_out) {
    if (!b) return bfail(PHIA_EINVAL, "batch is NULL");
    const bool field_mode = spins_in != nullptr;
    if (!field_mode) {
        if (!sched) return bfail(PHIA_EINVAL, "schedule is NULL");
        if (!(sched->eps > 0.0f) || !(sched->gamma > 0.0f) || sched->refresh < 0 || (sched->deriv != 0 && sched->deriv != 1) ||
            sched->reserved != 0)
            return bfail(PHIA_EINVAL, "invalid schedule");
        if (sched->accept_test != 0)
            return bfail(PHIA_ENOTSUP, "schedule.accept_test = 1 runs on the resident tcgen05 and FP32 paths only");
        if (steps < 1 || t0 < 0 || total < t0 + steps) return bfail(PHIA_EINVAL, "need steps >= 1, t0 + steps <= total");
        if (total > ((int64_t)1 << 31)) return bfail(PHIA_ERANGE, "total_steps must be < 2^31");
    }
    if (R_real < 1) return bfail(PHIA_EINVAL, "replicas must be >= 1");
    const int R = round_up(R_real, 256);
    BCU(cudaSetDevice(b->device));
    if (!field_mode && !reset && (!b->ran || b->R_real != R_real))
        return bfail(PHIA_ESTATE, "reset_best = 0 needs a previous run with the same replica count");
    int rc = ensure_state(b, R);
    if (rc) return rc;
    b->R_real = R_real;
    layout(b, R);
    const int ncsr = (int)b->inst.size();
    if (field_mode && !b->dense_pub.empty()) return bfail(PHIA_ENOTSUP, "field-only runs take CSR instances");
    if ((x_in || x_out) && !b->dense_pub.empty())
        return bfail(PHIA_ENOTSUP, "runs from a given state take CSR instances");
    if (ncsr > 0)
        BCU(cudaMemcpyAsync(b->d_inst, b->inst.data(), sizeof(CsrInst) * ncsr, cudaMemcpyHostToDevice, b->stream));
    const int64_t reps = (int64_t)R * b->count;
    int64_t nbits = 0;
    for (int k = 0; k < b->count; ++k) nbits += (int64_t)R * words_of(b->N[k]);
    int launches = 0;
    if (reset && !field_mode) {
        const int64_t n = std::max(reps, nbits);
        batch_reset_records<<<(unsigned)((n + 255) / 256), 256, 0, b->stream>>>(
            reps, nbits, b->d_best_e, b->d_best_step, b->d_hit, b->d_bits, b->d_hit_ns, b->d_start_ns);
        BCU(cudaGetLastError());
        ++launches;
    }
    BCU(cudaMemsetAsync(b->d_min_hit, 0xFF, 8, b->stream));
    BCU(cudaMemsetAsync(b->d_iters, 0, 8, b->stream));
    BCU(cudaMemsetAsync(b->d_err, 0, 4, b->stream));
    CsrArgs C;
    memset(&C, 0, sizeof C);
    RunArgs &a = C.a;
    a.R = R;
    a.t0 = t0; a.nsteps = field_mode ? 1 : steps; a.T_total = field_mode ? 1 : total;
    if (!field_mode) {
        a.beta0 = sched->beta0; a.beta1 = sched->beta1; a.eps = sched->eps; a.gamma = sched->gamma;
        a.refresh = sched->refresh;
        a.deriv = sched->deriv;
        a.has_target = (sched->has_target || b->any_target) ? 1 : 0;
        a.stop_at_target = sched->stop_at_target;
        a.target = sched->target_k;
    }
    a.seed = seed;
    a.field_mode = field_mode ? 1 : 0;
    a.spins_in = spins_in; a.field_out = field_out; a.energy_out = energy_out;
    a.best_e = b->d_best_e; a.best_step = b->d_best_step; a.hit_step = b->d_hit;
    a.hit_ns = b->d_hit_ns;
    a.min_hit = b->d_min_hit; a.replica_iters = b->d_iters; a.err = b->d_err;
    C.inst = b->d_inst; C.count = ncsr;
    C.blocks = b->d_blocks; C.nblocks = (int32_t)b->blocks.size();
    C.row_ptr = b->d_rowptr; C.col = b->d_col; C.val = b->d_val; C.hk = b->d_hk;
    C.X = b->d_X; C.V = b->d_V;
    C.x_in = x_in; C.v_in = v_in; C.x_out = x_out; C.v_out = v_out;
    C.S = b->d_S;
    C.total_swords = b->total_rows * (R / 32);
    C.Esum = b->d_Esum; C.flags = b->d_flags; C.total_reps = reps;
    C.best_bits = b->d_bits;
    // per-instance targets: the instance's own, else the schedule's (CSR members, by CSR index)
    auto target_of = [&](int k) {
        return b->targets[(size_t)k] != LLONG_MIN ? b->targets[(size_t)k]
                                                  : (sched->has_target ? (long long)sched->target_k : LLONG_MIN);
    };
    if (!field_mode && (b->any_target) && ncsr > 0) {
        std::vector<long long> tg((size_t)ncsr);
        for (int c = 0; c < ncsr; ++c) tg[(size_t)c] = target_of(b->csr_pub[(size_t)c]);
        BCU(cudaMemcpyAsync(b->d_targets, tg.data(), tg.size() * sizeof(long long), cudaMemcpyHostToDevice, b->stream));
        BCU(cudaStreamSynchronize(b->stream));
        C.targets = b->d_targets;
    }
    C.R = R; C.R_real = R_real;
    C.max_words = b->max_words;
    C.total_rows = b->total_rows;
    // Small dense members: a table of CTAs (8 replicas each) per (operand, spin tiles)
    // group, every instance's own couplings, field, scale, Philox id, target and records.
    std::vector<std::pair<size_t, size_t>> groups;   // [begin, end) in small_host
    std::vector<std::pair<int, int>> group_key;      // (operand, spin tiles)
    std::vector<int> group_kpad;
    if (!b->dense_pub.empty()) {
        b->small_host.clear();
        for (int op : {kOpE4M3, kOpBF16})
            for (int mt = 1; mt <= 3; ++mt) {
                const size_t beg = b->small_host.size();
                int nmax = 0;
                for (size_t m = 0; m < b->dense_pub.size(); ++m) {
                    const int k = b->dense_pub[m], n = b->N[(size_t)k];
                    if (b->dense_op[m] != op || (n + 127) / 128 != mt) continue;
                    nmax = std::max(nmax, n);
                    for (int r0 = 0; r0 < R_real; r0 += 8) {
                        SmallCta c{};
                        c.Jk = b->d_dJ + b->dense_joff[m];
                        c.hk = b->d_hk + b->h_off[(size_t)k];
                        c.N = n;
                        c.W = (int32_t)words_of(n);
                        c.inst = b->inst_id[(size_t)k];
                        c.q = ldexpf(1.0f, -b->frac[(size_t)k]);
                        c.rbase = r0;
                        c.rec_off = (int64_t)k * R;
                        c.bits_off = b->bits_pub[(size_t)k];
                        c.target = target_of(k);
                        b->small_host.push_back(c);
                    }
                }
                if (b->small_host.size() > beg) {
                    groups.emplace_back(beg, b->small_host.size());
                    group_key.emplace_back(op, mt);
                    group_kpad.push_back(op == kOpE4M3 ? (nmax + 31) / 32 * 32 : (nmax + 15) / 16 * 16);
                }
            }
        if (b->small_host.size() > b->small_cap) {
            cudaFree(b->d_small);
            b->d_small = nullptr;
            if (cudaMalloc((void **)&b->d_small, b->small_host.size() * sizeof(SmallCta)) != cudaSuccess)
                return bfail(PHIA_ENOMEM, "CTA table allocation failed");
            b->small_cap = b->small_host.size();
        }
        BCU(cudaMemcpyAsync(b->d_small, b->small_host.data(), b->small_host.size() * sizeof(SmallCta),
                            cudaMemcpyHostToDevice, b->stream));
    }
    BCU(cudaEventRecord(b->ev0, b->stream));
    C.ctl = b->d_ctl;
    C.sync = b->d_sync;
    C.persistent = (b->csr_mode == 1 && !field_mode) ? 1 : 0;
    if (ncsr > 0) {
        cudaError_t e = launch_csr(C, b->graphs, b->stream, &launches);
        if (e != cudaSuccess) return bfail(PHIA_ECUDA, "kernel launch failed: %s", cudaGetErrorString(e));
    }
    for (size_t gi = 0; gi < groups.size(); ++gi) {
        RunArgs ad = a;
        ad.R = R_real;
        ad.best_bits = b->d_bits;        // the CSR path keeps its best states in C.best_bits
        if (!ad.best_e || !ad.best_step || !ad.hit_step || !ad.hit_ns || !ad.best_bits || !ad.replica_iters || !ad.err)
            return bfail(PHIA_ECUDA, "internal: a record array of the dense launch is missing");
        ad.small_cta = b->d_small + groups[gi].first;
        ad.small_ctas = (int32_t)(groups[gi].second - groups[gi].first);
        ad.has_target = b->any_target || sched->has_target;
        cudaError_t e = launch_tc_small_batch(ad, group_key[gi].first, group_key[gi].second, group_kpad[gi], b->stream);
        if (e != cudaSuccess) return bfail(PHIA_ECUDA, "kernel launch failed: %s", cudaGetErrorString(e));
        ++launches;
    }
    BCU(cudaEventRecord(b->ev1, b->stream));
    if (!field_mode) {
        b->ran = true;
        b->R = R;
        b->last_steps = steps;
        b->last_launches = launches;
        b->last_stop = sched->stop_at_target;
    }
    return PHIA_OK;
}

// Per-replica records of one instance (first R_real replicas).
int batch_records(phia_batch_s *b, int inst, std::vector<int64_t> &be, std::vector<int64_t> &bs,
                  std::vector<int64_t> &hs) {
    if (!b->ran) return bfail(PHIA_ESTATE, "no run on this batch yet");
    if (inst < 0 || inst >= b->count) return bfail(PHIA_EINVAL, "instance %d out of range", inst);
    BCU(cudaSetDevice(b->device));
    BCU(cudaStreamSynchronize(b->stream));
    int32_t err = 0;
    BCU(cudaMemcpy(&err, b->d_err, 4, cudaMemcpyDeviceToHost));
    if (err) return bfail(PHIA_ETIMEOUT, "a bounded device wait expired during the run");
    const int n = b->R_real;
    const size_t off = (size_t)inst * b->R;
    be.resize(n); bs.resize(n); hs.resize(n);
    BCU(cudaMemcpy(be.data(), b->d_best_e + off, (size_t)n * 8, cudaMemcpyDeviceToHost));
    BCU(cudaMemcpy(bs.data(), b->d_best_step + off, (size_t)n * 8, cudaMemcpyDeviceToHost));
    BCU(cudaMemcpy(hs.data(), b->d_hit + off, (size_t)n * 8, cudaMemcpyDeviceToHost));
    return PHIA_OK;
}

int batch_pick(const phia_batch_s *b, const std::vector<int64_t> &be, const std::vector<int64_t> &bs,
               const std::vector<int64_t> &hs) {
    int best = -1;
    if (b->last_stop) {
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

int batch_bits(phia_batch_s *b, int inst, int r, uint32_t *dst, int nreps) {
    // bits of replicas r .. r+nreps-1 of one instance
    int64_t off = 0;
    for (int k = 0; k < inst; ++k) off += (int64_t)b->R * words_of(b->N[k]);
    const int64_t W = words_of(b->N[inst]);
    BCU(cudaMemcpy(dst, b->d_bits + off + (int64_t)r * W, (size_t)nreps * W * 4, cudaMemcpyDeviceToHost));
    return PHIA_OK;
}

int batch_best(phia_batch_s *b, int inst, int64_t *energy_k, int8_t *spins) {
    std::vector<int64_t> be, bs, hs;
    int rc = batch_records(b, inst, be, bs, hs);
    if (rc) return rc;
    const int r = batch_pick(b, be, bs, hs);
    if (r < 0) return bfail(PHIA_ESTATE, "no replica recorded a state");
    if (energy_k) *energy_k = be[r];
    if (spins) {
        const int n = b->N[inst];
        std::vector<uint32_t> w(words_of(n));
        rc = batch_bits(b, inst, r, w.data(), 1);
        if (rc) return rc;
        for (int i = 0; i < n; ++i) spins[i] = ((w[i >> 5] >> (i & 31)) & 1u) ? 1 : -1;
    }
    return PHIA_OK;
}

int batch_replica_results(phia_batch_s *b, int inst, int32_t R, int64_t *be_out, int64_t *bs_out, int64_t *hs_out,
                          uint32_t *bits_out) {
    std::vector<int64_t> be, bs, hs;
    int rc = batch_records(b, inst, be, bs, hs);
    if (rc) return rc;
    if (R != b->R_real) return bfail(PHIA_EINVAL, "replicas (%d) differs from the last run (%d)", R, b->R_real);
    if (be_out) memcpy(be_out, be.data(), (size_t)R * 8);
    if (bs_out) memcpy(bs_out, bs.data(), (size_t)R * 8);
    if (hs_out) memcpy(hs_out, hs.data(), (size_t)R * 8);
    if (bits_out) return batch_bits(b, inst, 0, bits_out, R);
    return PHIA_OK;
}

int batch_stats(phia_batch_s *b, int inst, phia_stats *out) {
    if (!out) return bfail(PHIA_EINVAL, "NULL argument");
    memset(out, 0, sizeof *out);
    std::vector<int64_t> be, bs, hs;
    int rc = batch_records(b, inst < 0 ? 0 : inst, be, bs, hs);
    if (rc) return rc;
    unsigned long long iters = 0;
    BCU(cudaMemcpy(&iters, b->d_iters, 8, cudaMemcpyDeviceToHost));
    float ms = 0.f;
    BCU(cudaEventElapsedTime(&ms, b->ev0, b->ev1));
    int64_t spins_total = 0;
    for (int k = 0; k < b->count; ++k) spins_total += b->N[k];
    out->replicas = b->R_real;
    out->steps = b->last_steps;
    // padded replicas excluded: every instance runs R_real real replicas
    out->spin_updates = (int64_t)b->R_real * b->last_steps * (inst < 0 ? spins_total : b->N[inst]);
    const int r = batch_pick(b, be, bs, hs);
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
        BCU(cudaMemcpy(&t_hit, b->d_hit_ns + (size_t)(inst < 0 ? 0 : inst) * b->R + out->hit_replica, 8,
                       cudaMemcpyDeviceToHost));
        BCU(cudaMemcpy(&t_start, b->d_start_ns, 8, cudaMemcpyDeviceToHost));
        if (t_hit >= t_start && t_start != 0) out->hit_ns = (int64_t)(t_hit - t_start);
    }
    out->device_ms = ms;
    out->path = b->inst.empty() ? PHIA_PATH_TC : PHIA_PATH_CSR;   // the sparse path whenever it runs
    out->kernel_launches = b->last_launches;
    (void)iters;
    return PHIA_OK;
}

}  // namespace phia

extern "C" {

int phia_batch_create(phia_batch_t **out, int32_t count, const phia_instance_desc *descs, const phia_opts *opts) {
    return batch_create(out, count, descs, opts);
}

int phia_batch_anneal(phia_batch_t *b, const phia_schedule *sched, int32_t replicas, int64_t steps, uint64_t seed) {
    return batch_run(b, sched, replicas, 0, steps, steps, seed, nullptr, nullptr, nullptr, nullptr, 1, nullptr, nullptr,
                     nullptr);
}

int phia_batch_best(phia_batch_t *b, int32_t instance, int64_t *energy_k, int8_t *spins) {
    if (!b) return bfail(PHIA_EINVAL, "batch is NULL");
    return batch_best(b, instance, energy_k, spins);
}

int phia_batch_replica_results(phia_batch_t *b, int32_t instance, int32_t replicas, int64_t *best_energy_k,
                               int64_t *best_step, int64_t *hit_step, uint32_t *best_bits) {
    if (!b) return bfail(PHIA_EINVAL, "batch is NULL");
    return batch_replica_results(b, instance, replicas, best_energy_k, best_step, hit_step, best_bits);
}

int phia_batch_stats_get(phia_batch_t *b, phia_stats *out) {
    if (!b) return bfail(PHIA_EINVAL, "batch is NULL");
    return batch_stats(b, -1, out);
}

int phia_batch_autotune(phia_batch_t *b, const phia_schedule *sched, int32_t replicas, int32_t probe_iters,
                        phia_tune_result *out) {
    if (!b || !sched) return bfail(PHIA_EINVAL, "NULL argument");
    if (replicas < 1 || probe_iters < 1) return bfail(PHIA_EINVAL, "need replicas >= 1 and probe_iters >= 1");
    float best_ms = 1e30f, worst_ms = 0.f;
    int best_mode = b->csr_mode;
    const int saved = b->csr_mode;
    for (int mode : {1, 2}) {
        b->csr_mode = mode;
        float ms = 0.f;
        for (int rep = 0; rep < 2; ++rep) {   // the first run warms up
            int rc = batch_run(b, sched, replicas, 0, probe_iters, probe_iters, 1, nullptr, nullptr, nullptr, nullptr, 1,
                               nullptr, nullptr, nullptr);
            if (rc) { b->csr_mode = saved; return rc; }
            BCU(cudaEventSynchronize(b->ev1));
            BCU(cudaEventElapsedTime(&ms, b->ev0, b->ev1));
        }
        if (ms < best_ms) { best_ms = ms; best_mode = mode; }
        worst_ms = std::max(worst_ms, ms);
    }
    b->csr_mode = best_mode;
    if (out) {
        memset(out, 0, sizeof *out);
        out->tc_kernel = best_mode;
        out->candidates = 2;
        out->best_us_per_iter = 1000.f * best_ms / probe_iters;
        out->worst_us_per_iter = 1000.f * worst_ms / probe_iters;
    }
    return PHIA_OK;
}

int phia_batch_sync(phia_batch_t *b) {
    if (!b) return bfail(PHIA_EINVAL, "batch is NULL");
    BCU(cudaSetDevice(b->device));
    BCU(cudaStreamSynchronize(b->stream));
    return PHIA_OK;
}

void phia_batch_destroy(phia_batch_t *b) {
    if (!b) return;
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    free_state(b);
    cudaFree(b->d_inst); cudaFree(b->d_blocks); cudaFree(b->d_rowptr); cudaFree(b->d_col); cudaFree(b->d_val);
    cudaFree(b->d_hk); cudaFree(b->d_targets); cudaFree(b->d_min_hit); cudaFree(b->d_start_ns); cudaFree(b->d_iters); cudaFree(b->d_err);
    cudaFree(b->d_dJ); cudaFree(b->d_small); cudaFree(b->d_sync);
    cudaFree(b->d_ctl);
    step_graphs_free(b->graphs);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    delete b;
}

}  // extern "C"
