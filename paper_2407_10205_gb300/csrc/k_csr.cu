// k_csr.cu -- sparse PHIA path: many instances of uneven N in one launch per iteration,
// the field I = J s + h (Eq. 6) gathered warp-per-row from CSR couplings over
// bit-packed spins, fused with the update of Eqs. 5, 8 and A7.
//
// Layout per instance b (N_b spins, R replicas, R a multiple of 256):
//   spins   4 rotating buffers of uint32 [N_b][R/32]: bit r%32 of word r/32 of row j is
//           (s_j of replica r = +1); iteration t reads buffer t%4, writes t+1%4.
//   x, v    float32 [N_b][R] (spin-major, so a row's 256 replicas are 1 KB contiguous)
//   best    uint32 [R][ceil(N_b/32)] bit-packed over spins (as on every path)
// Work unit: a block of 64 consecutive rows of one instance and 256 replicas; a warp
// takes 8 rows, a lane 8 replicas (one byte of each spin row).
// For a row i and its entries (j, k): acc_r = sum k [s_j^r = +1], ksum = sum k, so
// I_r = 2 acc_r - ksum + kh_i (exact integers).  Energy partials s_i (I_i + h_i) are
// reduced per block in shared memory and added to a per-(instance, replica) int64 sum.
// Records are lagged as in the dense per-iteration kernel: the launch for iteration t
// settles t-1 (block 0 of each instance) and copies the spins of t-2 for the replicas
// that improved then (every block, its 64 rows).
#include <algorithm>

#include "device_common.cuh"
#include "phia_internal.h"

namespace phia {

namespace {

constexpr int kRowsPerBlock = 64;
constexpr int kWarps = 8;
constexpr int kRowsPerWarp = kRowsPerBlock / kWarps;
constexpr int kGroup = 256;          // replicas per block (8 per lane)

__device__ __forceinline__ void settle_csr(const CsrArgs &C, const CsrInst &in, int b, int r, int64_t tt) {
    const RunArgs &a = C.a;
    const size_t rec = (size_t)in.rec_off + r;
    unsigned long long *slot =
        reinterpret_cast<unsigned long long *>(C.Esum) + (size_t)(tt & 1) * C.total_reps + rec;
    const long long twice = (long long)*slot;
    *slot = 0ull;
    const long long E = -twice / 2;
    int imp = 0;
    const bool frozen = a.stop_at_target && a.hit_step[rec] >= 0;
    if (!frozen && E < a.best_e[rec]) {
        a.best_e[rec] = E;
        a.best_step[rec] = tt;
        imp = 1;
    }
    const long long target = C.targets ? C.targets[b] : a.target;
    if (a.has_target && a.hit_step[rec] < 0 && E <= target) {
        a.hit_step[rec] = tt;
        if (a.hit_ns) a.hit_ns[rec] = globaltimer_ns();
    }
    C.flags[(size_t)(tt & 1) * C.total_reps + rec] = (int8_t)imp;
    (void)b;
}

__device__ __forceinline__ const uint32_t *spin_buf(const CsrArgs &C, const CsrInst &in, int64_t tt) {
    return C.S + (size_t)(tt & 3) * C.total_swords + in.s_off;
}

// One work unit of iteration t: 64 rows (block `bi` of the list) x 256 replicas (group g).
// Uses the block's shared arrays; every thread of the block calls it.
__device__ __forceinline__ void csr_unit(const CsrArgs &C, int bi, int g, int64_t t, int64_t t_first, int64_t t_end,
                                         int32_t (*part)[kGroup], uint32_t (*sbits)[kGroup / 32]) {
    const RunArgs &a = C.a;
    const CsrBlock blk = C.blocks[bi];
    const CsrInst in = C.inst[blk.inst];
    const int b = blk.inst;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int N = in.N, R = C.R, RW = R / 32;

    // (a) records of iteration t-1 (block 0 of each instance).
    if (blk.i0 == 0 && t - 1 >= t_first) settle_csr(C, in, b, g * kGroup + tid, t - 1);
    // (b) best spins of iteration t-2 for the replicas that improved then: this block's
    //     64 rows of spin bits go through shared memory, one thread per replica.
    if (t - 2 >= t_first) {
        const int rows = min(kRowsPerBlock, N - blk.i0);
        const uint32_t *Sb = spin_buf(C, in, t - 2);
        for (int e = tid; e < kRowsPerBlock * 8; e += 32 * kWarps) {
            const int row = e >> 3, w = e & 7;
            sbits[row][w] = row < rows ? Sb[(size_t)(blk.i0 + row) * RW + g * 8 + w] : 0u;
        }
        __syncthreads();
        const int r = g * kGroup + tid;
        if (C.flags[(size_t)((t - 2) & 1) * C.total_reps + in.rec_off + r]) {
            const int W = (N + 31) / 32;
            uint32_t w0 = 0, w1 = 0;
            for (int row = 0; row < 32; ++row) w0 |= ((sbits[row][tid >> 5] >> (tid & 31)) & 1u) << row;
            for (int row = 32; row < 64; ++row) w1 |= ((sbits[row][tid >> 5] >> (tid & 31)) & 1u) << (row - 32);
            uint32_t *dst = C.best_bits + in.bits_off + (size_t)r * W;
            const int word = blk.i0 / 32;
            dst[word] = w0;
            if (word + 1 < W) dst[word + 1] = w1;
        }
    }

    // (c) field and update, 8 rows per warp, 8 replicas per lane.
    const uint8_t *Scur = reinterpret_cast<const uint8_t *>(spin_buf(C, in, t));
    uint32_t *Snext = const_cast<uint32_t *>(spin_buf(C, in, t + 1));
    const float bgq = beta_at(t, inv_tm1_of(a.T_total), a.beta0, a.beta1) * (a.gamma * in.q);
    const float eps = a.eps, gamma = a.gamma;
    const bool more = t + 1 < t_end;
    const bool refresh_next = more && refresh_at(t + 1, a.refresh);
    const int r0 = g * kGroup + lane * 8;          // first replica of this lane
    int32_t epart[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int q = 0; q < kRowsPerWarp; ++q) {
        const int i = blk.i0 + warp * kRowsPerWarp + q;
        if (i >= N) break;
        const int p_beg = C.row_ptr[in.rp_off + i], p_end = C.row_ptr[in.rp_off + i + 1];
        // acc_r = sum_j k_j [s_j^r = +1] for this lane's 8 replicas r.  Rows are padded to
        // multiples of 8 entries (k = 0), so the warp reads 8 columns and 8 couplings at
        // a time with broadcast vector loads.  The spin bytes of 4 neighbours form one
        // word B; (B >> r) & 0x01010101 holds replica r's four bits, one per byte, and a
        // 4-way int8 dot product with the four couplings adds k [s = +1] for all four.
        const int32_t *colp = C.col + in.nz_off;
        const int8_t *valp = C.val + in.nz_off;
        const uint8_t *Sl = Scur + g * 32 + lane;     // this lane's byte of spin row 0
        const size_t rowb = (size_t)RW * 4;           // bytes per spin row
        int32_t acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        int32_t ksum = 0;
        // The next round's columns and couplings load while this round's spins do.
        int4 c0n = make_int4(0, 0, 0, 0), c1n = c0n;
        int2 kkn = make_int2(0, 0);
        if (p_beg < p_end) {
            c0n = *reinterpret_cast<const int4 *>(colp + p_beg);
            c1n = *reinterpret_cast<const int4 *>(colp + p_beg + 4);
            kkn = *reinterpret_cast<const int2 *>(valp + p_beg);
        }
        for (int p = p_beg; p < p_end; p += 8) {
            const int4 c0 = c0n, c1 = c1n;
            const int2 kk = kkn;
            if (p + 8 < p_end) {
                c0n = *reinterpret_cast<const int4 *>(colp + p + 8);
                c1n = *reinterpret_cast<const int4 *>(colp + p + 12);
                kkn = *reinterpret_cast<const int2 *>(valp + p + 8);
            }
            const uint32_t s0 = Sl[(size_t)c0.x * rowb], s1 = Sl[(size_t)c0.y * rowb];
            const uint32_t s2 = Sl[(size_t)c0.z * rowb], s3 = Sl[(size_t)c0.w * rowb];
            const uint32_t s4 = Sl[(size_t)c1.x * rowb], s5 = Sl[(size_t)c1.y * rowb];
            const uint32_t s6 = Sl[(size_t)c1.z * rowb], s7 = Sl[(size_t)c1.w * rowb];
            const uint32_t B0 = __byte_perm(__byte_perm(s0, s1, 0x0040), __byte_perm(s2, s3, 0x0040), 0x5410);
            const uint32_t B1 = __byte_perm(__byte_perm(s4, s5, 0x0040), __byte_perm(s6, s7, 0x0040), 0x5410);
            ksum = __dp4a(kk.x, 0x01010101, ksum);
            ksum = __dp4a(kk.y, 0x01010101, ksum);
#pragma unroll
            for (int rr = 0; rr < 8; ++rr) {
                acc[rr] = __dp4a((int)((B0 >> rr) & 0x01010101u), kk.x, acc[rr]);
                acc[rr] = __dp4a((int)((B1 >> rr) & 0x01010101u), kk.y, acc[rr]);
            }
        }
        const int32_t hk = C.hk[in.h_off + i];
        const size_t xo = in.x_off + (size_t)i * R + r0;
        float4 xa = *reinterpret_cast<const float4 *>(C.X + xo);
        float4 xb = *reinterpret_cast<const float4 *>(C.X + xo + 4);
        float4 va = *reinterpret_cast<const float4 *>(C.V + xo);
        float4 vb = *reinterpret_cast<const float4 *>(C.V + xo + 4);
        float xs[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
        float vs[8] = {va.x, va.y, va.z, va.w, vb.x, vb.y, vb.z, vb.w};
        uint32_t nbyte = 0;
        float If[8];
#pragma unroll
        for (int rr = 0; rr < 8; ++rr) {
            const int32_t I = 2 * acc[rr] - ksum + hk;                    // Eq. 6, exact
            epart[rr] += (xs[rr] >= 0.0f ? 1 : -1) * (I + hk);
            If[rr] = (float)I;
        }
        float vn[8];
        if (a.deriv == 1) {
#pragma unroll
            for (int rr = 0; rr < 8; ++rr) vn[rr] = momentum_quad(vs[rr], xs[rr], If[rr], eps, bgq, gamma);
        } else {
#pragma unroll
            for (int rr = 0; rr < 8; ++rr) vn[rr] = momentum_exact(vs[rr], xs[rr], If[rr], eps, bgq, gamma);
        }
#pragma unroll
        for (int rr = 0; rr < 8; ++rr) {
            float v = vn[rr];
            float x = xs[rr];
            if (more) {
                if (refresh_next) v = draw_v(a.seed, in.inst_id, (uint32_t)(r0 + rr), (uint32_t)i, (uint32_t)(t + 1));
                x = x + eps * v;
            }
            xs[rr] = x;
            vs[rr] = v;
            nbyte |= (uint32_t)(x >= 0.0f) << rr;
        }
        if (more) {
            *reinterpret_cast<float4 *>(C.X + xo) = make_float4(xs[0], xs[1], xs[2], xs[3]);
            *reinterpret_cast<float4 *>(C.X + xo + 4) = make_float4(xs[4], xs[5], xs[6], xs[7]);
            reinterpret_cast<uint8_t *>(Snext)[(size_t)i * (RW * 4) + g * 32 + lane] = (uint8_t)nbyte;
        }
        *reinterpret_cast<float4 *>(C.V + xo) = make_float4(vs[0], vs[1], vs[2], vs[3]);
        *reinterpret_cast<float4 *>(C.V + xo + 4) = make_float4(vs[4], vs[5], vs[6], vs[7]);
    }
#pragma unroll
    for (int rr = 0; rr < 8; ++rr) part[warp][lane * 8 + rr] = epart[rr];
    __syncthreads();
    {
        long long s = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) s += part[w][tid];
        atomicAdd(reinterpret_cast<unsigned long long *>(C.Esum) + (size_t)(t & 1) * C.total_reps + in.rec_off +
                      g * kGroup + tid,
                  (unsigned long long)s);
    }
    __syncthreads();   // the shared arrays are free for the next unit
}

// One launch per iteration: a block per work unit; the iteration comes from C.ctl.
__global__ void __launch_bounds__(32 * kWarps, 4) csr_step(const CsrArgs C) {
    __shared__ int32_t part[kWarps][kGroup];
    __shared__ uint32_t sbits[kRowsPerBlock][kGroup / 32];
    const int64_t t = C.ctl->t, t_first = C.ctl->t_first, t_end = C.ctl->t_end;
    csr_unit(C, blockIdx.x, blockIdx.y, t, t_first, t_end, part, sbits);
    if (threadIdx.x == 0) iter_ctl_finish(C.ctl);
}

// Grid-wide barrier of a cooperative launch (every block resident): bar[0] counts the
// blocks arrived, bar[1] is the generation.  The wait is bounded; false when it expired.
__device__ bool grid_barrier(unsigned *bar, uint64_t timeout_ns) {
    __syncthreads();
    int ok = 1;
    if (threadIdx.x == 0) {
        volatile unsigned *gen = bar + 1;
        const unsigned g0 = *gen;
        __threadfence();
        if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const uint64_t t_start = globaltimer_ns();
            while (*gen == g0) {
                if (globaltimer_ns() - t_start > timeout_ns) { ok = 0; break; }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    return __syncthreads_and(ok) != 0;
}

// All iterations of the run in one cooperative launch: per iteration every block takes
// work units from a counter (units of uneven cost balance themselves), then the grid
// meets at a barrier.  ctr[t & 1] hands out iteration t's units; the last block to reach
// the barrier after iteration t clears it for t + 2.
__global__ void __launch_bounds__(32 * kWarps, 4) csr_persistent(const CsrArgs C, unsigned *bar, unsigned *ctr) {
    __shared__ int32_t part[kWarps][kGroup];
    __shared__ uint32_t sbits[kRowsPerBlock][kGroup / 32];
    __shared__ int unit;
    const int64_t t_first = C.a.t0, t_end = C.a.t0 + C.a.nsteps;
    const int groups = C.R / kGroup, units = C.nblocks * groups;
    for (int64_t t = t_first; t < t_end; ++t) {
        for (;;) {
            if (threadIdx.x == 0) unit = (int)atomicAdd(&ctr[t & 1], 1u);
            __syncthreads();
            const int u = unit;
            __syncthreads();
            if (u >= units) break;
            csr_unit(C, u % C.nblocks, u / C.nblocks, t, t_first, t_end, part, sbits);
        }
        // The counter of iteration t is cleared once every block has left it: the barrier
        // below waits for all; block 0 clears it after the barrier, before iteration t + 2.
        if (!grid_barrier(bar, kWaitTimeoutNs)) {
            if (threadIdx.x == 0) atomicExch(C.a.err, 1);
            return;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) ctr[t & 1] = 0u;
    }
}

// Initial state (or given, [R][N] per instance), refresh at t0, first position update,
// spins of iteration t0.  One thread per (instance-spin row, lane of 8 replicas).
__global__ void csr_prologue(const CsrArgs C) {
    const RunArgs &a = C.a;
    const int64_t gidx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // over total_rows * R / 8
    if (gidx == 0) iter_ctl_start(C.ctl, a.t0, a.nsteps);
    const int R = C.R, per_row = R / 8;
    const int64_t row = gidx / per_row;
    if (row >= C.total_rows) return;
    const int l8 = (int)(gidx - row * per_row);
    // find the instance of this global row (rows are stored instance after instance)
    int lo = 0, hi = C.count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (C.inst[mid].row_base <= row) lo = mid; else hi = mid - 1;
    }
    const CsrInst in = C.inst[lo];
    const int i = (int)(row - in.row_base);
    uint32_t byte = 0;
    for (int rr = 0; rr < 8; ++rr) {
        const int r = l8 * 8 + rr;
        float x, v;
        if (C.x_in && r < C.R_real) {
            x = C.x_in[in.xin_off + (size_t)r * in.N + i];
            v = C.v_in[in.xin_off + (size_t)r * in.N + i];
        } else {
            const U4 o = draw_raw(a.seed, in.inst_id, (uint32_t)r, (uint32_t)i, 0u);
            x = box_muller(o.x, o.y);
            v = box_muller(o.z, o.w);
        }
        if (refresh_at(a.t0, a.refresh)) v = draw_v(a.seed, in.inst_id, (uint32_t)r, (uint32_t)i, (uint32_t)a.t0);
        x = x + a.eps * v;
        C.X[in.x_off + (size_t)i * R + r] = x;
        C.V[in.x_off + (size_t)i * R + r] = v;
        byte |= (uint32_t)(x >= 0.0f) << rr;
    }
    uint8_t *S = reinterpret_cast<uint8_t *>(const_cast<uint32_t *>(spin_buf(C, in, a.t0)));
    S[(size_t)i * (R / 8) + l8] = (uint8_t)byte;
}

// Final state back to [R][N] per instance (caller layout).
__global__ void csr_export(const CsrArgs C) {
    const int64_t gidx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // over total_rows * R
    const int R = C.R;
    const int64_t row = gidx / R;
    if (row >= C.total_rows) return;
    const int r = (int)(gidx - row * R);
    int lo = 0, hi = C.count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (C.inst[mid].row_base <= row) lo = mid; else hi = mid - 1;
    }
    const CsrInst in = C.inst[lo];
    const int i = (int)(row - in.row_base);
    if (r >= C.R_real) return;
    C.x_out[in.xin_off + (size_t)r * in.N + i] = C.X[in.x_off + (size_t)i * R + r];
    C.v_out[in.xin_off + (size_t)r * in.N + i] = C.V[in.x_off + (size_t)i * R + r];
}

__global__ void csr_settle_all(const CsrArgs C, int64_t tt) {
    const int b = blockIdx.x;
    const CsrInst in = C.inst[b];
    for (int r = threadIdx.x; r < C.R; r += blockDim.x) settle_csr(C, in, b, r, tt);
}

// Copies for iterations not handled by a later launch; one thread per (replica, word).
__global__ void csr_copy_all(const CsrArgs C, int64_t t_from, int64_t t_last) {
    const int b = blockIdx.y;
    const CsrInst in = C.inst[b];
    const int W = (in.N + 31) / 32;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)C.R * W) return;
    const int r = (int)(idx / W), w = (int)(idx - (int64_t)r * W);
    for (int64_t tt = t_from; tt <= t_last; ++tt) {
        if (!C.flags[(size_t)(tt & 1) * C.total_reps + in.rec_off + r]) continue;
        const uint32_t *Sb = spin_buf(C, in, tt);
        uint32_t bits = 0;
        for (int q = 0; q < 32; ++q) {
            const int i = w * 32 + q;
            if (i < in.N && ((Sb[(size_t)i * (C.R / 32) + (r >> 5)] >> (r & 31)) & 1u)) bits |= 1u << q;
        }
        C.best_bits[in.bits_off + (size_t)r * W + w] = bits;
    }
}

// Field only: spins given as int8 [R][N] per instance -> field int32 [R][N], energy [R].
__global__ void csr_field_only(const CsrArgs C) {
    const RunArgs &a = C.a;
    const int64_t gidx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // over total_rows * R
    const int R = C.R;
    const int64_t row = gidx / R;
    if (row >= C.total_rows) return;
    const int r = (int)(gidx - row * R);
    int lo = 0, hi = C.count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (C.inst[mid].row_base <= row) lo = mid; else hi = mid - 1;
    }
    const CsrInst in = C.inst[lo];
    const int i = (int)(row - in.row_base);
    if (r >= C.R_real) return;
    const int8_t *s = a.spins_in + in.xin_off + (size_t)r * in.N;
    int32_t I = C.hk[in.h_off + i];
    for (int p = C.row_ptr[in.rp_off + i]; p < C.row_ptr[in.rp_off + i + 1]; ++p)
        I += (int32_t)C.val[in.nz_off + p] * s[C.col[in.nz_off + p]];
    if (a.field_out) a.field_out[in.xin_off + (size_t)r * in.N + i] = I;
    atomicAdd(reinterpret_cast<unsigned long long *>(C.Esum) + in.rec_off + r,
              (unsigned long long)(long long)(s[i] * (I + C.hk[in.h_off + i])));
}

__global__ void csr_field_energy(const CsrArgs C) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= C.total_reps) return;
    unsigned long long *slot = reinterpret_cast<unsigned long long *>(C.Esum) + idx;
    const int b = (int)(idx / C.R), r = (int)(idx - (int64_t)b * C.R);
    if (C.a.energy_out && r < C.R_real) C.a.energy_out[(size_t)b * C.R_real + r] = -((long long)*slot) / 2;
    *slot = 0ull;
}

__global__ void csr_count(const CsrArgs C) {
    if (threadIdx.x == 0 && blockIdx.x == 0)
        atomicAdd(C.a.replica_iters, (unsigned long long)((long long)C.total_reps * C.a.nsteps));
}

}  // namespace

cudaError_t launch_csr(const CsrArgs &Cin, StepGraphCache *graphs, cudaStream_t st, int *launches) {
    const CsrArgs &C = Cin;
    int n = 0;
    cudaError_t e = cudaMemsetAsync(C.Esum, 0, 2 * (size_t)C.total_reps * sizeof(int64_t), st);
    if (e != cudaSuccess) return e;
    if (C.a.field_mode) {
        const int64_t work = C.total_rows * C.R;
        csr_field_only<<<(unsigned)((work + 255) / 256), 256, 0, st>>>(C);
        csr_field_energy<<<(unsigned)((C.total_reps + 255) / 256), 256, 0, st>>>(C);
        if (launches) *launches += 2;
        return cudaGetLastError();
    }
    const int64_t pw = C.total_rows * (C.R / 8);
    csr_prologue<<<(unsigned)((pw + 255) / 256), 256, 0, st>>>(C);
    ++n;
    const dim3 grid(C.nblocks, C.R / kGroup);
    if (C.persistent) {
        // Every iteration in one cooperative launch: as many blocks as can be resident.
        int per_sm = 0, dev = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, csr_persistent, 32 * kWarps, 0);
        if (e == cudaSuccess) e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        const int units = C.nblocks * (C.R / kGroup);
        const unsigned blocks = (unsigned)std::max(1, std::min(units, per_sm * sms));
        e = cudaMemsetAsync(C.sync, 0, 4 * sizeof(unsigned), st);
        if (e != cudaSuccess) return e;
        CsrArgs Cp = C;
        Cp.x_in = Cp.v_in = nullptr;
        Cp.x_out = Cp.v_out = nullptr;
        unsigned *bar = C.sync, *ctr = C.sync + 2;
        void *args[3] = {&Cp, &bar, &ctr};
        e = cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(csr_persistent), dim3(blocks),
                                        dim3(32 * kWarps), args, 0, st);
        if (e != cudaSuccess) return e;
        ++n;
    } else {
        // The step kernel reads its iteration from C.ctl: every launch is the same, and
        // the arguments leave out what only the prologue and the export read.
        CsrArgs Cs = C;
        Cs.a.t0 = 0;
        Cs.a.nsteps = 0;
        Cs.x_in = Cs.v_in = nullptr;
        Cs.x_out = Cs.v_out = nullptr;
        void *args[1] = {&Cs};
        e = launch_steps(graphs, reinterpret_cast<const void *>(csr_step), grid, dim3(32 * kWarps), 0, args, &Cs,
                         sizeof Cs, C.a.nsteps, st);
        if (e != cudaSuccess) return e;
        n += (int)C.a.nsteps;
    }
    const int64_t t_last = C.a.t0 + C.a.nsteps - 1;
    csr_settle_all<<<C.count, 256, 0, st>>>(C, t_last);
    const dim3 cg((unsigned)(((int64_t)C.R * C.max_words + 255) / 256), C.count);
    csr_copy_all<<<cg, 256, 0, st>>>(C, t_last - 1 >= C.a.t0 ? t_last - 1 : t_last, t_last);
    csr_count<<<1, 32, 0, st>>>(C);
    n += 3;
    if (C.x_out) {
        const int64_t work = C.total_rows * C.R;
        csr_export<<<(unsigned)((work + 255) / 256), 256, 0, st>>>(C);
        ++n;
    }
    if (launches) *launches += n;
    return cudaGetLastError();
}

}  // namespace phia
