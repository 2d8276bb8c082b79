// k_tc_small.cu -- tensor-core PHIA kernel for small dense instances (N <= 384 with
// e4m3 operands, N <= 256 with bf16), all iterations in one launch.
//
// One CTA owns 16 replicas of one instance for the whole run:
//  - A = the couplings k (Eq. 6's J in units of q), re-encoded exactly as e4m3 or
//    bf16, resident in shared memory for the whole run ([M = output spin][K = input spin]);
//  - B = the 16 replicas' spins s = sgn x, written by the epilogue straight into
//    shared memory in the MMA's operand layout ([N = replica][K = spin]);
//  - D = J s (integer-valued FP32 in TMEM: lane = output spin, column = replica).
//    Every product is an integer and every partial sum stays below 2^24 in
//    magnitude, so FP32 accumulation is exact and the field is an exact int32.
//  - x and v (FP32) stay in registers: thread (spin i, 8 replicas) for the whole run.
// Per iteration (Eq. A7): MMA -> field I = D + h (Eq. 6) -> energy
// E = -1/2 sum s (I + h) (Eq. 2) -> v update (Eqs. 5, 8) -> optional momentum refresh
// -> x update and sign of the next iteration, written into B -> best-state keeping
// (Table 3, state 5).
#include <algorithm>

#include <cuda_fp8.h>
#include <cuda_bf16.h>

#include "device_common.cuh"
#include "phia_internal.h"

namespace phia {

namespace {

constexpr int kNB = 16;  // MMA N: replica columns per CTA (live ones first, the rest zero)

constexpr int kMaxWarps = 48;   // 4 lane quadrants x up to 3 output tiles x up to 4 replica splits
constexpr int kMaxRPT = 8;

struct SmallShared {
    uint64_t mbar;
    uint32_t tmem_base;
    int32_t stop[2];                       // by iteration parity
    int32_t e_part[2][kMaxWarps][kMaxRPT]; // per-warp sums of s_i (I_i + h_i), by iteration parity
    long long best_e[kNB];
    long long best_step[kNB];
    long long hit[kNB];
    unsigned long long hit_ns[kNB];        // %globaltimer of the first hit (written out at the end)
    int32_t improved[2][kNB];              // by iteration parity
};

// State of the acceptance test (Table 3, state 4; kernels with METRO only), after SmallShared.
struct MetroShared {
    float hx[kMaxWarps][kMaxRPT];   // per-warp sums of x.x at a trajectory's end point
    float hv[kMaxWarps][kMaxRPT];   // ... of v.v
    float sx[kMaxWarps][kMaxRPT];   // per-warp sums of x.x at the current trajectory's start
    float sv[kMaxWarps][kMaxRPT];   // ... of v.v
    long long e_start[kNB];         // E(sgn x) at the current trajectory's start
    int32_t has_start[kNB];         // start known (not the call's first trajectory)
    int32_t revert[kNB];            // the trajectory that just ended was rejected
    int32_t prop[kNB], acc[kNB];    // tests and acceptances
};

template <int OP>
__device__ __forceinline__ uint8_t *operand_ptr(uint8_t *base, int row, int col, uint32_t sbo) {
    constexpr int ESZ = OP == kOpE4M3 ? 1 : 2;
    const int kb = col * ESZ;
    return base + (row >> 3) * sbo + (kb >> 4) * 128 + (row & 7) * 16 + (kb & 15);
}

template <int OP>
__device__ __forceinline__ void put_operand(uint8_t *base, int row, int col, uint32_t sbo, float value) {
    uint8_t *p = operand_ptr<OP>(base, row, col, sbo);
    if constexpr (OP == kOpE4M3) {
        *p = __nv_fp8_e4m3(value).__x;
    } else {
        *reinterpret_cast<__nv_bfloat16 *>(p) = __float2bfloat16_rn(value);
    }
}

template <int OP>
__device__ __forceinline__ void put_spin(uint8_t *p, bool plus) {
    if constexpr (OP == kOpE4M3) {
        *p = plus ? 0x38 : 0xB8;  // e4m3 +1.0 / -1.0
    } else {
        *reinterpret_cast<uint16_t *>(p) = plus ? 0x3F80 : 0xBF80;  // bf16 +1.0 / -1.0
    }
}

// Two accumulators per output tile (even and odd K-steps) so the tensor core sees
// independent MMA chains; their sum is exact (both are integers below 2^24).
__host__ __device__ constexpr uint32_t pow2_cols(uint32_t c) {
    return c <= 32 ? 32 : c <= 64 ? 64 : c <= 128 ? 128 : c <= 256 ? 256 : 512;
}

template <int RPT>
__device__ __forceinline__ void tmem_ld_sync(uint32_t taddr, float (&v)[RPT]) {
    static_assert(RPT == 2 || RPT == 4 || RPT == 8, "unsupported replicas per thread");
    if constexpr (RPT == 8) tmem_ld_x8_sync(taddr, v);
    else if constexpr (RPT == 4) tmem_ld_x4_sync(taddr, v);
    else tmem_ld_x2_sync(taddr, v);
}

// Both accumulators (even and odd K-steps) of this thread's RPT columns: the two loads go
// out together and one wait covers them; the registers pass through the wait so no use
// is scheduled before it.
template <int RPT>
__device__ __forceinline__ void tmem_ld2_sync(uint32_t t0, uint32_t t1, float (&a)[RPT], float (&b)[RPT]) {
    static_assert(RPT == 2 || RPT == 4 || RPT == 8, "unsupported replicas per thread");
    uint32_t x[RPT], y[RPT];
    if constexpr (RPT == 2) {
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];" : "=r"(x[0]), "=r"(x[1]) : "r"(t0));
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];" : "=r"(y[0]), "=r"(y[1]) : "r"(t1));
        asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(x[0]), "+r"(x[1]), "+r"(y[0]), "+r"(y[1]) : : "memory");
    } else if constexpr (RPT == 4) {
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                     : "=r"(x[0]), "=r"(x[1]), "=r"(x[2]), "=r"(x[3]) : "r"(t0));
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                     : "=r"(y[0]), "=r"(y[1]), "=r"(y[2]), "=r"(y[3]) : "r"(t1));
        asm volatile("tcgen05.wait::ld.sync.aligned;"
                     : "+r"(x[0]), "+r"(x[1]), "+r"(x[2]), "+r"(x[3]), "+r"(y[0]), "+r"(y[1]), "+r"(y[2]), "+r"(y[3])
                     :
                     : "memory");
    } else {
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(x[0]), "=r"(x[1]), "=r"(x[2]), "=r"(x[3]), "=r"(x[4]), "=r"(x[5]), "=r"(x[6]), "=r"(x[7])
                     : "r"(t0));
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(y[0]), "=r"(y[1]), "=r"(y[2]), "=r"(y[3]), "=r"(y[4]), "=r"(y[5]), "=r"(y[6]), "=r"(y[7])
                     : "r"(t1));
        asm volatile("tcgen05.wait::ld.sync.aligned;"
                     : "+r"(x[0]), "+r"(x[1]), "+r"(x[2]), "+r"(x[3]), "+r"(x[4]), "+r"(x[5]), "+r"(x[6]), "+r"(x[7]),
                       "+r"(y[0]), "+r"(y[1]), "+r"(y[2]), "+r"(y[3]), "+r"(y[4]), "+r"(y[5]), "+r"(y[6]), "+r"(y[7])
                     :
                     : "memory");
    }
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        a[k] = __uint_as_float(x[k]);
        b[k] = __uint_as_float(y[k]);
    }
}

// MT: 128-spin output tiles; OP: operand encoding; CH: warps sharing one TMEM lane
// quadrant (split over replicas); RPT: replicas per thread.  Live replicas per CTA =
// CH * RPT (8 or 16); the MMA always runs 16 replica columns.
// AT: the couplings (A operand) live in tensor memory instead of shared memory, so
// each MMA reads only the 16-replica spin tile from shared memory.
// Warps 0 .. 4*MT*CH-1 run the epilogue (warp w reads TMEM lane quadrant w % 4); MT
// control warps follow: lane 0 of control warp m issues the field MMAs of output tile m
// (in parallel with the other tiles' issue), the first RL lanes of control warp 0 keep
// the records, so MMA issue and records overlap the epilogue warps' work.
// METRO: the acceptance test of Table 3, state 4 (schedule accept_test = 1).  At the last
// iteration t of a trajectory the epilogue warps leave out the refresh and the next
// position and store warp sums of x.x and v.v instead; control warp 0 decides per replica
// after the records (dH under beta_t, uniform of counter (0xFFFFFFFF, r, t + 1)); after a
// second barrier the epilogue warps put rejected positions back to the trajectory start,
// draw the momentum d = t + 1, keep the new start and its sums, and write the next spins;
// the next field MMAs go out after a third barrier.
template <int MT, int OP, int CH, int RPT, bool AT, int DERIV, bool METRO, bool BATCHED = false>
__global__ void __launch_bounds__(128 * MT * CH + 64 * MT, CH == 1 ? 2 : 1) tc_small_kernel(const RunArgs a, int Kpad) {
    constexpr int ESZ = OP == kOpE4M3 ? 1 : 2;
    constexpr int RL = CH * RPT;
    constexpr int NEPI = 4 * MT * CH;        // epilogue warps
    constexpr uint32_t IDESC = make_idesc(OP == kOpE4M3 ? 0u : 1u, 128, kNB);
    constexpr uint32_t ACC_COLS = 2 * MT * kNB;
    static_assert(RL <= kNB, "live replicas exceed the MMA width");
    static_assert(NEPI <= kMaxWarps && RPT <= kMaxRPT, "shared energy slots too small");
    const int Kbytes = Kpad * ESZ;
    const int KS = Kbytes / 32;            // MMA K-steps (32 bytes of K each)
    const uint32_t SBO = (uint32_t)Kbytes * 8u;
    const uint32_t A_COLS = AT ? (uint32_t)(Kbytes / 4) : 0u;   // TMEM columns per output tile of A
    const uint32_t TCOLS = pow2_cols(ACC_COLS + MT * A_COLS);

    // The instance of this CTA: the run's own, or in a batched run of small dense
    // instances the CTA's entry of the instance table (couplings, field, size, Philox id,
    // scale, first replica, record offsets, target).
    SmallCta ic;
    if constexpr (BATCHED) {
        ic = a.small_cta[blockIdx.x];
    } else {
        ic = SmallCta{a.Jk, a.hk, a.N, a.W, a.inst, a.q, (int32_t)blockIdx.x * RL, 0, 0, a.target};
    }
    int64_t *const rec_best_e = a.best_e + ic.rec_off;
    int64_t *const rec_best_step = a.best_step + ic.rec_off;
    int64_t *const rec_hit_step = a.hit_step + ic.rec_off;
    uint64_t *const rec_hit_ns = a.hit_ns ? a.hit_ns + ic.rec_off : nullptr;
    uint32_t *const rec_best_bits = a.best_bits + ic.bits_off;
    int64_t *const rec_proposed = a.proposed ? a.proposed + ic.rec_off : nullptr;
    int64_t *const rec_accepted = a.accepted ? a.accepted + ic.rec_off : nullptr;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *sA = smem;
    uint8_t *sB = AT ? smem : sA + MT * 128 * Kbytes;
    SmallShared *sm = reinterpret_cast<SmallShared *>(sB + kNB * Kbytes);
    MetroShared *ms = reinterpret_cast<MetroShared *>(sm + 1);   // METRO kernels only

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool ctl = warp >= NEPI;         // control warps
    const int cw = warp - NEPI;            // control warp: output tile cw % MT, K-step parity cw / MT
    const int q4 = warp & 3;               // TMEM lane quadrant this warp may access
    const int mt = (warp >> 2) % MT;       // output-spin tile
    const int ch = warp / (4 * MT);        // which RPT of the RL replicas
    const int N = ic.N;
    const int i = mt * 128 + q4 * 32 + lane;
    const bool live_i = !ctl && i < N;
    const int rbase = ic.rbase;

    if (warp == 0) {
        tmem_alloc(&sm->tmem_base, TCOLS);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(&sm->mbar, 2 * MT);      // one commit per (output tile, K-step parity)
        fence_mbarrier_init();
    }
    // Couplings into A (zero-padded to MT*128 rows x Kpad columns), B cleared.
    if constexpr (!AT) {
        for (int idx = tid; idx < MT * 128 * Kpad; idx += blockDim.x) {
            const int row = idx / Kpad, col = idx - row * Kpad;
            const float val = (row < N && col < N) ? (float)ic.Jk[(size_t)row * N + col] : 0.0f;
            put_operand<OP>(sA, row, col, SBO, val);
        }
    }
    for (int idx = tid; idx < kNB * Kbytes / 16; idx += blockDim.x)
        reinterpret_cast<uint4 *>(sB)[idx] = make_uint4(0, 0, 0, 0);
    if (tid < kNB) {
        const int r = rbase + tid;
        sm->improved[0][tid] = 0;
        sm->improved[1][tid] = 0;
        const bool rec = !a.field_mode && tid < RL && r < a.R;
        sm->best_e[tid] = rec ? rec_best_e[r] : LLONG_MAX;
        sm->best_step[tid] = rec ? rec_best_step[r] : -1;
        sm->hit[tid] = rec ? rec_hit_step[r] : -1;
        sm->hit_ns[tid] = (rec && rec_hit_ns) ? rec_hit_ns[r] : 0ull;
        if constexpr (METRO) {
            ms->has_start[tid] = 0;
            ms->revert[tid] = 0;
            ms->prop[tid] = 0;
            ms->acc[tid] = 0;
        }
    }
    if (tid == 0) sm->stop[0] = sm->stop[1] = 0;
    tc_fence_before();
    __syncthreads();  // B cleared before spins are written into it; TMEM base published
    tc_fence_after();
    if constexpr (AT) {
        // Row i of A (output spin i) into TMEM lane i % 128 of tile i / 128: 32 bytes of K
        // (8 columns) per store.  One warp per (lane quadrant, tile) does it.
        if (!ctl && ch == 0) {
            const uint32_t base = sm->tmem_base + ((uint32_t)(q4 * 32) << 16) + ACC_COLS + mt * A_COLS;
            for (int c8 = 0; c8 < Kbytes / 32; ++c8) {
                uint32_t w[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    uint32_t word = 0;
#pragma unroll
                    for (int b = 0; b < 4 / ESZ; ++b) {
                        const int col = (c8 * 32 + q * 4) / ESZ + b;
                        const float val = (live_i && col < N) ? (float)ic.Jk[(size_t)i * N + col] : 0.0f;
                        uint32_t enc;
                        if constexpr (OP == kOpE4M3) enc = __nv_fp8_e4m3(val).__x;
                        else enc = __bfloat16_as_ushort(__float2bfloat16_rn(val));
                        word |= enc << (8 * ESZ * b);
                    }
                    w[q] = word;
                }
                tmem_st_x8(base + c8 * 8, w);
            }
            tmem_st_wait();
        }
    }

    // This thread's spin slots in B: replica c = ch*RPT + k sits at row c, column i.
    uint8_t *my_b = operand_ptr<OP>(sB, ctl ? 0 : ch * RPT, live_i ? i : 0, SBO);
    const int32_t hki = live_i ? ic.hk[i] : 0;
    float x[RPT], v[RPT];
    float xs[RPT];     // METRO: positions at the current trajectory's start
#pragma unroll
    for (int k = 0; k < RPT; ++k) xs[k] = 0.0f;
    uint32_t cur = 0;  // bit k: spin i of replica ch*RPT+k is +1 in the B of this iteration
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        const int c = ch * RPT + k, r = rbase + c;
        x[k] = 0.0f; v[k] = 0.0f;
        if (!live_i) continue;
        if (a.field_mode) {
            if (r < a.R) {
                const bool plus = a.spins_in[(size_t)r * N + i] > 0;
                put_spin<OP>(my_b + k * 16, plus);
                cur |= (uint32_t)plus << k;
            }
            continue;
        }
        if (a.x_in) {
            x[k] = r < a.R ? a.x_in[(size_t)r * N + i] : 0.0f;
            v[k] = r < a.R ? a.v_in[(size_t)r * N + i] : 0.0f;
        } else {
            const U4 o = draw_raw(a.seed, ic.inst, (uint32_t)r, (uint32_t)i, 0u);
            x[k] = box_muller(o.x, o.y);
            v[k] = box_muller(o.z, o.w);
        }
        if (refresh_at(a.t0, a.refresh)) v[k] = draw_v(a.seed, ic.inst, (uint32_t)r, (uint32_t)i, (uint32_t)a.t0);
        x[k] = x[k] + a.eps * v[k];                 // position half of Eq. A7
        const bool plus = x[k] >= 0.0f;             // sgn with sgn(0) = +1
        put_spin<OP>(my_b + k * 16, plus);
        cur |= (uint32_t)plus << k;
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm->tmem_base;
    const uint32_t my_taddr = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(2 * mt * kNB + ch * RPT);
    const int word = (mt * 128 + q4 * 32) >> 5;

    const int nit = a.field_mode ? 1 : (int)a.nsteps;
    const float inv_tm1 = inv_tm1_of(a.T_total);
    const float eps = a.eps, gamma = a.gamma, gq = a.gamma * ic.q;
    int rc = a.refresh > 0 ? (int)((a.t0 + 1) % a.refresh) : 1;   // (t + 1) mod refresh
    uint32_t phase = 0, prv = 0;
    bool timed_out = false, stopped = false;
    int it = 0;
    // Field MMAs of output tile m for one iteration: D[m] = A[m] B^T over all K-steps,
    // K-step ks into D[m][ks & 1] (lane 0 of control warp m).  Descriptors advance by
    // adding (byte offset >> 4) to the start-address field.
    const uint64_t adesc0 = smem_desc_noswizzle(smem_u32(sA), 128, SBO);
    const uint64_t bdesc0 = smem_desc_noswizzle(smem_u32(sB), 128, SBO);
    auto issue_field = [&](int w) {
        tc_fence_after();
        const int m = w % MT, par = w / MT;
        const uint64_t am = adesc0 + (uint64_t)((m * 16 * SBO) >> 4);
#pragma unroll 1
        for (int ks = par; ks < KS; ks += 2) {
            const uint64_t bd = bdesc0 + (uint64_t)(ks * 16);   // 256 bytes per K-step
            const uint32_t d = tmem + (uint32_t)((2 * m + (ks & 1)) * kNB);
            if constexpr (AT) {
                const uint32_t at = tmem + ACC_COLS + m * A_COLS + ks * 8;   // 32 bytes = 8 columns
                if constexpr (OP == kOpE4M3) mma_e4m3_ta(d, at, bd, IDESC, ks > 1);
                else mma_bf16_ta(d, at, bd, IDESC, ks > 1);
            } else {
                const uint64_t ad = am + (uint64_t)(ks * 16);
                if constexpr (OP == kOpE4M3) mma_e4m3(d, ad, bd, IDESC, ks > 1);
                else mma_bf16(d, ad, bd, IDESC, ks > 1);
            }
        }
        mma_commit(&sm->mbar);
    };
    const bool two_acc = KS > 1;
    if (ctl && lane == 0) issue_field(cw);
    for (; it < nit; ++it) {
        const int64_t t = a.t0 + it;
        bool ok = true;
        uint32_t nxt = 0;
        if (!ctl) {
            ok = mbar_wait_bounded(&sm->mbar, phase, kWaitTimeoutNs);
            tc_fence_after();
            float acc[RPT];
            if (two_acc) {
                float acc2[RPT];
                tmem_ld2_sync<RPT>(my_taddr, my_taddr + kNB, acc, acc2);
#pragma unroll
                for (int k = 0; k < RPT; ++k) acc[k] += acc2[k];
            } else {
                tmem_ld_sync<RPT>(my_taddr, acc);
            }
            // Field (Eq. 6, exact) and energy terms s_i (I_i + h_i) of every replica first,
            // then their warp sums, then the updates: straight-line code across replicas.
            int32_t Ik[RPT], part[RPT];
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                Ik[k] = __float2int_rn(acc[k]) + hki;
                part[k] = live_i ? (((cur >> k) & 1u) ? (Ik[k] + hki) : -(Ik[k] + hki)) : 0;
            }
#pragma unroll
            for (int k = 0; k < RPT; ++k) part[k] = __reduce_add_sync(0xffffffffu, part[k]);
            if (lane == 0) {
#pragma unroll
                for (int k = 0; k < RPT; ++k) sm->e_part[it & 1][warp][k] = part[k];
            }
            if (a.field_mode) {
#pragma unroll
                for (int k = 0; k < RPT; ++k) {
                    const int r = rbase + ch * RPT + k;
                    if (live_i && r < a.R && a.field_out) a.field_out[(size_t)r * N + i] = Ik[k];
                }
            } else if (METRO && it + 1 < nit && a.refresh > 0 && rc == 0) {
                // Last iteration of a trajectory under the acceptance test: the update of v,
                // then warp sums of x.x and v.v of the end point; refresh and position wait
                // for the decision.
                if (live_i) {
                    const float bgq = beta_at(t, inv_tm1, a.beta0, a.beta1) * gq;
#pragma unroll
                    for (int k = 0; k < RPT; ++k) v[k] = DERIV == 1 ? momentum_quad(v[k], x[k], (float)Ik[k], eps, bgq, gamma)
                                                                    : momentum_exact(v[k], x[k], (float)Ik[k], eps, bgq, gamma);
                }
#pragma unroll
                for (int k = 0; k < RPT; ++k) {
                    float px = live_i ? x[k] * x[k] : 0.0f, pv = live_i ? v[k] * v[k] : 0.0f;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        px += __shfl_xor_sync(0xffffffffu, px, o);
                        pv += __shfl_xor_sync(0xffffffffu, pv, o);
                    }
                    if (lane == 0) {
                        ms->hx[warp][k] = px;
                        ms->hv[warp][k] = pv;
                    }
                }
            } else if (live_i) {
                const float bgq = beta_at(t, inv_tm1, a.beta0, a.beta1) * gq;
                const bool more = it + 1 < nit;
                if constexpr (DERIV == 1) {
#pragma unroll
                    for (int k = 0; k < RPT; ++k) v[k] = momentum_quad(v[k], x[k], (float)Ik[k], eps, bgq, gamma);
                } else {
#pragma unroll
                    for (int k = 0; k < RPT; ++k) v[k] = momentum_exact(v[k], x[k], (float)Ik[k], eps, bgq, gamma);
                }
                if (more) {
                    if (a.refresh > 0 && rc == 0) {
#pragma unroll
                        for (int k = 0; k < RPT; ++k)
                            v[k] = draw_v(a.seed, ic.inst, (uint32_t)(rbase + ch * RPT + k), (uint32_t)i, (uint32_t)(t + 1));
                    }
#pragma unroll
                    for (int k = 0; k < RPT; ++k) {
                        x[k] = x[k] + eps * v[k];
                        const bool plus = x[k] >= 0.0f;
                        put_spin<OP>(my_b + k * 16, plus);
                        nxt |= (uint32_t)plus << k;
                    }
                }
            }
            fence_proxy_async_smem();
            tc_fence_before();
        }
        phase ^= 1u;
        if (__syncthreads_or(!ok)) { timed_out = true; break; }
        const bool tested = METRO && !a.field_mode && it + 1 < nit && a.refresh > 0 && rc == 0;
        if (ctl) {
            // Next iteration's field first: B holds its spins and every TMEM read is done
            // (after a trajectory end under the acceptance test, once the spins are written).
            if (lane == 0 && it + 1 < nit && !tested) issue_field(cw);
            // Records of iteration t (Table 3, state 5), one lane per replica column.
            if (cw == 0 && lane < RL) {
                const int c = lane, r = rbase + c;
                long long twice = 0;   // sum_i s_i (I_i + h_i) over the 4*MT warps holding replica c
#pragma unroll
                for (int j = 0; j < 4 * MT; ++j) twice += sm->e_part[it & 1][(c / RPT) * 4 * MT + j][c % RPT];
                const long long E = -twice / 2;                                  // Eq. 2 via the field
                int imp = 0;
                if (a.field_mode) {
                    if (r < a.R && a.energy_out) a.energy_out[r] = E;
                } else if (r < a.R) {
                    const bool frozen = a.stop_at_target && sm->hit[c] >= 0;
                    if (!frozen && E < sm->best_e[c]) {
                        sm->best_e[c] = E;
                        sm->best_step[c] = t;
                        imp = 1;
                    }
                    if (a.has_target && sm->hit[c] < 0 && E <= ic.target) {
                        sm->hit[c] = t;
                        sm->hit_ns[c] = globaltimer_ns();
                        if (a.stop_at_target && !BATCHED) atomicMin(a.min_hit, (unsigned long long)t);
                    }
                    if (tested) {
                        // Table 3, state 4: H = beta E + x.x/2 + v.v/2 (Eq. 4) of the end point
                        // against the start, both under beta_t.
                        float xx = 0.0f, vv = 0.0f;
#pragma unroll
                        for (int j = 0; j < 4 * MT; ++j) {
                            xx += ms->hx[(c / RPT) * 4 * MT + j][c % RPT];
                            vv += ms->hv[(c / RPT) * 4 * MT + j][c % RPT];
                        }
                        int rev = 0;
                        if (ms->has_start[c]) {
                            float sx = 0.0f, sv = 0.0f;
#pragma unroll
                            for (int j = 0; j < 4 * MT; ++j) {
                                sx += ms->sx[(c / RPT) * 4 * MT + j][c % RPT];
                                sv += ms->sv[(c / RPT) * 4 * MT + j][c % RPT];
                            }
                            const float beta = beta_at(t, inv_tm1, a.beta0, a.beta1);
                            const float dH = beta * ic.q * (float)(E - ms->e_start[c]) + 0.5f * (xx - sx) +
                                             0.5f * (vv - sv);
                            ms->prop[c] += 1;
                            if (metropolis_accept(dH, accept_uniform(a.seed, ic.inst, (uint32_t)r, (uint32_t)(t + 1)))) {
                                ms->acc[c] += 1;
                                ms->e_start[c] = E;
                            } else {
                                rev = 1;
                            }
                        } else {
                            ms->e_start[c] = E;
                            ms->has_start[c] = 1;
                        }
                        ms->revert[c] = rev;
                    }
                }
                sm->improved[it & 1][c] = imp;
            }
            if (cw == 0 && lane == 0)
                sm->stop[it & 1] = (a.stop_at_target && !a.field_mode && !BATCHED)
                                       ? (*(volatile unsigned long long *)a.min_hit <= (unsigned long long)t)
                                       : 0;
        } else if (it > 0) {
            // Best spins of iteration t-1 (its records were settled before this barrier).
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                const int c = ch * RPT + k;
                if (sm->improved[(it - 1) & 1][c]) {
                    const uint32_t bits = __ballot_sync(0xffffffffu, live_i && ((prv >> k) & 1u));
                    if (lane == 0 && word < ic.W) rec_best_bits[(size_t)(rbase + c) * ic.W + word] = bits;
                }
            }
        }
        if constexpr (METRO) {
            if (tested) {
                // The decision is in shared memory: rejected replicas go back to the start,
                // then the momentum draw d = t + 1, the new start and its sums, and the next
                // position and spins; the field MMAs follow once B holds them.
                __syncthreads();
                if (!ctl) {
#pragma unroll
                    for (int k = 0; k < RPT; ++k) {
                        const int c = ch * RPT + k;
                        if (live_i) {
                            if (ms->revert[c]) x[k] = xs[k];
                            v[k] = draw_v(a.seed, ic.inst, (uint32_t)(rbase + c), (uint32_t)i, (uint32_t)(t + 1));
                            xs[k] = x[k];
                        }
                        float px = live_i ? x[k] * x[k] : 0.0f, pv = live_i ? v[k] * v[k] : 0.0f;
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) {
                            px += __shfl_xor_sync(0xffffffffu, px, o);
                            pv += __shfl_xor_sync(0xffffffffu, pv, o);
                        }
                        if (lane == 0) {
                            ms->sx[warp][k] = px;
                            ms->sv[warp][k] = pv;
                        }
                        if (live_i) {
                            x[k] = x[k] + eps * v[k];
                            const bool plus = x[k] >= 0.0f;
                            put_spin<OP>(my_b + k * 16, plus);
                            nxt |= (uint32_t)plus << k;
                        }
                    }
                    fence_proxy_async_smem();
                    tc_fence_before();
                }
                __syncthreads();
                if (ctl && lane == 0) issue_field(cw);
            }
        }
        prv = cur;
        cur = nxt;
        rc = (a.refresh > 0 && rc + 1 == a.refresh) ? 0 : rc + 1;
        if (it > 0 && sm->stop[(it - 1) & 1]) { stopped = true; ++it; break; }
    }
    // A field issued for an iteration that will not run (stop) must finish before TMEM is freed.
    if (stopped && it < nit && ctl && cw == 0 && lane == 0) mbar_wait_bounded(&sm->mbar, phase, kWaitTimeoutNs);

    if (!timed_out) {
        __syncthreads();  // records of the last iteration settled
        const int last = it - 1;
        if (!ctl) {
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                const int c = ch * RPT + k;
                if (last >= 0 && sm->improved[last & 1][c]) {
                    const uint32_t bits = __ballot_sync(0xffffffffu, live_i && ((prv >> k) & 1u));
                    if (lane == 0 && word < ic.W) rec_best_bits[(size_t)(rbase + c) * ic.W + word] = bits;
                }
            }
        }
    }
    if (!a.field_mode && !timed_out && !stopped && a.x_out && live_i) {
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const int r = rbase + ch * RPT + k;
            if (r < a.R) {
                a.x_out[(size_t)r * N + i] = x[k];
                a.v_out[(size_t)r * N + i] = v[k];
            }
        }
    }
    if (ctl && cw == 0 && lane < RL && !a.field_mode) {
        const int r = rbase + lane;
        if (r < a.R) {
            rec_best_e[r] = sm->best_e[lane];
            rec_best_step[r] = sm->best_step[lane];
            rec_hit_step[r] = sm->hit[lane];
            if (rec_hit_ns) rec_hit_ns[r] = sm->hit_ns[lane];
            if constexpr (METRO) {
                rec_proposed[r] = ms->prop[lane];
                rec_accepted[r] = ms->acc[lane];
            }
        }
    }
    if (ctl && cw == 0 && lane == 0) {
        const int valid = min(RL, a.R - rbase);
        if (!a.field_mode) atomicAdd(a.replica_iters, (unsigned long long)((long long)valid * it));
        if (timed_out) {
            atomicExch(a.err, 1);
            mbar_wait_bounded(&sm->mbar, phase ^ 1u, kWaitTimeoutNs);  // let the MMA in flight drain
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, TCOLS);
    }
}

template <int MT, int OP, int CH, int RPT, bool AT = false, bool METRO = false>
cudaError_t launch_cfg(const RunArgs &a, int Kpad, cudaStream_t st) {
    constexpr int ESZ = OP == kOpE4M3 ? 1 : 2;
    constexpr int RL = CH * RPT;
    const size_t smem = (size_t)((AT ? 0 : MT * 128) + kNB) * Kpad * ESZ + sizeof(SmallShared) +
                        (METRO ? sizeof(MetroShared) : 0) + 16;
    // The derivative mode is a template parameter: the update loop stays straight-line.
    auto kern = a.deriv == 1 ? tc_small_kernel<MT, OP, CH, RPT, AT, 1, METRO>
                             : tc_small_kernel<MT, OP, CH, RPT, AT, 0, METRO>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = (a.R + RL - 1) / RL;
    kern<<<grid, 128 * MT * CH + 64 * MT, smem, st>>>(a, Kpad);
    return cudaGetLastError();
}

}  // namespace

// Live replicas per CTA: the requested variant (4, 8 or 16), else 16 when that already
// gives one CTA per SM, else 8.
int tc_small_tile_replicas(int R, int requested) {
    if (requested == 4 || requested == 8 || requested == 16) return requested;
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return (R + 15) / 16 >= sms ? 16 : 8;
}

namespace {

template <int MT, int OP, bool AT, bool METRO = false>
cudaError_t launch_at(const RunArgs &a, int Kpad, cudaStream_t st) {
    const int rl = tc_small_tile_replicas(a.R, a.tile_rl);
    if (rl == 16) return launch_cfg<MT, OP, 2, 8, AT, METRO>(a, Kpad, st);
    if (rl == 8) return launch_cfg<MT, OP, 2, 4, AT, METRO>(a, Kpad, st);
    return launch_cfg<MT, OP, 1, 4, AT, METRO>(a, Kpad, st);
}

template <int MT, int OP>
cudaError_t launch_mt(const RunArgs &a, int Kpad, cudaStream_t st) {
    // The acceptance test (with trajectories to test) runs with J in shared memory.
    if (a.accept_test == 1 && a.refresh > 0 && !a.field_mode) return launch_at<MT, OP, false, true>(a, Kpad, st);
    if (a.coupling_mem == 2) return launch_at<MT, OP, true>(a, Kpad, st);
    return launch_at<MT, OP, false>(a, Kpad, st);
}

}  // namespace

int tc_small_max_n(int op) { return op == kOpE4M3 ? 384 : 256; }

namespace {

template <int MT, int OP>
cudaError_t launch_batch_mt(const RunArgs &a, int Kpad, cudaStream_t st) {
    // Every instance of the launch shares MT and the operand; K is padded for the group's
    // largest N (Kpad), so that one shared-memory layout serves all of them (the couplings
    // and spins past an instance's N are zero).
    constexpr int ESZ = OP == kOpE4M3 ? 1 : 2;
    const size_t smem = (size_t)(MT * 128 + kNB) * Kpad * ESZ + sizeof(SmallShared) + 16;
    auto kern = a.deriv == 1 ? tc_small_kernel<MT, OP, 2, 4, false, 1, false, true>
                             : tc_small_kernel<MT, OP, 2, 4, false, 0, false, true>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<a.small_ctas, 128 * MT * 2 + 64 * MT, smem, st>>>(a, Kpad);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tc_small_batch(const RunArgs &a, int op, int mt, int kpad, cudaStream_t st) {
    if (a.small_ctas < 1) return cudaSuccess;
    if (op == kOpE4M3) {
        if (mt == 1) return launch_batch_mt<1, kOpE4M3>(a, kpad, st);
        if (mt == 2) return launch_batch_mt<2, kOpE4M3>(a, kpad, st);
        if (mt == 3) return launch_batch_mt<3, kOpE4M3>(a, kpad, st);
    } else {
        if (mt == 1) return launch_batch_mt<1, kOpBF16>(a, kpad, st);
        if (mt == 2) return launch_batch_mt<2, kOpBF16>(a, kpad, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_tc_small(const RunArgs &a, int op, cudaStream_t st, int *launches) {
    const int MT = (a.N + 127) / 128;
    const int Kpad = op == kOpE4M3 ? (a.N + 31) / 32 * 32 : (a.N + 15) / 16 * 16;
    if (launches) *launches += 1;
    if (op == kOpE4M3) {
        if (MT == 1) return launch_mt<1, kOpE4M3>(a, Kpad, st);
        if (MT == 2) return launch_mt<2, kOpE4M3>(a, Kpad, st);
        if (MT == 3) return launch_mt<3, kOpE4M3>(a, Kpad, st);
    } else {
        if (MT == 1) return launch_mt<1, kOpBF16>(a, Kpad, st);
        if (MT == 2) return launch_mt<2, kOpBF16>(a, Kpad, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace phia
