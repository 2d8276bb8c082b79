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
#include <cuda_fp8.h>
#include <cuda_bf16.h>

#include "device_common.cuh"
#include "phia_internal.h"

namespace phia {

namespace {

constexpr int kRB = 16;  // replicas per CTA = MMA N

struct SmallShared {
    uint64_t mbar;
    uint32_t tmem_base;
    int32_t stop;
    unsigned long long e_acc[kRB];
    long long best_e[kRB];
    long long best_step[kRB];
    long long hit[kRB];
    int32_t improved[kRB];
};

template <int OP>
__device__ __forceinline__ void put_operand(uint8_t *base, int row, int col, uint32_t sbo, float value) {
    constexpr int ESZ = OP == kOpE4M3 ? 1 : 2;
    const int kb = col * ESZ;
    uint8_t *p = base + (row >> 3) * sbo + (kb >> 4) * 128 + (row & 7) * 16 + (kb & 15);
    if constexpr (OP == kOpE4M3) {
        *p = __nv_fp8_e4m3(value).__x;
    } else {
        *reinterpret_cast<__nv_bfloat16 *>(p) = __float2bfloat16_rn(value);
    }
}

template <int OP>
__device__ __forceinline__ void put_spin(uint8_t *base, int row, int col, uint32_t sbo, bool plus) {
    constexpr int ESZ = OP == kOpE4M3 ? 1 : 2;
    const int kb = col * ESZ;
    uint8_t *p = base + (row >> 3) * sbo + (kb >> 4) * 128 + (row & 7) * 16 + (kb & 15);
    if constexpr (OP == kOpE4M3) {
        *p = plus ? 0x38 : 0xB8;  // e4m3 +1.0 / -1.0
    } else {
        *reinterpret_cast<uint16_t *>(p) = plus ? 0x3F80 : 0xBF80;  // bf16 +1.0 / -1.0
    }
}

template <int MT>
__host__ __device__ constexpr uint32_t tmem_cols() { return MT * kRB <= 32 ? 32 : (MT * kRB <= 64 ? 64 : 128); }

template <int MT, int OP>
__global__ void __launch_bounds__(256 * MT, 1) tc_small_kernel(const RunArgs a, int Kpad) {
    constexpr int ESZ = OP == kOpE4M3 ? 1 : 2;
    constexpr uint32_t IDESC = make_idesc(OP == kOpE4M3 ? 0u : 1u, 128, kRB);
    constexpr uint32_t TCOLS = tmem_cols<MT>();
    const int Kbytes = Kpad * ESZ;
    const int KS = Kbytes / 32;            // MMA K-steps (32 bytes of K each)
    const uint32_t SBO = (uint32_t)Kbytes * 8u;

    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *sA = smem;
    uint8_t *sB = sA + MT * 128 * Kbytes;
    SmallShared *sm = reinterpret_cast<SmallShared *>(sB + kRB * Kbytes);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q4 = warp & 3;               // TMEM lane quadrant this warp may access
    const int mt = (warp >> 2) % MT;       // output-spin tile
    const int ch = warp / (4 * MT);        // which 8 of the 16 replicas
    const int N = a.N;
    const int i = mt * 128 + q4 * 32 + lane;
    const bool live_i = i < N;
    const int rbase = blockIdx.x * kRB;

    if (warp == 0) {
        tmem_alloc(&sm->tmem_base, TCOLS);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(&sm->mbar, 1);
        fence_mbarrier_init();
    }
    // Couplings into A (zero-padded to MT*128 rows x Kpad columns), B cleared.
    for (int idx = tid; idx < MT * 128 * Kpad; idx += blockDim.x) {
        const int row = idx / Kpad, col = idx - row * Kpad;
        const float val = (row < N && col < N) ? (float)a.Jk[(size_t)row * N + col] : 0.0f;
        put_operand<OP>(sA, row, col, SBO, val);
    }
    for (int idx = tid; idx < kRB * Kbytes / 16; idx += blockDim.x)
        reinterpret_cast<uint4 *>(sB)[idx] = make_uint4(0, 0, 0, 0);
    if (tid < kRB) {
        const int r = rbase + tid;
        sm->e_acc[tid] = 0;
        sm->improved[tid] = 0;
        const bool rec = !a.field_mode && r < a.R;
        sm->best_e[tid] = rec ? a.best_e[r] : LLONG_MAX;
        sm->best_step[tid] = rec ? a.best_step[r] : -1;
        sm->hit[tid] = rec ? a.hit_step[r] : -1;
    }
    if (tid == 0) sm->stop = 0;
    __syncthreads();  // B cleared before spins are written into it

    const int32_t hki = live_i ? a.hk[i] : 0;
    float x[8], v[8];
    uint32_t smask = 0;  // bit k: spin i of replica ch*8+k is +1 in the current B
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int c = ch * 8 + k, r = rbase + c;
        x[k] = 0.0f; v[k] = 0.0f;
        if (!live_i) continue;
        if (a.field_mode) {
            if (r < a.R) {
                const bool plus = a.spins_in[(size_t)r * N + i] > 0;
                put_spin<OP>(sB, c, i, SBO, plus);
                smask |= (uint32_t)plus << k;
            }
            continue;
        }
        if (a.x_in) {
            x[k] = r < a.R ? a.x_in[(size_t)r * N + i] : 0.0f;
            v[k] = r < a.R ? a.v_in[(size_t)r * N + i] : 0.0f;
        } else {
            const U4 o = draw_raw(a.seed, a.inst, (uint32_t)r, (uint32_t)i, 0u);
            x[k] = box_muller(o.x, o.y);
            v[k] = box_muller(o.z, o.w);
        }
        if (refresh_at(a.t0, a.refresh)) v[k] = draw_v(a.seed, a.inst, (uint32_t)r, (uint32_t)i, (uint32_t)a.t0);
        x[k] = x[k] + a.eps * v[k];                 // position half of Eq. A7
        const bool plus = x[k] >= 0.0f;             // sgn with sgn(0) = +1
        put_spin<OP>(sB, c, i, SBO, plus);
        smask |= (uint32_t)plus << k;
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm->tmem_base;
    const uint32_t my_taddr = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(mt * kRB + ch * 8);

    const int64_t t_end = a.field_mode ? a.t0 + 1 : a.t0 + a.nsteps;
    uint32_t phase = 0;
    bool timed_out = false, stopped = false;
    int64_t iters = 0;
    for (int64_t t = a.t0; t < t_end; ++t) {
        if (tid == 0) {
            tc_fence_after();
            const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll 1
            for (int m = 0; m < MT; ++m) {
#pragma unroll 1
                for (int ks = 0; ks < KS; ++ks) {
                    const uint64_t ad = smem_desc_noswizzle(a0 + m * 16 * SBO + ks * 256, 128, SBO);
                    const uint64_t bd = smem_desc_noswizzle(b0 + ks * 256, 128, SBO);
                    if constexpr (OP == kOpE4M3) mma_e4m3(tmem + m * kRB, ad, bd, IDESC, ks > 0);
                    else mma_bf16(tmem + m * kRB, ad, bd, IDESC, ks > 0);
                }
            }
            mma_commit(&sm->mbar);
        }
        const bool ok = mbar_wait_bounded(&sm->mbar, phase, kWaitTimeoutNs);
        phase ^= 1u;
        tc_fence_after();
        float acc[8];
        tmem_ld_x8_sync(my_taddr, acc);

        const float beta = beta_at(t, a.T_total, a.beta0, a.beta1);
        const float bgq = beta * a.gamma * a.q;
        const bool more = t + 1 < t_end;
        const bool refresh_next = more && refresh_at(t + 1, a.refresh);
        uint32_t newmask = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int c = ch * 8 + k, r = rbase + c;
            const int32_t Ik = __float2int_rn(acc[k]) + hki;       // Eq. 6, exact
            const int32_t sk = ((smask >> k) & 1u) ? 1 : -1;
            int32_t part = live_i ? sk * (Ik + hki) : 0;            // s_i (I_i + h_i)
            part = __reduce_add_sync(0xffffffffu, part);
            if (lane == 0) atomicAdd(&sm->e_acc[c], (unsigned long long)(long long)part);
            if (a.field_mode) {
                if (live_i && r < a.R && a.field_out) a.field_out[(size_t)r * N + i] = Ik;
                continue;
            }
            if (!live_i) continue;
            v[k] = momentum_update(v[k], x[k], (float)Ik, a.eps, bgq, a.gamma);
            if (more) {
                if (refresh_next) v[k] = draw_v(a.seed, a.inst, (uint32_t)r, (uint32_t)i, (uint32_t)(t + 1));
                x[k] = x[k] + a.eps * v[k];
                const bool plus = x[k] >= 0.0f;
                put_spin<OP>(sB, c, i, SBO, plus);
                newmask |= (uint32_t)plus << k;
            }
        }
        fence_proxy_async_smem();
        tc_fence_before();
        if (__syncthreads_or(!ok)) { timed_out = true; break; }

        if (tid < kRB) {
            const int c = tid, r = rbase + c;
            const long long E = -((long long)sm->e_acc[c]) / 2;    // Eq. 2 via the field
            sm->e_acc[c] = 0;
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
                if (a.has_target && sm->hit[c] < 0 && E <= a.target) {
                    sm->hit[c] = t;
                    if (a.stop_at_target) atomicMin(a.min_hit, (unsigned long long)t);
                }
            }
            sm->improved[c] = imp;
        }
        if (tid == 0)
            sm->stop = (a.stop_at_target && !a.field_mode)
                           ? (*(volatile unsigned long long *)a.min_hit <= (unsigned long long)t)
                           : 0;
        __syncthreads();
        ++iters;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int c = ch * 8 + k;
            if (sm->improved[c]) {
                const uint32_t bits = __ballot_sync(0xffffffffu, live_i && ((smask >> k) & 1u));
                const int word = (mt * 128 + q4 * 32) >> 5;
                if (lane == 0 && word < a.W) a.best_bits[(size_t)(rbase + c) * a.W + word] = bits;
            }
        }
        smask = newmask;
        if (sm->stop) { stopped = true; break; }
    }

    if (!a.field_mode && !timed_out && !stopped && a.x_out && live_i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int r = rbase + ch * 8 + k;
            if (r < a.R) {
                a.x_out[(size_t)r * N + i] = x[k];
                a.v_out[(size_t)r * N + i] = v[k];
            }
        }
    }
    if (tid < kRB && !a.field_mode) {
        const int r = rbase + tid;
        if (r < a.R) {
            a.best_e[r] = sm->best_e[tid];
            a.best_step[r] = sm->best_step[tid];
            a.hit_step[r] = sm->hit[tid];
        }
    }
    if (tid == 0) {
        const int valid = min(kRB, a.R - rbase);
        if (!a.field_mode) atomicAdd(a.replica_iters, (unsigned long long)(valid * iters));
        if (timed_out) {
            atomicExch(a.err, 1);
            mbar_wait_bounded(&sm->mbar, phase, kWaitTimeoutNs);  // let an MMA in flight drain
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, TCOLS);
    }
}

template <int MT, int OP>
cudaError_t launch_mt(const RunArgs &a, int Kpad, cudaStream_t st) {
    constexpr int ESZ = OP == kOpE4M3 ? 1 : 2;
    const size_t smem = (size_t)(MT * 128 + kRB) * Kpad * ESZ + sizeof(SmallShared) + 16;
    auto kern = tc_small_kernel<MT, OP>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = (a.R + kRB - 1) / kRB;
    kern<<<grid, 256 * MT, smem, st>>>(a, Kpad);
    return cudaGetLastError();
}

}  // namespace

int tc_small_max_n(int op) { return op == kOpE4M3 ? 384 : 256; }

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
