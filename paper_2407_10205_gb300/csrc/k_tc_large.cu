// k_tc_large.cu -- tensor-core PHIA path for dense instances of any size: one launch per
// iteration (Eq. A7), each CTA computing a 128-spin x 128-replica block of the field
// I = J s + h (Eq. 6) and running the fused update on it.
//
// Operands (K-major, 128-byte swizzle, staged by TMA through a 3-deep mbarrier ring):
//   A = couplings k re-encoded exactly (e4m3 or bf16), [Mpad][Kpad]
//   B = spins of this iteration in the same encoding, [Rpad][Kpad], one of 4 rotating
//       buffers (iteration t reads buffer t % 4 and writes t+1 % 4; buffers t-1 and t-2
//       stay intact for the lagged best-state copies).
// D = J s accumulates in TMEM (FP32, integer-valued, exact below 2^24): lane = output
// spin, column = replica.
// Warp roles: warp 0 issues TMA, warp 1 issues the MMAs (one thread each), warps 2-9 run
// the epilogue: field + h, s (I + h) energy partials, momentum update (Eqs. 5, 8),
// refresh, position update and the sign written as next iteration's B operand; x and v
// stream from/to global memory ([R][N] FP32).
// Records (Table 3, state 5) are lagged so no CTA waits for another: the launch for
// iteration t lets the CTAs of output tile 0 settle the energies of iteration t-1 (sum
// of every tile's partials) and every CTA copy, for replicas that improved at t-2, its
// 128 spins of buffer t-2 into the bit-packed best state.  A final pair of launches
// settles the last two iterations.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "device_common.cuh"
#include "phia_internal.h"

namespace phia {

namespace {

constexpr int kBM = 128;       // output spins per CTA (TMEM lanes)
constexpr int kBN = 128;       // replicas per CTA (TMEM columns)
constexpr int kBKB = 128;      // bytes of K per pipeline stage (one 128-byte swizzle row)
constexpr int kStages = 3;
constexpr int kEpiWarps = 8;   // two per TMEM lane quadrant, each half of the columns
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr uint32_t kStageA = kBM * kBKB;
constexpr uint32_t kStageB = kBN * kBKB;

struct LargeShared {
    uint64_t full[kStages];
    uint64_t empty[kStages];
    uint64_t accf;
    uint32_t tmem_base;
    int32_t timed_out;
    int32_t part[4][kBN];   // per lane-quadrant warp sums of s_i (I_i + h_i)
};

constexpr size_t kSmemBytes = 1024 + kStages * (kStageA + kStageB) + sizeof(LargeShared);

struct LargeArgs {
    RunArgs a;
    uint8_t *S;         // [4][Rpad][Kbytes] spin operand buffers
    int64_t *Epart;     // [2][Rpad] sums of s (I + h) over output tiles, by iteration parity
    int8_t *flags;      // [2][Rpad] improved at an iteration, by parity
    float *X, *V;       // [R][N] state
    int32_t Kbytes, Rpad, mtiles;
    int64_t t;          // iteration of this launch
    int64_t t_first;    // first iteration of this call
};

template <int OP>
__device__ __forceinline__ void put_spin_byte(uint8_t *row, int i, bool plus) {
    if constexpr (OP == kOpE4M3) {
        row[i] = plus ? 0x38 : 0xB8;
    } else {
        reinterpret_cast<uint16_t *>(row)[i] = plus ? 0x3F80 : 0xBF80;
    }
}

template <int OP>
__device__ __forceinline__ bool spin_is_plus(const uint8_t *row, int i) {
    // The sign bit sits in the top byte of the encoding (e4m3: the byte; bf16: byte 1).
    if constexpr (OP == kOpE4M3) return (row[i] & 0x80) == 0;
    else return (row[2 * i + 1] & 0x80) == 0;
}

// Record step for replica r at iteration tt (Table 3, state 5): E from the sum the
// output tiles accumulated, best/target records, improved flag; the sum slot is cleared
// for iteration tt + 2.
__device__ __forceinline__ void settle_replica(const LargeArgs &L, int r, int64_t tt) {
    const RunArgs &a = L.a;
    unsigned long long *slot = reinterpret_cast<unsigned long long *>(L.Epart) + (size_t)(tt & 1) * L.Rpad + r;
    const long long twice = (long long)*slot;
    *slot = 0ull;
    const long long E = -twice / 2;
    int imp = 0;
    const bool frozen = a.stop_at_target && a.hit_step[r] >= 0;
    if (!frozen && E < a.best_e[r]) {
        a.best_e[r] = E;
        a.best_step[r] = tt;
        imp = 1;
    }
    if (a.has_target && a.hit_step[r] < 0 && E <= a.target) a.hit_step[r] = tt;
    L.flags[(size_t)(tt & 1) * L.Rpad + r] = (int8_t)imp;
}

template <int OP>
__global__ void __launch_bounds__(kThreads, 2)
    tc_large_step(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                  const LargeArgs L) {
    constexpr int ESZ = OP == kOpE4M3 ? 1 : 2;
    constexpr uint32_t IDESC = make_idesc(OP == kOpE4M3 ? 0u : 1u, kBM, kBN);
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sA = smem;
    uint8_t *sB = smem + kStages * kStageA;
    LargeShared *sh = reinterpret_cast<LargeShared *>(sB + kStages * kStageB);

    const RunArgs &a = L.a;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m = blockIdx.x, n = blockIdx.y;
    const int64_t t = L.t;
    const int KB = L.Kbytes / kBKB;
    const int N = a.N, R = a.R;

    if (warp == 0) {
        tmem_alloc(&sh->tmem_base, kBN);
        tmem_relinquish();
    }
    if (tid == 32) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&sh->full[s], 1);
            mbar_init(&sh->empty[s], 1);
        }
        mbar_init(&sh->accf, 1);
        sh->timed_out = 0;
        fence_mbarrier_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh->tmem_base;

    if (warp == 0) {
        // TMA producer.
        if (lane == 0) {
            const int ybuf = (int)(t & 3) * L.Rpad + n * kBN;
            for (int kb = 0; kb < KB; ++kb) {
                const int s = kb % kStages;
                if (kb >= kStages && !mbar_wait_bounded(&sh->empty[s], ((kb / kStages) - 1) & 1, kWaitTimeoutNs)) {
                    sh->timed_out = 1;
                    break;
                }
                mbar_arrive_expect_tx(&sh->full[s], kStageA + kStageB);
                tma_load_2d(sA + s * kStageA, &tmA, &sh->full[s], kb * (kBKB / ESZ), m * kBM);
                tma_load_2d(sB + s * kStageB, &tmB, &sh->full[s], kb * (kBKB / ESZ), ybuf);
            }
        }
    } else if (warp == 1) {
        // MMA issuer: 4 K-steps of 32 bytes per stage.
        if (lane == 0) {
            bool ok = true;
            for (int kb = 0; kb < KB; ++kb) {
                const int s = kb % kStages;
                if (!mbar_wait_bounded(&sh->full[s], (kb / kStages) & 1, kWaitTimeoutNs)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint64_t ad = smem_desc_sw128(smem_u32(sA + s * kStageA));
                const uint64_t bd = smem_desc_sw128(smem_u32(sB + s * kStageB));
#pragma unroll
                for (int k = 0; k < kBKB / 32; ++k) {
                    if constexpr (OP == kOpE4M3) mma_e4m3(tmem, ad + 2 * k, bd + 2 * k, IDESC, (kb | k) != 0);
                    else mma_bf16(tmem, ad + 2 * k, bd + 2 * k, IDESC, (kb | k) != 0);
                }
                mma_commit(&sh->empty[s]);
            }
            if (!ok) sh->timed_out = 1;
            mma_commit(&sh->accf);
        }
    } else {
        // Epilogue warps.
        const int ew = warp - 2;
        const int q4 = warp & 3;
        const int half = ew >> 2;
        const int i = m * kBM + q4 * 32 + lane;
        const bool live_i = i < N;
        const int et = ew * 32 + lane;

        // (a) records of iteration t-1 for this replica tile (output tile 0 only).
        if (m == 0 && t - 1 >= L.t_first && et < kBN) {
            const int r = n * kBN + et;
            if (r < R) settle_replica(L, r, t - 1);
        }
        // (b) best spins of iteration t-2 for the replicas that improved then.
        if (t - 2 >= L.t_first) {
            const int rb = n * kBN + half * 64;
            const int8_t *F = L.flags + (size_t)((t - 2) & 1) * L.Rpad;
            const bool f0 = rb + lane < R && F[rb + lane];
            const bool f1 = rb + 32 + lane < R && F[rb + 32 + lane];
            uint64_t todo = (uint64_t)__ballot_sync(0xffffffffu, f0) | ((uint64_t)__ballot_sync(0xffffffffu, f1) << 32);
            const uint8_t *Sb = L.S + (size_t)((t - 2) & 3) * L.Rpad * L.Kbytes;
            const int word = (m * kBM + q4 * 32) >> 5;
            while (todo) {
                // Up to 8 replicas per round, their loads in flight together.
                int js[8];
                bool plus[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    js[u] = todo ? __ffsll((long long)todo) - 1 : -1;
                    if (todo) todo &= todo - 1;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    plus[u] = js[u] >= 0 && live_i && spin_is_plus<OP>(Sb + (size_t)(rb + js[u]) * L.Kbytes, i);
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    if (js[u] < 0) break;
                    const uint32_t bits = __ballot_sync(0xffffffffu, plus[u]);
                    if (lane == 0 && word < a.W) a.best_bits[(size_t)(rb + js[u]) * a.W + word] = bits;
                }
            }
        }
        // (c) the field of this iteration.  x and v of a 16-replica chunk are loaded
        // together (predicated, all in flight at once); chunk 0 before the MMAs finish.
        const int32_t hki = live_i ? a.hk[i] : 0;
        const float bgq = beta_at(t, inv_tm1_of(a.T_total), a.beta0, a.beta1) * (a.gamma * a.q);
        const float eps = a.eps, gamma = a.gamma;
        const bool more = t + 1 < L.t_first + a.nsteps;
        const bool refresh_next = more && refresh_at(t + 1, a.refresh);
        uint8_t *Sn = L.S + (size_t)((t + 1) & 3) * L.Rpad * L.Kbytes;
        const uint32_t tbase = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(half * 64);
        const int rc0 = n * kBN + half * 64;   // first replica of this warp's columns
        float xs[16], vs[16];
        auto load_chunk = [&](int c) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int r = rc0 + c * 16 + j;
                const bool lv = live_i && r < R;
                const size_t idx = (size_t)r * N + i;
                xs[j] = lv ? L.X[idx] : 0.0f;
                vs[j] = lv ? L.V[idx] : 0.0f;
            }
        };
        if (!a.field_mode) load_chunk(0);
        const bool ok = mbar_wait_bounded(&sh->accf, 0, kWaitTimeoutNs);
        if (!ok) sh->timed_out = 1;
        tc_fence_after();
#pragma unroll 1
        for (int c = 0; c < 4; ++c) {
            float acc[16];
            tmem_ld_x16_sync(tbase + c * 16, acc);
            if (a.field_mode) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int r = rc0 + c * 16 + j;
                    int32_t part = 0;
                    if (live_i && r < R && ok) {
                        const size_t idx = (size_t)r * N + i;
                        const int32_t Ik = __float2int_rn(acc[j]) + hki;
                        part = (a.spins_in[idx] > 0 ? 1 : -1) * (Ik + hki);
                        if (a.field_out) a.field_out[idx] = Ik;
                    }
                    part = __reduce_add_sync(0xffffffffu, part);
                    if (lane == 0) sh->part[q4][half * 64 + c * 16 + j] = part;
                }
                continue;
            }
            if (c > 0) load_chunk(c);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int r = rc0 + c * 16 + j;
                const bool lv = live_i && r < R && ok;
                const int32_t Ik = __float2int_rn(acc[j]) + hki;            // Eq. 6, exact
                float x = xs[j], v = vs[j];
                int32_t part = lv ? (x >= 0.0f ? 1 : -1) * (Ik + hki) : 0;
                v = momentum_update(v, x, (float)Ik, eps, bgq, gamma);
                if (more) {
                    if (refresh_next && lv) v = draw_v(a.seed, a.inst, (uint32_t)r, (uint32_t)i, (uint32_t)(t + 1));
                    x = x + eps * v;
                }
                if (lv) {
                    const size_t idx = (size_t)r * N + i;
                    if (more) {
                        L.X[idx] = x;
                        put_spin_byte<OP>(Sn + (size_t)r * L.Kbytes, i, x >= 0.0f);
                    }
                    L.V[idx] = v;
                }
                part = __reduce_add_sync(0xffffffffu, part);
                if (lane == 0) sh->part[q4][half * 64 + c * 16 + j] = part;
            }
        }
        named_barrier_sync(1, 32 * kEpiWarps);
        if (et < kBN) {
            const int r = n * kBN + et;
            const long long s4 = (long long)sh->part[0][et] + sh->part[1][et] + sh->part[2][et] + sh->part[3][et];
            atomicAdd(reinterpret_cast<unsigned long long *>(L.Epart) + (size_t)(t & 1) * L.Rpad + r,
                      (unsigned long long)s4);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && sh->timed_out) atomicExch(a.err, 1);
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, kBN);
    }
}

// Initial state (or given), refresh at t0, first position update, spins of iteration t0.
template <int OP>
__global__ void tc_large_prologue(const LargeArgs L) {
    const RunArgs &a = L.a;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)a.R * a.N) return;
    const int r = (int)(idx / a.N), i = (int)(idx - (int64_t)r * a.N);
    float x, v;
    if (a.x_in) {
        x = a.x_in[idx];
        v = a.v_in[idx];
    } else {
        const U4 o = draw_raw(a.seed, a.inst, (uint32_t)r, (uint32_t)i, 0u);
        x = box_muller(o.x, o.y);
        v = box_muller(o.z, o.w);
    }
    if (refresh_at(a.t0, a.refresh)) v = draw_v(a.seed, a.inst, (uint32_t)r, (uint32_t)i, (uint32_t)a.t0);
    x = x + a.eps * v;
    L.X[idx] = x;
    L.V[idx] = v;
    put_spin_byte<OP>(L.S + ((size_t)(a.t0 & 3) * L.Rpad + r) * L.Kbytes, i, x >= 0.0f);
}

// Field-only mode: spins given, field and energy out (no records).
template <int OP>
__global__ void tc_large_field_prologue(const LargeArgs L) {
    const RunArgs &a = L.a;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)a.R * a.N) return;
    const int r = (int)(idx / a.N), i = (int)(idx - (int64_t)r * a.N);
    put_spin_byte<OP>(L.S + (size_t)r * L.Kbytes, i, a.spins_in[idx] > 0);
}

__global__ void tc_large_settle(const LargeArgs L, int64_t tt) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < L.a.R) settle_replica(L, r, tt);
}

// Best spins of the iterations not copied by a later launch (tt in {t_last-1, t_last}).
template <int OP>
__global__ void tc_large_copy(const LargeArgs L, int64_t t_from, int64_t t_last) {
    const RunArgs &a = L.a;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)a.R * a.W) return;
    const int r = (int)(idx / a.W), w = (int)(idx - (int64_t)r * a.W);
    for (int64_t tt = t_from; tt <= t_last; ++tt) {
        if (!L.flags[(size_t)(tt & 1) * L.Rpad + r]) continue;
        const uint8_t *row = L.S + ((size_t)(tt & 3) * L.Rpad + r) * L.Kbytes;
        uint32_t bits = 0;
        for (int b = 0; b < 32; ++b) {
            const int i = w * 32 + b;
            if (i < a.N && spin_is_plus<OP>(row, i)) bits |= 1u << b;
        }
        a.best_bits[idx] = bits;
    }
}

// Field-only epilogue: the field of buffer 0 and its energy.
__global__ void tc_large_field_out(const LargeArgs L) {
    const RunArgs &a = L.a;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.R) return;
    unsigned long long *slot = reinterpret_cast<unsigned long long *>(L.Epart) + r;
    if (a.energy_out) a.energy_out[r] = -((long long)*slot) / 2;
    *slot = 0ull;
}

__global__ void tc_large_count(const LargeArgs L) {
    if (threadIdx.x == 0 && blockIdx.x == 0)
        atomicAdd(L.a.replica_iters, (unsigned long long)((long long)L.a.R * L.a.nsteps));
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

bool make_map(CUtensorMap *m, const void *base, int op, uint64_t inner_elems, uint64_t rows, uint64_t row_bytes,
              uint32_t box_rows) {
    auto enc = encode_fn();
    if (!enc) return false;
    const CUtensorMapDataType dt = op == kOpE4M3 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const cuuint64_t dims[2] = {inner_elems, rows};
    const cuuint64_t strides[1] = {row_bytes};
    const cuuint32_t box[2] = {(cuuint32_t)(kBKB / (op == kOpE4M3 ? 1 : 2)), box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(m, dt, 2, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int OP>
cudaError_t run_large(const LargeBuffers &B, const RunArgs &a, cudaStream_t st, int *launches) {
    LargeArgs L;
    L.a = a;
    L.S = B.S;
    L.Epart = B.Epart;
    L.flags = B.flags;
    L.Kbytes = B.Kbytes;
    L.Rpad = B.Rpad;
    L.mtiles = B.Mpad / kBM;
    L.t_first = a.t0;
    L.X = a.x_out ? a.x_out : B.X;
    L.V = a.v_out ? a.v_out : B.V;
    CUtensorMap tmA, tmB;
    const int esz = OP == kOpE4M3 ? 1 : 2;
    if (!make_map(&tmA, B.Jop, OP, (uint64_t)B.Kbytes / esz, (uint64_t)B.Mpad, (uint64_t)B.Kbytes, kBM) ||
        !make_map(&tmB, B.S, OP, (uint64_t)B.Kbytes / esz, (uint64_t)4 * B.Rpad, (uint64_t)B.Kbytes, kBN))
        return cudaErrorInvalidValue;
    auto step = tc_large_step<OP>;
    cudaError_t e = cudaFuncSetAttribute(step, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    const dim3 grid(B.Mpad / kBM, B.Rpad / kBN);
    e = cudaMemsetAsync(B.Epart, 0, 2 * (size_t)B.Rpad * sizeof(int64_t), st);   // energy sums start at 0
    if (e != cudaSuccess) return e;
    const int64_t RN = (int64_t)a.R * a.N;
    const unsigned eg = (unsigned)((RN + 255) / 256);
    int n = 0;
    if (a.field_mode) {
        L.t = 0;
        L.t_first = 0;
        L.a.nsteps = 1;
        L.a.T_total = 1;
        tc_large_field_prologue<OP><<<eg, 256, 0, st>>>(L);
        step<<<grid, kThreads, kSmemBytes, st>>>(tmA, tmB, L);
        tc_large_field_out<<<(a.R + 255) / 256, 256, 0, st>>>(L);
        n += 3;
        if (launches) *launches += n;
        return cudaGetLastError();
    }
    tc_large_prologue<OP><<<eg, 256, 0, st>>>(L);
    ++n;
    for (int64_t t = a.t0; t < a.t0 + a.nsteps; ++t) {
        L.t = t;
        step<<<grid, kThreads, kSmemBytes, st>>>(tmA, tmB, L);
        ++n;
    }
    const int64_t t_last = a.t0 + a.nsteps - 1;
    tc_large_settle<<<(a.R + 255) / 256, 256, 0, st>>>(L, t_last);
    const int64_t RW = (int64_t)a.R * a.W;
    tc_large_copy<OP><<<(unsigned)((RW + 255) / 256), 256, 0, st>>>(L, t_last - 1 >= a.t0 ? t_last - 1 : t_last,
                                                                     t_last);
    tc_large_count<<<1, 32, 0, st>>>(L);
    n += 3;
    if (launches) *launches += n;
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tc_large(const LargeBuffers &B, const RunArgs &a, int op, cudaStream_t st, int *launches) {
    if (op == kOpE4M3) return run_large<kOpE4M3>(B, a, st, launches);
    return run_large<kOpBF16>(B, a, st, launches);
}

size_t tc_large_smem_bytes() { return kSmemBytes; }

}  // namespace phia
