// k_inc.cu -- incremental-field PHIA kernel for small dense instances (N <= 384), all
// iterations in one launch.
//
// Eq. 6 is linear in s: if the spins of iteration t+1 differ from those of iteration t
// in the positions F, then I(t+1) = I(t) + sum_{j in F} J[:, j] (s_j(t+1) - s_j(t)) with
// s_j(t+1) - s_j(t) = 2 s_j(t+1).  In an anneal a few percent of the spins change sign
// per iteration early on and well under one percent late, so gathering the changed
// columns replaces the full product.  Every term is an integer, so the field is
// bit-identical to J s + h computed from scratch (and to the tensor-core kernels).
//
// One CTA owns RL = RPT * G replicas of one instance for the whole run.  The couplings k
// (int8, exact) sit in shared memory as rows J[j][0..S) (J is symmetric, so row j is
// column j, and the 32 lanes of a warp read 32 consecutive bytes).  Thread (group g,
// spin i) keeps x, v and the integer field I (h included) of spin i for replicas
// g*RPT .. g*RPT+RPT-1 in registers.  Per iteration (Eq. A7): energy terms s (I + h) and
// their warp sums (Eq. 2), momentum and position update (Eqs. 5, 8), optional refresh,
// the new signs; each replica's changed spins are appended to a shared list (one shared
// atomic per warp and replica); one barrier; then the gather of the listed columns.  A
// control warp keeps the records (Table 3, state 5) in parallel with the next
// iteration.  The lists rotate over three buffers, so a buffer is cleared one iteration
// before it is filled and after it was last read.
#include <climits>

#include "device_common.cuh"
#include "phia_internal.h"

namespace phia {

namespace {

constexpr int kIncMaxRL = 16;
constexpr int kIncMaxWarps = 32;
constexpr int kIncMaxRPT = 4;

struct IncShared {
    int32_t cnt[3][kIncMaxRL];                    // list lengths, by iteration mod 3
    int32_t e_part[2][kIncMaxWarps][kIncMaxRPT];  // per-warp sums of s_i (I_i + h_i), by parity
    long long best_e[kIncMaxRL];
    long long best_step[kIncMaxRL];
    long long hit[kIncMaxRL];
    int32_t improved[2][kIncMaxRL];
    int32_t stop[2];
};

__host__ __device__ constexpr int align16(int x) { return (x + 15) & ~15; }

// Shared-memory bytes: J rows [N][S], the initial spins [RL][S], 3 lists [RL][N] of int32.
__host__ __device__ inline int inc_smem_bytes(int N, int RL) {
    const int S = (N + 31) / 32 * 32;
    return align16(N * S) + align16(RL * S) + 3 * RL * N * 4 + (int)sizeof(IncShared);
}

template <int RPT, int G>
__global__ void __launch_bounds__(1024) inc_small_kernel(const RunArgs a) {
    constexpr int RL = RPT * G;
    static_assert(RL <= kIncMaxRL && RPT <= kIncMaxRPT, "shared records too small");
    extern __shared__ __align__(16) uint8_t smem[];
    const int N = a.N;
    const int WG = (N + 31) / 32;          // warps per replica group
    const int S = WG * 32;                 // spin slots: row stride of J in shared memory
    const int NW = WG * G;                 // update warps; warp NW is the control warp
    int8_t *Js = reinterpret_cast<int8_t *>(smem);
    int8_t *sp0 = Js + align16(N * S);                                     // [RL][S] spins of t0
    int32_t *lists = reinterpret_cast<int32_t *>(sp0 + align16(RL * S));   // [3][RL][N]
    IncShared *sm = reinterpret_cast<IncShared *>(lists + 3 * RL * N);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool ctl = warp >= NW;
    const int g = ctl ? 0 : warp / WG;     // replica group of this warp
    const int i = (warp - g * WG) * 32 + lane;
    const bool live_i = !ctl && i < N;
    const int c0 = g * RPT;                // first replica column of this thread
    const int rbase = blockIdx.x * RL;

    for (int idx = tid; idx < N * S; idx += blockDim.x) {
        const int j = idx / S, col = idx - j * S;
        Js[idx] = col < N ? a.Jk[(size_t)j * N + col] : (int8_t)0;
    }
    if (tid < 3 * kIncMaxRL) (&sm->cnt[0][0])[tid] = 0;
    if (tid < RL) {
        const int r = rbase + tid;
        sm->improved[0][tid] = 0;
        sm->improved[1][tid] = 0;
        const bool rec = r < a.R;
        sm->best_e[tid] = rec ? a.best_e[r] : LLONG_MAX;
        sm->best_step[tid] = rec ? a.best_step[r] : -1;
        sm->hit[tid] = rec ? a.hit_step[r] : -1;
    }
    if (tid == 0) sm->stop[0] = sm->stop[1] = 0;

    // Initial state (given, or Philox draw d = 0), refresh at t0, first position update.
    const int32_t hki = live_i ? a.hk[i] : 0;
    float x[RPT], v[RPT];
    int32_t I[RPT];
    uint32_t cur = 0;   // bit k: spin i of replica c0 + k is +1 at the current iteration
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        const int r = rbase + c0 + k;
        x[k] = 0.0f; v[k] = 0.0f; I[k] = hki;
        if (!live_i) continue;
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
        cur |= (uint32_t)(x[k] >= 0.0f) << k;       // sgn with sgn(0) = +1
    }
    if (!ctl) {
#pragma unroll
        for (int k = 0; k < RPT; ++k) sp0[(c0 + k) * S + i] = live_i ? (((cur >> k) & 1u) ? 1 : -1) : 0;
    }
    __syncthreads();
    // Field of the initial spins, Eq. 6 in full.
    if (live_i) {
        for (int j = 0; j < N; ++j) {
            const int32_t kij = Js[j * S + i];
#pragma unroll
            for (int k = 0; k < RPT; ++k) I[k] += kij * (int32_t)sp0[(c0 + k) * S + j];
        }
    }
    const int word = warp - g * WG;        // 32-spin word of the best state this warp writes
    const int nit = (int)a.nsteps;
    const float inv_tm1 = inv_tm1_of(a.T_total);
    const float eps = a.eps, gamma = a.gamma, gq = a.gamma * a.q;
    int rc = a.refresh > 0 ? (int)((a.t0 + 1) % a.refresh) : 1;   // (t + 1) mod refresh
    uint32_t prv = 0;
    bool stopped = false;
    int it = 0;
    for (; it < nit; ++it) {
        const int64_t t = a.t0 + it;
        const int buf = it % 3;
        uint32_t nxt = 0;
        if (!ctl) {
            // Energy terms of iteration t and their warp sums.
            int32_t part[RPT];
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                const int32_t e = I[k] + hki;
                part[k] = live_i ? (((cur >> k) & 1u) ? e : -e) : 0;
            }
#pragma unroll
            for (int k = 0; k < RPT; ++k) part[k] = __reduce_add_sync(0xffffffffu, part[k]);
            if (lane == 0) {
#pragma unroll
                for (int k = 0; k < RPT; ++k) sm->e_part[it & 1][warp][k] = part[k];
            }
            const bool more = it + 1 < nit;
            if (live_i) {
                const float bgq = beta_at(t, inv_tm1, a.beta0, a.beta1) * gq;
                if (a.deriv == 1) {
#pragma unroll
                    for (int k = 0; k < RPT; ++k) v[k] = momentum_quad(v[k], x[k], (float)I[k], eps, bgq, gamma);
                } else {
#pragma unroll
                    for (int k = 0; k < RPT; ++k) v[k] = momentum_exact(v[k], x[k], (float)I[k], eps, bgq, gamma);
                }
                if (more) {
                    if (a.refresh > 0 && rc == 0) {
#pragma unroll
                        for (int k = 0; k < RPT; ++k)
                            v[k] = draw_v(a.seed, a.inst, (uint32_t)(rbase + c0 + k), (uint32_t)i, (uint32_t)(t + 1));
                    }
#pragma unroll
                    for (int k = 0; k < RPT; ++k) {
                        x[k] = x[k] + eps * v[k];
                        nxt |= (uint32_t)(x[k] >= 0.0f) << k;
                    }
                }
            }
            // Spins that change sign between t and t+1, per replica: entry 2 (j S) + [s_j = +1],
            // j S being the offset of row j of J in shared memory.
            // Lane k reserves the warp's slots of replica c0 + k (the RPT atomics go out
            // together), then every lane places its own entries.
            if (more) {
                const uint32_t lt_mask = (1u << lane) - 1u;
                const uint32_t flips = live_i ? (cur ^ nxt) : 0u;
                uint32_t m[RPT];
#pragma unroll
                for (int k = 0; k < RPT; ++k) m[k] = __ballot_sync(0xffffffffu, (flips >> k) & 1u);
                uint32_t mine = 0;
#pragma unroll
                for (int k = 0; k < RPT; ++k) mine = lane == k ? m[k] : mine;
                int base = 0;
                if (lane < RPT && mine) base = atomicAdd(&sm->cnt[buf][c0 + lane], __popc(mine));
#pragma unroll
                for (int k = 0; k < RPT; ++k) {
                    const int b = __shfl_sync(0xffffffffu, base, k);
                    if ((flips >> k) & 1u)
                        lists[(buf * RL + c0 + k) * N + b + __popc(m[k] & lt_mask)] = 2 * (i * S) + (int32_t)((nxt >> k) & 1u);
                }
            }
        } else if (lane < RL) {
            // The buffer of the iteration after next was last read two iterations ago.
            sm->cnt[(it + 1) % 3][lane] = 0;
        }
        __syncthreads();
        if (ctl) {
            // Records of iteration t (Table 3, state 5), one lane per replica column.
            if (lane < RL) {
                const int c = lane, r = rbase + c;
                long long twice = 0;   // sum_i s_i (I_i + h_i) over the WG warps of replica c's group
                for (int w = 0; w < WG; ++w) twice += sm->e_part[it & 1][(c / RPT) * WG + w][c % RPT];
                const long long E = -twice / 2;                                  // Eq. 2 via the field
                int imp = 0;
                if (r < a.R) {
                    const bool frozen = a.stop_at_target && sm->hit[c] >= 0;
                    if (!frozen && E < sm->best_e[c]) {
                        sm->best_e[c] = E;
                        sm->best_step[c] = t;
                        imp = 1;
                    }
                    if (a.has_target && sm->hit[c] < 0 && E <= a.target) {
                        sm->hit[c] = t;
                        if (a.hit_ns) a.hit_ns[r] = globaltimer_ns();
                        if (a.stop_at_target) atomicMin(a.min_hit, (unsigned long long)t);
                    }
                }
                sm->improved[it & 1][c] = imp;
            }
            if (lane == 0)
                sm->stop[it & 1] = a.stop_at_target
                                       ? (*(volatile unsigned long long *)a.min_hit <= (unsigned long long)t)
                                       : 0;
        } else {
            if (it > 0) {
                // Best spins of iteration t-1 (its records were settled before this barrier).
#pragma unroll
                for (int k = 0; k < RPT; ++k) {
                    if (sm->improved[(it - 1) & 1][c0 + k]) {
                        const uint32_t bits = __ballot_sync(0xffffffffu, live_i && ((prv >> k) & 1u));
                        if (lane == 0 && word < a.W) a.best_bits[(size_t)(rbase + c0 + k) * a.W + word] = bits;
                    }
                }
            }
            // Field of iteration t+1: the changed columns, each adding 2 s_j(t+1) k_ij.
            if (live_i && it + 1 < nit) {
                const int8_t *Ji = Js + i;
#pragma unroll
                for (int k = 0; k < RPT; ++k) {
                    const int n = sm->cnt[buf][c0 + k];
                    const int32_t *L = lists + (buf * RL + c0 + k) * N;
                    int32_t acc0 = 0, acc1 = 0;
                    int f = 0;
                    for (; f + 1 < n; f += 2) {
                        const int32_t e0 = L[f], e1 = L[f + 1];
                        const int32_t k0 = Ji[e0 >> 1], k1 = Ji[e1 >> 1];
                        acc0 += (e0 & 1) ? k0 : -k0;
                        acc1 += (e1 & 1) ? k1 : -k1;
                    }
                    if (f < n) {
                        const int32_t e0 = L[f];
                        const int32_t k0 = Ji[e0 >> 1];
                        acc0 += (e0 & 1) ? k0 : -k0;
                    }
                    I[k] += 2 * (acc0 + acc1);
                }
            }
        }
        prv = cur;
        cur = nxt;
        rc = (a.refresh > 0 && rc + 1 == a.refresh) ? 0 : rc + 1;
        if (it > 0 && sm->stop[(it - 1) & 1]) { stopped = true; ++it; break; }
    }
    __syncthreads();   // records of the last iteration settled
    const int last = it - 1;
    if (!ctl) {
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            if (last >= 0 && sm->improved[last & 1][c0 + k]) {
                const uint32_t bits = __ballot_sync(0xffffffffu, live_i && ((prv >> k) & 1u));
                if (lane == 0 && word < a.W) a.best_bits[(size_t)(rbase + c0 + k) * a.W + word] = bits;
            }
        }
    }
    if (!stopped && a.x_out && live_i) {
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const int r = rbase + c0 + k;
            if (r < a.R) {
                a.x_out[(size_t)r * N + i] = x[k];
                a.v_out[(size_t)r * N + i] = v[k];
            }
        }
    }
    if (ctl && lane < RL) {
        const int r = rbase + lane;
        if (r < a.R) {
            a.best_e[r] = sm->best_e[lane];
            a.best_step[r] = sm->best_step[lane];
            a.hit_step[r] = sm->hit[lane];
        }
    }
    if (ctl && lane == 0) {
        const int valid = min(RL, a.R - rbase);
        atomicAdd(a.replica_iters, (unsigned long long)((long long)valid * it));
    }
}

template <int RPT, int G>
cudaError_t launch_g(const RunArgs &a, cudaStream_t st) {
    constexpr int RL = RPT * G;
    const int smem = inc_smem_bytes(a.N, RL);
    auto kern = inc_small_kernel<RPT, G>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int WG = (a.N + 31) / 32;
    const int grid = (a.R + RL - 1) / RL;
    kern<<<grid, 32 * (WG * G + 1), smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

int inc_small_max_n() { return 384; }

// Replicas per CTA the kernel can take for N: 4, 8 or 16 (threads and shared memory
// permitting), the requested one if possible, else the largest not above it.
int inc_small_tile_replicas(int N, int requested) {
    const int WG = (N + 31) / 32;
    int rl = requested == 4 || requested == 8 || requested == 16 ? requested : 8;
    while (rl > 4 && (WG * (rl / 4) + 1 > 32 || inc_smem_bytes(N, rl) > 227 * 1024)) rl /= 2;
    return rl;
}

cudaError_t launch_inc_small(const RunArgs &a, cudaStream_t st, int *launches) {
    if (a.field_mode || a.N > inc_small_max_n()) return cudaErrorInvalidValue;
    if (launches) *launches += 1;
    const int rl = inc_small_tile_replicas(a.N, a.tile_rl);
    const int WG = (a.N + 31) / 32;
    // Two replicas per thread where the block has room (more warps hide more latency).
    if (rl == 16) return launch_g<4, 4>(a, st);
    if (rl == 8) return WG * 4 + 1 <= 32 ? launch_g<2, 4>(a, st) : launch_g<4, 2>(a, st);
    return WG * 2 + 1 <= 32 ? launch_g<2, 2>(a, st) : launch_g<4, 1>(a, st);
}

}  // namespace phia
