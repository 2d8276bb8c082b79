// k_imma.cu -- resident PHIA kernel on the int8 tensor-core path (warp-level
// mma.sync m16n8k32 s8 x s8 -> s32) for small dense instances, all iterations in one
// launch.  The field I = J s + h (Eq. 6) is an exact int32 product of the int8
// couplings and the +-1 spins.
//
// One CTA owns 8 * NT replicas; warp w owns output spins [16w, 16w + 16).
//  - A = the warp's 16 rows of J as mma A fragments, loaded once into registers;
//  - B = the spins of the CTA's replicas, int8 [replica][K] in shared memory (four
//    rotating buffers: iteration t reads t % 4, writes t + 1 % 4; t - 1 stays intact for
//    the lagged best-state copy);
//  - D = J s lands in registers: lane (g, tq) holds spins 16w + g and 16w + g + 8 for
//    replicas 2 tq and 2 tq + 1 of each 8-replica tile.
// x and v of those (spin, replica) pairs stay in registers.  Per iteration: MMAs ->
// field -> energy terms s (I + h) (Eq. 2 via Eq. 6) reduced per replica -> momentum
// update (Eqs. 5, 8, A7) -> refresh -> position and sign written into the next B ->
// one __syncthreads -> records (Table 3, state 5) by the first 8 NT threads and the
// best spins of the previous iteration by ballot.
#include "device_common.cuh"
#include "phia_internal.h"

namespace phia {

namespace {

constexpr int kMaxWarpsImma = 16;    // N <= 256

struct ImmaShared {
    int32_t e_part[2][kMaxWarpsImma][16];   // per-warp sums of s (I + h), by iteration parity
    long long best_e[16];
    long long best_step[16];
    long long hit[16];
    int32_t improved[2][16];
    int32_t stop[2];
};

__device__ __forceinline__ void imma_16832(int32_t (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// KS: K-steps of 32 spins (Kpad = 32 KS); NT: 8-replica tiles per CTA.
template <int KS, int NT>
__global__ void __launch_bounds__(64 * KS, 1) imma_small_kernel(const RunArgs a, int nwarps) {
    constexpr int RL = 8 * NT;
    constexpr int KP = 32 * KS + 16;     // B row pitch in bytes (16-byte skew: conflict-free B loads)
    extern __shared__ __align__(16) uint8_t smem[];
    int8_t *B = reinterpret_cast<int8_t *>(smem);                   // [4][RL][KP]
    ImmaShared *sm = reinterpret_cast<ImmaShared *>(smem + 4 * RL * KP);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, tq = lane & 3;
    const int N = a.N;
    const int rbase = blockIdx.x * RL;
    const int i0 = 16 * warp + g, i1 = i0 + 8;       // this thread's two output spins
    const bool l0 = i0 < N, l1 = i1 < N;

    // A fragments of this warp's rows, once.
    uint32_t af[KS][4];
    auto jbyte = [&](int row, int col) -> uint32_t {
        return (row < N && col < N) ? (uint32_t)(uint8_t)a.Jk[(size_t)row * N + col] : 0u;
    };
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
        const int c0 = 32 * ks + 4 * tq;
        uint32_t w[4] = {0, 0, 0, 0};
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            w[0] |= jbyte(i0, c0 + b) << (8 * b);
            w[1] |= jbyte(i1, c0 + b) << (8 * b);
            w[2] |= jbyte(i0, c0 + 16 + b) << (8 * b);
            w[3] |= jbyte(i1, c0 + 16 + b) << (8 * b);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) af[ks][q] = w[q];
    }
    for (int e = tid; e < 4 * RL * KP / 16; e += blockDim.x) reinterpret_cast<uint4 *>(B)[e] = make_uint4(0, 0, 0, 0);
    if (tid < 16) {
        const int r = rbase + tid;
        sm->improved[0][tid] = sm->improved[1][tid] = 0;
        const bool rec = !a.field_mode && tid < RL && r < a.R;
        sm->best_e[tid] = rec ? a.best_e[r] : LLONG_MAX;
        sm->best_step[tid] = rec ? a.best_step[r] : -1;
        sm->hit[tid] = rec ? a.hit_step[r] : -1;
    }
    if (tid == 0) sm->stop[0] = sm->stop[1] = 0;
    const int32_t h0 = l0 ? a.hk[i0] : 0, h1 = l1 ? a.hk[i1] : 0;
    __syncthreads();

    // State: q = 4 nt + 2 j + u -> spin (u ? i1 : i0), replica nt * 8 + 2 tq + j.
    float x[4 * NT], v[4 * NT];
    const int8_t *Bt = B + (size_t)(a.t0 & 3) * RL * KP;
    int8_t *Bw = const_cast<int8_t *>(Bt);
#pragma unroll
    for (int q = 0; q < 4 * NT; ++q) {
        const int nt = q >> 2, j = (q >> 1) & 1, u = q & 1;
        const int c = nt * 8 + 2 * tq + j, r = rbase + c;
        const int i = u ? i1 : i0;
        const bool live = u ? l1 : l0;
        x[q] = 0.0f; v[q] = 0.0f;
        if (!live) continue;
        if (a.field_mode) {
            if (r < a.R) Bw[c * KP + i] = a.spins_in[(size_t)r * N + i] > 0 ? 1 : -1;
            continue;
        }
        if (a.x_in) {
            x[q] = r < a.R ? a.x_in[(size_t)r * N + i] : 0.0f;
            v[q] = r < a.R ? a.v_in[(size_t)r * N + i] : 0.0f;
        } else {
            const U4 o = draw_raw(a.seed, a.inst, (uint32_t)r, (uint32_t)i, 0u);
            x[q] = box_muller(o.x, o.y);
            v[q] = box_muller(o.z, o.w);
        }
        if (refresh_at(a.t0, a.refresh)) v[q] = draw_v(a.seed, a.inst, (uint32_t)r, (uint32_t)i, (uint32_t)a.t0);
        x[q] = x[q] + a.eps * v[q];
        Bw[c * KP + i] = x[q] >= 0.0f ? 1 : -1;
    }
    __syncthreads();

    const int nit = a.field_mode ? 1 : (int)a.nsteps;
    const float inv_tm1 = inv_tm1_of(a.T_total);
    const float eps = a.eps, gamma = a.gamma, gq = a.gamma * a.q;
    int rc = a.refresh > 0 ? (int)((a.t0 + 1) % a.refresh) : 1;
    bool stopped = false;
    int it = 0;
    for (; it < nit; ++it) {
        const int64_t t = a.t0 + it;
        const int8_t *Bc = B + (size_t)((t) & 3) * RL * KP;
        int8_t *Bn = B + (size_t)((t + 1) & 3) * RL * KP;
        // Field: D = J s over the K-steps (exact int32).
        int32_t d[NT][4];
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) d[nt][0] = d[nt][1] = d[nt][2] = d[nt][3] = 0;
#pragma unroll
        for (int ks = 0; ks < KS; ++ks) {
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                const int8_t *row = Bc + (nt * 8 + g) * KP + 32 * ks + 4 * tq;
                const uint32_t b0 = *reinterpret_cast<const uint32_t *>(row);
                const uint32_t b1 = *reinterpret_cast<const uint32_t *>(row + 16);
                imma_16832(d[nt], af[ks], b0, b1);
            }
        }
        // Energy terms, warp sums per replica, then the updates.
        int32_t Ik[4 * NT], part[2 * NT];
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            Ik[4 * nt + 0] = d[nt][0] + h0;   // (i0, j = 0)
            Ik[4 * nt + 1] = d[nt][2] + h1;   // (i1, j = 0)
            Ik[4 * nt + 2] = d[nt][1] + h0;   // (i0, j = 1)
            Ik[4 * nt + 3] = d[nt][3] + h1;   // (i1, j = 1)
        }
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                int32_t p = 0;
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int q = 4 * nt + 2 * j + u;
                    const bool live = u ? l1 : l0;
                    const int32_t hh = u ? h1 : h0;
                    const bool plus = a.field_mode
                                          ? (Bc[(nt * 8 + 2 * tq + j) * KP + (u ? i1 : i0)] > 0)
                                          : (x[q] >= 0.0f);
                    if (live) p += plus ? (Ik[q] + hh) : -(Ik[q] + hh);
                }
                part[2 * nt + j] = p;
            }
#pragma unroll
        for (int e = 0; e < 2 * NT; ++e) {
            part[e] += __shfl_xor_sync(0xffffffffu, part[e], 4);
            part[e] += __shfl_xor_sync(0xffffffffu, part[e], 8);
            part[e] += __shfl_xor_sync(0xffffffffu, part[e], 16);
        }
        if (g == 0) {
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                sm->e_part[it & 1][warp][nt * 8 + 2 * tq] = part[2 * nt];
                sm->e_part[it & 1][warp][nt * 8 + 2 * tq + 1] = part[2 * nt + 1];
            }
        }
        if (a.field_mode) {
#pragma unroll
            for (int q = 0; q < 4 * NT; ++q) {
                const int nt = q >> 2, j = (q >> 1) & 1, u = q & 1;
                const int r = rbase + nt * 8 + 2 * tq + j, i = u ? i1 : i0;
                if ((u ? l1 : l0) && r < a.R && a.field_out) a.field_out[(size_t)r * N + i] = Ik[q];
            }
        } else {
            const float bgq = beta_at(t, inv_tm1, a.beta0, a.beta1) * gq;
            const bool more = it + 1 < nit;
            if (a.deriv == 1) {
#pragma unroll
                for (int q = 0; q < 4 * NT; ++q) v[q] = momentum_quad(v[q], x[q], (float)Ik[q], eps, bgq, gamma);
            } else {
#pragma unroll
                for (int q = 0; q < 4 * NT; ++q) v[q] = momentum_exact(v[q], x[q], (float)Ik[q], eps, bgq, gamma);
            }
            if (more) {
                if (a.refresh > 0 && rc == 0) {
#pragma unroll
                    for (int q = 0; q < 4 * NT; ++q) {
                        const int nt = q >> 2, j = (q >> 1) & 1, u = q & 1;
                        v[q] = draw_v(a.seed, a.inst, (uint32_t)(rbase + nt * 8 + 2 * tq + j), (uint32_t)(u ? i1 : i0),
                                      (uint32_t)(t + 1));
                    }
                }
#pragma unroll
                for (int q = 0; q < 4 * NT; ++q) {
                    const int nt = q >> 2, j = (q >> 1) & 1, u = q & 1;
                    x[q] = x[q] + eps * v[q];
                    if (u ? l1 : l0) Bn[(nt * 8 + 2 * tq + j) * KP + (u ? i1 : i0)] = x[q] >= 0.0f ? 1 : -1;
                }
            }
        }
        __syncthreads();
        // Records of iteration t, one thread per replica.
        if (tid < RL) {
            const int c = tid, r = rbase + c;
            long long twice = 0;
            for (int w = 0; w < nwarps; ++w) twice += sm->e_part[it & 1][w][c];
            const long long E = -twice / 2;
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
                    if (a.hit_ns) a.hit_ns[r] = globaltimer_ns();
                    if (a.stop_at_target) atomicMin(a.min_hit, (unsigned long long)t);
                }
            }
            sm->improved[it & 1][c] = imp;
        }
        if (tid == 0)
            sm->stop[it & 1] = (a.stop_at_target && !a.field_mode)
                                   ? (*(volatile unsigned long long *)a.min_hit <= (unsigned long long)t)
                                   : 0;
        // Best spins of iteration t-1 (buffer (t-1) % 4 is intact until iteration t+2).
        if (it > 0 && warp < a.W) {
            const int8_t *Bp = B + (size_t)((t - 1) & 3) * RL * KP;
            for (int c = 0; c < RL; ++c) {
                if (!sm->improved[(it - 1) & 1][c]) continue;
                const int i = 32 * warp + lane;
                const uint32_t bits = __ballot_sync(0xffffffffu, i < N && Bp[c * KP + i] > 0);
                if (lane == 0) a.best_bits[(size_t)(rbase + c) * a.W + warp] = bits;
            }
        }
        rc = (a.refresh > 0 && rc + 1 == a.refresh) ? 0 : rc + 1;
        if (it > 0 && sm->stop[(it - 1) & 1]) { stopped = true; ++it; break; }
    }
    __syncthreads();   // records of the last iteration settled
    if (it > 0 && warp < a.W) {
        const int64_t tl = a.t0 + it - 1;
        const int8_t *Bp = B + (size_t)(tl & 3) * RL * KP;
        for (int c = 0; c < RL; ++c) {
            if (!sm->improved[(it - 1) & 1][c]) continue;
            const int i = 32 * warp + lane;
            const uint32_t bits = __ballot_sync(0xffffffffu, i < N && Bp[c * KP + i] > 0);
            if (lane == 0) a.best_bits[(size_t)(rbase + c) * a.W + warp] = bits;
        }
    }
    if (!a.field_mode && !stopped && a.x_out) {
#pragma unroll
        for (int q = 0; q < 4 * NT; ++q) {
            const int nt = q >> 2, j = (q >> 1) & 1, u = q & 1;
            const int r = rbase + nt * 8 + 2 * tq + j, i = u ? i1 : i0;
            if ((u ? l1 : l0) && r < a.R) {
                a.x_out[(size_t)r * N + i] = x[q];
                a.v_out[(size_t)r * N + i] = v[q];
            }
        }
    }
    if (tid < RL && !a.field_mode) {
        const int r = rbase + tid;
        if (r < a.R) {
            a.best_e[r] = sm->best_e[tid];
            a.best_step[r] = sm->best_step[tid];
            a.hit_step[r] = sm->hit[tid];
        }
    }
    if (tid == 0 && !a.field_mode) {
        const int valid = min(RL, a.R - rbase);
        atomicAdd(a.replica_iters, (unsigned long long)((long long)valid * it));
    }
}

template <int KS, int NT>
cudaError_t launch_ks(const RunArgs &a, cudaStream_t st) {
    constexpr int RL = 8 * NT;
    constexpr int KP = 32 * KS + 16;
    const int nwarps = (a.N + 15) / 16;
    const size_t smem = (size_t)4 * RL * KP + sizeof(ImmaShared);
    auto kern = imma_small_kernel<KS, NT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(a.R + RL - 1) / RL, 32 * nwarps, smem, st>>>(a, nwarps);
    return cudaGetLastError();
}

template <int NT>
cudaError_t launch_nt(const RunArgs &a, cudaStream_t st) {
    const int ks = (a.N + 31) / 32;
    if (ks <= 2) return launch_ks<2, NT>(a, st);
    if (ks <= 4) return launch_ks<4, NT>(a, st);
    if (ks <= 7) return launch_ks<7, NT>(a, st);
    return launch_ks<8, NT>(a, st);
}

}  // namespace

int imma_small_max_n() { return 16 * kMaxWarpsImma; }

cudaError_t launch_imma_small(const RunArgs &a, cudaStream_t st, int *launches) {
    if (a.N > imma_small_max_n()) return cudaErrorInvalidValue;
    if (launches) *launches += 1;
    if (a.tile_rl == 16) return launch_nt<2>(a, st);
    return launch_nt<1>(a, st);
}

}  // namespace phia
