// k_gahmc.cu -- vanilla GAHMC: the exact solution of the dynamics of
// H(x, v) = beta E(sgn x) + x.x/2 + v.v/2 (Eq. 4, App. A) by zero crossings, the method of
// the paper's reference [Pakman & Paninski 2013] that Sec. 2.1 names as the exact
// alternative to PHIA's approximate gradient and Sec. 3.2 uses as an ablation.
//
// Inside an orthant each coordinate rotates on the unit circle:
// x_i(t) = x_i cos t + v_i sin t, v_i(t) = -x_i sin t + v_i cos t.  At a wall x_j = 0 the
// potential would jump by dU = beta q dE, dE = 2 s_j I_j (the flip identity of Eqs. 2 and
// 6); with wall speed A_j = sqrt(x_j^2 + v_j^2) the coordinate crosses with speed
// sqrt(A_j^2 - 2 dU) when A_j^2 / 2 > dU (the spin flips and the field follows), else it
// is reflected.  After any wall event x_j = 0, so its next zero is pi later: with a
// travel time <= pi each coordinate has at most one event per trajectory, at a time fixed
// by the trajectory's start state.  Events are taken in time order (ties: lower index);
// each decision uses the field left by the earlier ones, so a replica's trajectory is
// serial -- replicas are independent, one warp each.
//
// Warp layout: lane l owns spins i = l + 32 m (m < ceil(N/32) <= 32).  Per warp, shared
// memory holds the trajectory's start state (x, v), the event time and outgoing velocity
// of every spin, the exact integer field I and the spins (for the initial field).  The
// next event is a warp argmin over the lanes' earliest pending spins; a crossing of spin
// j adds 2 s_j J[j][:] to the field (row j of J, read coalesced; J is symmetric).
#include <cuda_runtime.h>

#include <climits>
#include <cstdio>
#include <cstring>

#include "../../include/phia.h"
#include "device_common.cuh"
#include "phia_internal.h"

namespace phia {
namespace {

constexpr int kGWarps = 4;        // replicas (warps) per block
constexpr int kGMaxN = 1024;      // spins per replica: 32 per lane at most

struct GahmcArgs {
    int32_t N, R;
    const int8_t *Jk;
    const int32_t *hk;
    float q;
    float beta0, beta1, travel;
    int64_t K;                    // trajectories
    uint64_t seed;
    uint32_t inst;
    int32_t has_target;
    int64_t target;
    const float *x_in, *v_in;
    float *x_out, *v_out;
    int64_t *best_e, *best_step, *hit_step;
    uint32_t *best_bits;
    int32_t W;
    int64_t *counts;              // [R][2] crossings, reflections (or null)
    int32_t *events;              // [R][cap] (or null)
    int32_t events_cap;
    unsigned long long *replica_iters;
};

// Bytes of per-warp shared memory for N spins.
__host__ __device__ inline size_t gahmc_warp_bytes(int N) { return (size_t)N * (4 * 4 + 4 + 1) + 16; }

__global__ void __launch_bounds__(32 * kGWarps) gahmc_kernel(const GahmcArgs g) {
    extern __shared__ __align__(16) uint8_t gsm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = blockIdx.x * kGWarps + warp;
    if (r >= g.R) return;                       // whole warps only: no block-wide barrier below
    const int N = g.N, M = (N + 31) >> 5;
    uint8_t *base = gsm + (size_t)warp * ((gahmc_warp_bytes(N) + 15) & ~(size_t)15);
    float *xs = reinterpret_cast<float *>(base);
    float *vs = xs + N;
    float *tev = vs + N;
    float *wv = tev + N;
    int32_t *I = reinterpret_cast<int32_t *>(wv + N);
    int8_t *sp = reinterpret_cast<int8_t *>(I + N);

    // Initial state (Philox d = 0 as in PHIA, or given) and its spins.
    uint32_t sbits = 0;                          // bit m: spin lane + 32 m is +1
    for (int m = 0; m < M; ++m) {
        const int i = lane + 32 * m;
        if (i >= N) break;
        float x, v;
        if (g.x_in) {
            x = g.x_in[(size_t)r * N + i];
            v = g.v_in[(size_t)r * N + i];
        } else {
            const U4 o = draw_raw(g.seed, g.inst, (uint32_t)r, (uint32_t)i, 0u);
            x = box_muller(o.x, o.y);
            v = box_muller(o.z, o.w);
        }
        xs[i] = x;
        vs[i] = v;
        const bool plus = x >= 0.0f;
        sp[i] = plus ? 1 : -1;
        sbits |= (uint32_t)plus << m;
    }
    __syncwarp();
    // Field I = J s + h (Eq. 6), from the rows of J (symmetric): I_i = sum_k J[k][i] s_k + h_i.
    int32_t acc[32];
#pragma unroll
    for (int m = 0; m < 32; ++m) acc[m] = 0;
    for (int k = 0; k < N; ++k) {
        const int sk = sp[k];
        const int8_t *row = g.Jk + (size_t)k * N;
#pragma unroll
        for (int m = 0; m < 32; ++m) {
            const int i = lane + 32 * m;
            if (m < M && i < N) acc[m] += (int32_t)row[i] * sk;
        }
    }
    long long twice = 0;                          // sum_i s_i (I_i + h_i)
#pragma unroll
    for (int m = 0; m < 32; ++m) {
        const int i = lane + 32 * m;
        if (m < M && i < N) {
            const int32_t h = g.hk[i];
            I[i] = acc[m] + h;
            twice += (long long)(((sbits >> m) & 1u) ? 1 : -1) * (acc[m] + 2 * h);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) twice += __shfl_xor_sync(0xffffffffu, twice, o);
    long long E = -twice / 2;                     // Eq. 2 via the field
    long long best = E, best_k = 0, hit = (g.has_target && E <= g.target) ? 0 : -1;
    uint32_t bestw = 0;                           // lane m holds word m of the best spins
    for (int m = 0; m < M; ++m) {
        const uint32_t b = __ballot_sync(0xffffffffu, (lane + 32 * m < N) && ((sbits >> m) & 1u));
        if (lane == m) bestw = b;
    }
    long long ncross = 0, nrefl = 0, nev = 0;
    const float T = g.travel;
    for (int64_t k = 0; k < g.K; ++k) {
        const float beta = g.K > 1 ? g.beta0 + (g.beta1 - g.beta0) * ((float)k / (float)(g.K - 1)) : g.beta0;
        const float bq = beta * g.q;
        // Momentum draw d = k (k > 0), event times of this trajectory, pending set.
        uint32_t pend = 0;
        float my_t = INFINITY;
        int my_i = INT_MAX;
        for (int m = 0; m < M; ++m) {
            const int i = lane + 32 * m;
            if (i >= N) break;
            if (k > 0) vs[i] = draw_v(g.seed, g.inst, (uint32_t)r, (uint32_t)i, (uint32_t)k);
            const float x = xs[i], v = vs[i];
            const float t = ((sbits >> m) & 1u) ? atan2f(x, -v) : atan2f(-x, v);
            tev[i] = t;
            if (t < T) {
                pend |= 1u << m;
                if (t < my_t) { my_t = t; my_i = i; }
            }
        }
        // Events in time order.
        for (;;) {
            float bt = my_t;
            int bi = my_i;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float ot = __shfl_xor_sync(0xffffffffu, bt, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ot < bt || (ot == bt && oi < bi)) { bt = ot; bi = oi; }
            }
            if (bi == INT_MAX) break;
            const int owner = bi & 31, mj = bi >> 5;
            int cross = 0, sn = 0, dE = 0;
            if (lane == owner) {
                const float x = xs[bi], v = vs[bi];
                const float A2 = x * x + v * v;                   // squared speed at the wall
                const int s = ((sbits >> mj) & 1u) ? 1 : -1;
                dE = 2 * s * I[bi];                               // flip identity (Eqs. 2, 6)
                const float dU = bq * (float)dE;
                cross = 0.5f * A2 > dU;
                if (cross) {
                    sn = -s;
                    wv[bi] = (float)sn * sqrtf(A2 - 2.0f * dU);
                    sbits ^= 1u << mj;
                } else {
                    wv[bi] = (float)s * sqrtf(A2);
                }
                pend &= ~(1u << mj);
                my_t = INFINITY;
                my_i = INT_MAX;
                for (int m = 0; m < M; ++m)
                    if ((pend >> m) & 1u) {
                        const float t = tev[lane + 32 * m];
                        if (t < my_t) { my_t = t; my_i = lane + 32 * m; }
                    }
            }
            cross = __shfl_sync(0xffffffffu, cross, owner);
            if (g.events && lane == 0 && nev < g.events_cap) g.events[(size_t)r * g.events_cap + nev] = cross ? bi : -(bi + 1);
            ++nev;
            if (!cross) {
                ++nrefl;
                continue;
            }
            ++ncross;
            sn = __shfl_sync(0xffffffffu, sn, owner);
            dE = __shfl_sync(0xffffffffu, dE, owner);
            const int8_t *row = g.Jk + (size_t)bi * N;
            for (int m = 0; m < M; ++m) {
                const int i = lane + 32 * m;
                if (i < N) I[i] += 2 * sn * (int32_t)row[i];
            }
            E += dE;
            if (E < best) {
                best = E;
                best_k = k;
                for (int m = 0; m < M; ++m) {
                    const uint32_t b = __ballot_sync(0xffffffffu, (lane + 32 * m < N) && ((sbits >> m) & 1u));
                    if (lane == m) bestw = b;
                }
            }
            if (g.has_target && hit < 0 && E <= g.target) hit = k;
        }
        // Every coordinate to the end of the trajectory.
        for (int m = 0; m < M; ++m) {
            const int i = lane + 32 * m;
            if (i >= N) break;
            const float t = tev[i];
            if (t < T) {
                float sn_, cs_;
                sincosf(T - t, &sn_, &cs_);
                xs[i] = wv[i] * sn_;
                vs[i] = wv[i] * cs_;
            } else {
                float sn_, cs_;
                sincosf(T, &sn_, &cs_);
                const float x = xs[i], v = vs[i];
                xs[i] = x * cs_ + v * sn_;
                vs[i] = -x * sn_ + v * cs_;
            }
        }
        __syncwarp();
    }
    for (int m = 0; m < M; ++m) {
        const int i = lane + 32 * m;
        if (i >= N) break;
        if (g.x_out) g.x_out[(size_t)r * N + i] = xs[i];
        if (g.v_out) g.v_out[(size_t)r * N + i] = vs[i];
    }
    if (lane < g.W) g.best_bits[(size_t)r * g.W + lane] = bestw;
    if (lane == 0) {
        g.best_e[r] = best;
        g.best_step[r] = best_k;
        g.hit_step[r] = hit;
        if (g.counts) {
            g.counts[2 * (size_t)r] = ncross;
            g.counts[2 * (size_t)r + 1] = nrefl;
        }
        atomicAdd(g.replica_iters, (unsigned long long)g.K);
    }
}

}  // namespace

int gahmc_max_n() { return kGMaxN; }

cudaError_t launch_gahmc(const RunArgs &a, float travel, int64_t K, int64_t *counts, int32_t *events,
                         int32_t events_cap, cudaStream_t st) {
    if (a.N > kGMaxN) return cudaErrorInvalidValue;
    GahmcArgs g;
    memset(&g, 0, sizeof g);
    g.N = a.N; g.R = a.R; g.Jk = a.Jk; g.hk = a.hk; g.q = a.q;
    g.beta0 = a.beta0; g.beta1 = a.beta1; g.travel = travel; g.K = K;
    g.seed = a.seed; g.inst = a.inst; g.has_target = a.has_target; g.target = a.target;
    g.x_in = a.x_in; g.v_in = a.v_in; g.x_out = a.x_out; g.v_out = a.v_out;
    g.best_e = a.best_e; g.best_step = a.best_step; g.hit_step = a.hit_step; g.best_bits = a.best_bits; g.W = a.W;
    g.counts = counts; g.events = events; g.events_cap = events_cap;
    g.replica_iters = a.replica_iters;
    const size_t smem = (size_t)kGWarps * ((gahmc_warp_bytes(a.N) + 15) & ~(size_t)15);
    cudaError_t e = cudaFuncSetAttribute(gahmc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    gahmc_kernel<<<(a.R + kGWarps - 1) / kGWarps, 32 * kGWarps, smem, st>>>(g);
    return cudaGetLastError();
}

}  // namespace phia
