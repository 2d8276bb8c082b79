// k_fp32.cu -- the plain FP32 per-instance PHIA path: FP32 field on CUDA cores, one
// field+update launch and one record launch per iteration.  It is the comparator the
// tensor-core and batched forms are measured against, and it follows the same
// per-iteration semantics (Eq. A7 with the field at the new position, Eqs. 5, 8).
//
// Couplings are held as FP32 J = k q; spins as int8 [R][N] in two ping-pong buffers.
// For the integer / fixed-point couplings of this library every partial sum is an
// exact multiple of q below 2^24 q, so this FP32 field is exact as well.
#include "device_common.cuh"
#include "phia_internal.h"

namespace phia {

namespace {

constexpr int kTile = 32;   // 32 spins x 32 replicas per block
constexpr int kRows = 4;    // replicas per thread (block is 32 x 8 threads)

// Initial state (Philox d = 0 or given), refresh at t0, first position update and sign.
__global__ void fp32_prologue(const RunArgs a, float *x, float *v, int8_t *s) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)a.R * a.N) return;
    const int r = (int)(idx / a.N), i = (int)(idx - (int64_t)r * a.N);
    float xi, vi;
    if (a.x_in) {
        xi = a.x_in[idx];
        vi = a.v_in[idx];
    } else {
        const U4 o = draw_raw(a.seed, a.inst, (uint32_t)r, (uint32_t)i, 0u);
        xi = box_muller(o.x, o.y);
        vi = box_muller(o.z, o.w);
    }
    if (refresh_at(a.t0, a.refresh)) vi = draw_v(a.seed, a.inst, (uint32_t)r, (uint32_t)i, (uint32_t)a.t0);
    xi = xi + a.eps * vi;
    x[idx] = xi;
    v[idx] = vi;
    s[idx] = xi >= 0.0f ? 1 : -1;
}

// One iteration t: I = J s + h (FP32, Eq. 6), energy partials, v update, refresh,
// next position and sign.
__global__ void __launch_bounds__(256) fp32_step(const RunArgs a, int64_t t, float *x, float *v,
                                                 const int8_t *s_cur, int8_t *s_next, int64_t *e_acc) {
    __shared__ float sJ[kTile][kTile + 1];  // sJ[kk][ii] = J[i0+ii][k0+kk]
    __shared__ float sS[kTile][kTile + 1];  // sS[rr][kk] = s[r0+rr][k0+kk]
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    const int i0 = blockIdx.x * kTile, r0 = blockIdx.y * kTile;
    const int N = a.N, R = a.R;
    float acc[kRows] = {0.f, 0.f, 0.f, 0.f};
    for (int k0 = 0; k0 < N; k0 += kTile) {
        for (int e = tid; e < kTile * kTile; e += 256) {
            const int row = e / kTile, kk = e % kTile;
            const int gi = i0 + row, gr = r0 + row, gk = k0 + kk;
            sJ[kk][row] = (gi < N && gk < N) ? a.Jf[(size_t)gi * N + gk] : 0.0f;
            sS[row][kk] = (gr < R && gk < N) ? (float)s_cur[(size_t)gr * N + gk] : 0.0f;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < kTile; ++kk) {
            const float j = sJ[kk][tx];
#pragma unroll
            for (int q = 0; q < kRows; ++q) acc[q] = fmaf(sS[ty * kRows + q][kk], j, acc[q]);
        }
        __syncthreads();
    }
    const int i = i0 + tx;
    const bool live_i = i < N;
    const int32_t hki = live_i ? a.hk[i] : 0;
    const float hf = (float)hki * a.q;
    const float scale = ldexpf(1.0f, a.frac_bits);
    const float beta = beta_at(t, inv_tm1_of(a.T_total), a.beta0, a.beta1);
    const float bgq = beta * a.gamma;   // J and h already carry q here
    const bool more = t + 1 < a.t0 + a.nsteps;
    const bool refresh_next = more && refresh_at(t + 1, a.refresh);
    // With the acceptance test, a trajectory end leaves the refresh and the next position
    // to fp32_metropolis, which first decides whether x goes back to the start.
    const bool advance = more && !(refresh_next && a.accept_test == 1);
#pragma unroll
    for (int q = 0; q < kRows; ++q) {
        const int r = r0 + ty * kRows + q;
        const bool live = live_i && r < R;
        long long part = 0;
        if (live) {
            const size_t idx = (size_t)r * N + i;
            const float I = acc[q] + hf;                        // field in real units
            const long long Ik = llrintf(I * scale);            // units of q
            const int sgn = s_cur[idx];
            part = (long long)sgn * (Ik + hki);
            if (a.field_mode) {
                if (a.field_out) a.field_out[idx] = (int32_t)Ik;
            } else {
                float vi = momentum_update(v[idx], x[idx], I, a.eps, bgq, a.gamma, a.deriv);
                float xi = x[idx];
                if (advance) {
                    if (refresh_next) vi = draw_v(a.seed, a.inst, (uint32_t)r, (uint32_t)i, (uint32_t)(t + 1));
                    xi = xi + a.eps * vi;
                    x[idx] = xi;
                    s_next[idx] = xi >= 0.0f ? 1 : -1;
                }
                v[idx] = vi;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (tx == 0 && r < R) atomicAdd(reinterpret_cast<unsigned long long *>(&e_acc[r]), (unsigned long long)part);
    }
}

// Energy of iteration t per replica, best-state and target records (one warp per replica).
__global__ void fp32_record(const RunArgs a, int64_t t, const int8_t *s_cur, int64_t *e_acc, int64_t *e_last) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= a.R) return;
    const int r = warp;
    const long long E = -e_acc[r] / 2;
    __syncwarp();
    int imp = 0;
    if (lane == 0) {
        e_acc[r] = 0;
        if (e_last) e_last[r] = E;
        const bool frozen = a.stop_at_target && a.hit_step[r] >= 0;
        if (!frozen && E < a.best_e[r]) {
            a.best_e[r] = E;
            a.best_step[r] = t;
            imp = 1;
        }
        if (a.has_target && a.hit_step[r] < 0 && E <= a.target) {
            a.hit_step[r] = t;
            if (a.hit_ns) a.hit_ns[r] = globaltimer_ns();
        }
    }
    imp = __shfl_sync(0xffffffffu, imp, 0);
    if (!imp) return;
    for (int w = 0; w < a.W; ++w) {
        const int i = w * 32 + lane;
        const bool plus = i < a.N && s_cur[(size_t)r * a.N + i] > 0;
        const uint32_t bits = __ballot_sync(0xffffffffu, plus);
        if (lane == 0) a.best_bits[(size_t)r * a.W + w] = bits;
    }
}

// Sum of a float over the block (blockDim.x a multiple of 32, at most 1024); every thread
// gets the result.
__device__ float block_sum(float val, float *scratch) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
    __syncthreads();
    if (lane == 0) scratch[w] = val;
    __syncthreads();
    float s = 0.0f;
    for (int k = 0; k < nw; ++k) s += scratch[k];
    return s;
}

// End of a trajectory before iteration t (t % refresh == 0) with the acceptance test
// (Table 3, state 4): one block per replica.  H = beta E + x.x/2 + v.v/2 (Eq. 4) of the
// end point (E of iteration t-1) against the start point's, both under beta_{t-1}; the
// test uses the uniform of counter (0xFFFFFFFF, r, t, inst).  A rejection puts x back to
// the start.  Then the momentum draw d = t, the new start's x.x and v.v, and the first
// position update and sign of the new trajectory.  The call's first trajectory is kept
// untested (its start energy was never evaluated).
__global__ void fp32_metropolis(const RunArgs a, int64_t t, float *x, float *v, int8_t *s_next, Fp32Metro m) {
    __shared__ float red[32];
    __shared__ int revert;
    const int r = blockIdx.x, N = a.N;
    float xx = 0.0f, vv = 0.0f;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const float xi = x[(size_t)r * N + i], vi = v[(size_t)r * N + i];
        xx += xi * xi;
        vv += vi * vi;
    }
    xx = block_sum(xx, red);
    vv = block_sum(vv, red);
    if (threadIdx.x == 0) {
        const long long e_end = m.e_last[r];
        int rev = 0;
        if (m.has_start[r]) {
            const float beta = beta_at(t - 1, inv_tm1_of(a.T_total), a.beta0, a.beta1);
            const float dH = beta * a.q * (float)(e_end - m.e_start[r]) + 0.5f * (xx - m.xx_start[r]) +
                             0.5f * (vv - m.vv_start[r]);
            const bool acc = metropolis_accept(dH, accept_uniform(a.seed, a.inst, (uint32_t)r, (uint32_t)t));
            a.proposed[r] += 1;
            if (acc) {
                a.accepted[r] += 1;
                m.e_start[r] = e_end;
            } else {
                rev = 1;
            }
        } else {
            m.e_start[r] = e_end;
            m.has_start[r] = 1;
        }
        revert = rev;
    }
    __syncthreads();
    const bool rev = revert != 0;
    float sx = 0.0f, sv = 0.0f;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const size_t idx = (size_t)r * N + i;
        float xi = rev ? m.x_start[idx] : x[idx];
        const float vi = draw_v(a.seed, a.inst, (uint32_t)r, (uint32_t)i, (uint32_t)t);
        m.x_start[idx] = xi;
        sx += xi * xi;
        sv += vi * vi;
        xi = xi + a.eps * vi;
        x[idx] = xi;
        v[idx] = vi;
        s_next[idx] = xi >= 0.0f ? 1 : -1;
    }
    sx = block_sum(sx, red);
    sv = block_sum(sv, red);
    if (threadIdx.x == 0) {
        m.xx_start[r] = sx;
        m.vv_start[r] = sv;
    }
}

// Start of a call with the acceptance test: counts and start flags cleared.
__global__ void fp32_metro_reset(const RunArgs a, Fp32Metro m) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.R) return;
    a.proposed[r] = 0;
    a.accepted[r] = 0;
    m.has_start[r] = 0;
}

// Field-only mode: energies of the given spins, accumulator reset.
__global__ void fp32_field_energy(const RunArgs a, int64_t *e_acc) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.R) return;
    if (a.energy_out) a.energy_out[r] = -e_acc[r] / 2;
    e_acc[r] = 0;
}

__global__ void fp32_epilogue(const RunArgs a, const float *x, const float *v) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)a.R * a.N) return;
    if (a.x_out) {
        a.x_out[idx] = x[idx];
        a.v_out[idx] = v[idx];
    }
}

__global__ void fp32_count(const RunArgs a, int64_t iters) {
    if (threadIdx.x == 0 && blockIdx.x == 0)
        atomicAdd(a.replica_iters, (unsigned long long)((int64_t)a.R * iters));
}

}  // namespace

cudaError_t launch_fp32_run(const RunArgs &a, float *x, float *v, int8_t *s0, int8_t *s1, int64_t *e_acc,
                            const Fp32Metro &metro, cudaStream_t st, int *launches) {
    const int64_t RN = (int64_t)a.R * a.N;
    const int eb = 256;
    const unsigned eg = (unsigned)((RN + eb - 1) / eb);
    const dim3 grid((a.N + kTile - 1) / kTile, (a.R + kTile - 1) / kTile);
    const dim3 block(32, kTile / kRows);
    const unsigned rg = (unsigned)((a.R * 32 + 255) / 256);
    int n = 0;
    if (a.field_mode) {
        // Field only: spins in, field/energy out through the same step kernel.
        RunArgs f = a;
        f.accept_test = 0;
        f.nsteps = 1;
        fp32_step<<<grid, block, 0, st>>>(f, a.t0, x, v, a.spins_in, s1, e_acc);
        fp32_field_energy<<<(a.R + 255) / 256, 256, 0, st>>>(f, e_acc);
        n += 2;
        if (launches) *launches += n;
        return cudaGetLastError();
    }
    fp32_prologue<<<eg, eb, 0, st>>>(a, x, v, s0);
    ++n;
    const bool metro_on = a.accept_test == 1;
    if (metro_on) {
        fp32_metro_reset<<<(a.R + 255) / 256, 256, 0, st>>>(a, metro);
        ++n;
    }
    int8_t *cur = s0, *nxt = s1;
    for (int64_t t = a.t0; t < a.t0 + a.nsteps; ++t) {
        fp32_step<<<grid, block, 0, st>>>(a, t, x, v, cur, nxt, e_acc);
        fp32_record<<<rg, 256, 0, st>>>(a, t, cur, e_acc, metro_on ? metro.e_last : nullptr);
        n += 2;
        if (metro_on && t + 1 < a.t0 + a.nsteps && a.refresh > 0 && (t + 1) % a.refresh == 0) {
            fp32_metropolis<<<a.R, 256, 0, st>>>(a, t + 1, x, v, nxt, metro);
            ++n;
        }
        int8_t *tmp = cur; cur = nxt; nxt = tmp;
    }
    fp32_epilogue<<<eg, eb, 0, st>>>(a, x, v);
    fp32_count<<<1, 32, 0, st>>>(a, a.nsteps);
    n += 2;
    if (launches) *launches += n;
    return cudaGetLastError();
}

}  // namespace phia
