// device_common.cuh -- device helpers shared by every PHIA kernel of this library.
//
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and the Box-Muller transform
// (Box & Muller, 1958) written from their published definitions; the momentum
// update of Eqs. 5, 8 and A7; inline-PTX wrappers for mbarrier, tcgen05 (TMEM
// allocation, MMA, commit, loads, fences) used by the tensor-core kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace phia {

// ------------------------------------------------------------------ Philox

struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                            uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return U4{c0, c1, c2, c3};
}

// 24-bit uniforms: exactly representable in FP32, so host and device agree on them.
__device__ __forceinline__ float u01_open(uint32_t a) { return (float)((a >> 8) + 1u) * 5.9604644775390625e-8f; }
__device__ __forceinline__ float u01_half(uint32_t a) { return (float)(a >> 8) * 5.9604644775390625e-8f; }

// Box-Muller, cosine branch: sqrt(-2 ln u1) cos(2 pi u2).
__device__ __forceinline__ float box_muller(uint32_t a, uint32_t b) {
    return sqrtf(-2.0f * logf(u01_open(a))) * cospif(2.0f * u01_half(b));
}

// Counter (spin j, replica r, draw d, instance), key = seed: words 0-1 -> position
// draw, words 2-3 -> momentum draw.
__device__ __forceinline__ U4 draw_raw(uint64_t seed, uint32_t inst, uint32_t r, uint32_t j, uint32_t d) {
    return philox4x32_10(j, r, d, inst, (uint32_t)seed, (uint32_t)(seed >> 32));
}
__device__ __forceinline__ float draw_x(uint64_t seed, uint32_t inst, uint32_t r, uint32_t j, uint32_t d) {
    U4 o = draw_raw(seed, inst, r, j, d);
    return box_muller(o.x, o.y);
}
__device__ __forceinline__ float draw_v(uint64_t seed, uint32_t inst, uint32_t r, uint32_t j, uint32_t d) {
    U4 o = draw_raw(seed, inst, r, j, d);
    return box_muller(o.z, o.w);
}

// The uniform of the acceptance test (Table 3, state 4) of the trajectory that ends just
// before the momentum draw d = t: counter (0xFFFFFFFF, r, t, inst) -- a spin index no
// instance has -- word 0, on the 24-bit grid of (0, 1].
__device__ __forceinline__ float accept_uniform(uint64_t seed, uint32_t inst, uint32_t r, uint32_t t) {
    return u01_open(draw_raw(seed, inst, r, 0xFFFFFFFFu, t).x);
}

// Metropolis decision on the change dH = H_end - H_start of the Hamiltonian of Eq. 4:
// accept when u <= exp(-dH) (always when dH <= 0).
__device__ __forceinline__ bool metropolis_accept(float dH, float u) { return u <= expf(-dH); }

// ------------------------------------------------------------------ HMC update

// Eq. 8's derivative factor 1 - tanh^2(y) = sech^2(y), evaluated through the identity
// sech^2(y) = 4 e^{-2|y|} / (1 + e^{-2|y|})^2 with one fast exponential (relative error
// a few 1e-6; it goes to 0 without cancellation for large |y|).
// 2^x and 1/x by the hardware approximations (relative error about 2^-22; subnormal
// results flush to 0, which changes nothing here: the term they scale is then far
// below the rounding of v).
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Eq. A7 second line with the gradient of Eq. A8 under Eq. 8:
//   v' = v + eps * (beta gamma (1 - tanh^2(gamma x)) q I - x),   bgq = beta * gamma * q,
// with 1 - tanh^2(y) = sech^2(y) = 4 e / (1 + e)^2, e = exp(-2 |y|) = 2^(-2 log2(e) |y|)
// (e <= 1, so nothing overflows for any y).
// Callers branch on the run's derivative mode once per loop, not per element, so each
// kernel inlines one straight-line form and all kernels produce the same bits.
__device__ __forceinline__ float momentum_exact(float v, float x, float I, float eps, float bgq, float gamma) {
    const float e = ex2_approx(-2.8853900817779268f * fabsf(gamma * x));
    const float d = 1.0f + e;
    return v + eps * ((4.0f * bgq) * (e * rcp_approx(d * d)) * I - x);
}

// The same with the factor replaced by the quadratic stand-in max(0, 1 - (gamma x / 1.5)^2)
// (schedule deriv = 1; after the FPGA's quadratic fit, Sec. 2.2, coefficients chosen here:
// value 1 at 0 and integral 2, as the exact factor).
__device__ __forceinline__ float momentum_quad(float v, float x, float I, float eps, float bgq, float gamma) {
    const float u = __fmul_rn(__fmul_rn(gamma, x), 0.6666667f);   // gamma x / 1.5
    const float f = __fmul_rn(bgq, fmaxf(0.0f, __fmaf_rn(-u, u, 1.0f)));
    return __fmaf_rn(eps, __fmaf_rn(f, I, -x), v);
}

__device__ __forceinline__ float momentum_update(float v, float x, float I, float eps, float bgq, float gamma,
                                                 int deriv) {
    return deriv == 1 ? momentum_quad(v, x, I, eps, bgq, gamma) : momentum_exact(v, x, I, eps, bgq, gamma);
}

// beta_t linear from beta0 (t = 0) to beta1 (t = T-1); inv_tm1 = 1 / (T - 1), 0 if T <= 1.
__device__ __forceinline__ float beta_at(int64_t t, float inv_tm1, float beta0, float beta1) {
    return beta0 + (beta1 - beta0) * ((float)t * inv_tm1);
}
__host__ __device__ inline float inv_tm1_of(int64_t T) { return T > 1 ? 1.0f / (float)(T - 1) : 0.0f; }

__device__ __forceinline__ bool refresh_at(int64_t t, int32_t refresh) {
    return refresh > 0 && t > 0 && (t % refresh) == 0;
}

// ------------------------------------------------------------------ PTX wrappers

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// try_wait that lets the hardware suspend the thread (up to `hint_ns`) until the phase
// completes, so waiting warps do not take issue slots from working ones.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t *bar, uint32_t parity, uint32_t hint_ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase: false when `timeout_ns` of wall time passed.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t timeout_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t_start = globaltimer_ns();
    for (;;) {
        if (mbar_try_wait_sleep(bar, parity, 100000u)) return true;
        if (globaltimer_ns() - t_start > timeout_ns) return false;
    }
}

__device__ __forceinline__ void fence_mbarrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Make this thread's generic-proxy shared-memory writes visible to the async proxy
// (tensor-core operand reads).
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// TMEM allocation by one full warp; the base address is written to *dst_smem.
__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Shared-memory matrix descriptor, K-major, no swizzle: core matrices of 8 rows x 16
// bytes; lbo = byte distance between core matrices adjacent in K, sbo = byte distance
// between adjacent 8-row groups.
__device__ __forceinline__ uint64_t smem_desc_noswizzle(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
    return d;                // base offset 0, lbo mode 0, layout type 0 (no swizzle)
}

// Instruction descriptor: dense, D = F32, A/B formats `fmt` (kind::f16: 1 = BF16;
// kind::f8f6f4: 0 = E4M3), both K-major, N x M tile.
__host__ __device__ constexpr uint32_t make_idesc(uint32_t fmt, uint32_t M, uint32_t N) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_e4m3(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Same MMAs with the A operand read from tensor memory (lane = row of A, its K
// elements packed little-endian into consecutive 32-bit columns).
__device__ __forceinline__ void mma_bf16_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_e4m3_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// 32 lanes x 32 bits, 8 consecutive columns per thread, from registers into TMEM.
__device__ __forceinline__ void tmem_st_x8(uint32_t taddr, const uint32_t (&w)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr),
                 "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7])
                 : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor, K-major, 128-byte swizzle (rows of 128 bytes, 8-row
// atoms of 1024 bytes): stride between 8-row groups = 1024 bytes.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;                 // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024u >> 4) << 32;      // stride byte offset
    d |= (uint64_t)1 << 46;                 // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;                 // 128-byte swizzle
    return d;
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// 2-D tiled TMA load of box (x = inner element coordinate, y = row) into shared memory,
// completing `bytes` on `bar`.
__device__ __forceinline__ void tma_load_2d(void *dst, const void *tmap, uint64_t *bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(tmap), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// The same load multicast to every CTA of the cluster in `mask` (bit = cluster rank):
// the box lands at the same shared-memory offset in each, and each destination's
// mbarrier at the offset of `bar` receives the completed bytes.
__device__ __forceinline__ void tma_load_2d_mc(void *dst, const void *tmap, uint64_t *bar, int x, int y,
                                               uint16_t mask) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster"
        " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(smem_u32(dst)),
        "l"(tmap), "r"(x), "r"(y), "r"(smem_u32(bar)), "h"(mask)
        : "memory");
}

// Arrive once on the mbarrier at the offset of `bar` in every CTA of the cluster in
// `mask` when every tcgen05 operation issued so far by this thread has completed.
__device__ __forceinline__ void mma_commit_mc(uint64_t *bar, uint16_t mask) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
                     smem_u32(bar)),
                 "h"(mask)
                 : "memory");
}

__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Every thread of every CTA of the cluster: arrive, then wait for all (release / acquire).
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Per-thread asynchronous 4-byte copy global -> shared; with `valid` false nothing is
// read and the destination is zero-filled.
__device__ __forceinline__ void cp_async_4(void *dst, const void *src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src),
                 "r"(valid ? 4 : 0)
                 : "memory");
}
// An L2 eviction-priority policy covering every access made under it: its lines are
// evicted after normally cached ones (createpolicy, fraction 1).
__device__ __forceinline__ uint64_t l2_evict_last_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
// 16-byte global store (16-byte aligned) under an L2 policy from createpolicy.
__device__ __forceinline__ void st_global_f4_policy(float *p, float4 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(v.x), "f"(v.y),
                 "f"(v.z), "f"(v.w), "l"(pol)
                 : "memory");
}
// Per-thread asynchronous 16-byte copy global -> shared (both 16-byte aligned), L2 only.
__device__ __forceinline__ void cp_async_16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// Wait until at most `n` of this thread's committed copy groups are still pending.
template <int n>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(n) : "memory");
}

__device__ __forceinline__ void named_barrier_sync(uint32_t id, uint32_t threads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}
// Arrive without waiting; the thread's earlier memory accesses are performed for the
// threads that wait on the barrier.
__device__ __forceinline__ void named_barrier_arrive(uint32_t id, uint32_t threads) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// GPU-scope acquire load and release store of a 32-bit counter in global memory.
__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Order this thread's earlier generic-proxy accesses of global memory before its later
// async-proxy ones (TMA reads of data other CTAs wrote with ordinary stores).
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Bounded wait until the counter at p reaches v (acquire); false after `timeout_ns` of
// wall time or once *abort is set.
__device__ __forceinline__ bool wait_counter_at_least(const uint32_t *p, uint32_t v, uint64_t timeout_ns,
                                                      const volatile int32_t *abort) {
    if (ld_acquire_gpu(p) >= v) return true;
    const uint64_t t_start = globaltimer_ns();
    for (;;) {
        __nanosleep(32);
        if (ld_acquire_gpu(p) >= v) return true;
        if (*abort || globaltimer_ns() - t_start > timeout_ns) return false;
    }
}

// 32 lanes x 32 bits, 16 consecutive columns per thread, then the wait for the load.
__device__ __forceinline__ void tmem_ld_x16_sync(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

// Arrive once on `bar` when every tcgen05 async operation issued so far by this
// thread has completed.
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// 32 lanes x 32 bits, 2 consecutive columns per thread, then the wait for the load.
__device__ __forceinline__ void tmem_ld_x2_sync(uint32_t taddr, float (&v)[2]) {
    uint32_t r0, r1;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(r0), "+r"(r1) : : "memory");
    v[0] = __uint_as_float(r0); v[1] = __uint_as_float(r1);
}

// 32 lanes x 32 bits, 4 consecutive columns per thread, then the wait for the load.
__device__ __forceinline__ void tmem_ld_x4_sync(uint32_t taddr, float (&v)[4]) {
    uint32_t r0, r1, r2, r3;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(r0), "+r"(r1), "+r"(r2), "+r"(r3) : : "memory");
    v[0] = __uint_as_float(r0); v[1] = __uint_as_float(r1); v[2] = __uint_as_float(r2);
    v[3] = __uint_as_float(r3);
}

// 32 lanes x 32 bits, 8 consecutive columns per thread, issued without waiting: the
// registers become valid at the next tmem_ld_wait_x8 on them.
__device__ __forceinline__ void tmem_ld_x8_issue(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}
// Wait for this thread's TMEM loads; the registers of the last issue pass through it.
__device__ __forceinline__ void tmem_ld_wait_x8(uint32_t (&r)[8]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7])
                 :
                 : "memory");
}

// 32 lanes x 32 bits, 8 consecutive columns per thread, followed by the wait for the
// load; the registers pass through the wait so no use can be scheduled before it.
__device__ __forceinline__ void tmem_ld_x8_sync(uint32_t taddr, float (&v)[8]) {
    uint32_t r0, r1, r2, r3, r4, r5, r6, r7;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3), "=r"(r4), "=r"(r5), "=r"(r6), "=r"(r7)
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r0), "+r"(r1), "+r"(r2), "+r"(r3), "+r"(r4), "+r"(r5), "+r"(r6), "+r"(r7)
                 :
                 : "memory");
    v[0] = __uint_as_float(r0); v[1] = __uint_as_float(r1); v[2] = __uint_as_float(r2);
    v[3] = __uint_as_float(r3); v[4] = __uint_as_float(r4); v[5] = __uint_as_float(r5);
    v[6] = __uint_as_float(r6); v[7] = __uint_as_float(r7);
}

}  // namespace phia
