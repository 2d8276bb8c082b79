// k_tc_large.cu -- tensor-core PHIA path for dense instances of any size: one launch per
// iteration (Eq. A7).  The field I = J s + h (Eq. 6) is computed in 128-spin x
// 128-replica output tiles, each followed by the fused update on that tile.
//
// The step kernel is persistent: one CTA per SM walks a static list of output tiles.
// Variants (autotuned): x and v staged through a shared-memory ring (3 operand stages at
// 256-wide tiles) or prefetched into registers (4 stages); and the CTAs of a cluster of
// CL (1, 2 or 4) handling the same replica tile at CL consecutive spin tiles, each
// loading 1/CL of the spin operand and multicasting it to all CL, so each spin tile is
// read from L2 once per cluster instead of once per CTA.
// Operands (K-major, 128-byte swizzle, staged by TMA through an mbarrier ring):
//   A = couplings k re-encoded exactly (e4m3 or bf16), [Mpad][Kpad]
//   B = spins of this iteration in the same encoding, [Rpad][Kpad], one of 4 rotating
//       buffers (iteration t reads buffer t % 4 and writes t+1 % 4; buffers t-1 and t-2
//       stay intact for the lagged best-state copies).
// D = J s accumulates in TMEM (FP32, integer-valued, exact below 2^24): lane = output
// spin, column = replica; two accumulators (three in the overlapped kernel with 160-wide
// tiles), so the MMAs of a CTA's next tile run while the epilogue drains the current one.
// Warp roles: warp 0 issues TMA, warp 1 issues the MMAs (one thread each), warps 2-17 run
// the epilogue: field + h, s (I + h) energy partials, momentum update (Eqs. 5, 8),
// refresh, position update and the sign written as next iteration's B operand.
// x and v live in a replica-interleaved layout [Rpad/4][Mpad][4] (FP32): the 4 replicas
// of one group sit together for each spin, so a thread (one spin, an 8-replica chunk)
// moves its values as two 16-byte vectors, a warp's vector covers 512 contiguous bytes,
// and no padded element lies outside the array.
// They reach the epilogue through a per-thread shared-memory ring filled by cp.async one
// chunk ahead (across tile boundaries); results are stored straight to global memory.
// The prologue converts a caller's [R][N] state in, an export kernel converts it out.
// Records (Table 3, state 5) are lagged so no CTA waits for another: the launch for
// iteration t lets the tiles of output row 0 settle the energies of iteration t-1 (sum
// of every tile's partials) and every tile copy, for replicas that improved at t-2, its
// 128 spins of buffer t-2 into the bit-packed best state.  A final pair of launches
// settles the last two iterations.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cstddef>
#include <cstring>

#include "device_common.cuh"
#include "phia_internal.h"

namespace phia {

namespace {

constexpr int kBM = 128;       // output spins per tile (TMEM lanes)
constexpr int kBKB = 128;      // bytes of K per pipeline stage (one 128-byte swizzle row)
constexpr int kMaxStages = 6;
// Per-iteration kernel variant used when none is requested (see run_variant).
constexpr int kDefaultLargeVariant = 1;
constexpr int kMaxBN = 256;
constexpr int kEpiWarps = 16;  // four per TMEM lane quadrant, each a quarter of the columns
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kThreads = 64 + kEpiThreads;
constexpr int kChunk = 8;                      // replica columns per epilogue step (two x/v groups)
constexpr int kRing = 2;                       // x/v chunks per thread: the current + kRing - 1 ahead
constexpr uint32_t kStageA = kBM * kBKB;
constexpr uint32_t kRingBytes = kRing * kChunk * kEpiThreads * 4;   // per array (x or v)
static_assert(kChunk == 8, "a chunk is two 4-replica groups of the x/v layout");

struct LargeShared {
    uint64_t full[kMaxStages];
    uint64_t empty[kMaxStages];
    uint64_t accf[2];       // accumulator b holds a finished tile
    uint64_t acce[2];       // accumulator b drained by the epilogue warps
    uint64_t drain;         // every MMA issued has completed
    uint32_t tmem_base;
    int32_t timed_out;
    int32_t part[2][4][kMaxBN];   // per lane-quadrant warp sums of s_i (I_i + h_i), by accumulator
    int64_t rec_settled;          // overlapped variant: last iteration the records warp settled
    int64_t rec_copied;           // ... and whose best spins it copied
    uint64_t tiledone[2];         // ... the epilogue warps finished the tile in accumulator b
    alignas(16) uint32_t masks[kEpiWarps][8];  // per epilogue warp: the sign masks of its current
                                               // chunk (written as 16-byte vectors)
    uint64_t accf2, acce2, tiledone2;          // the same three barriers of a third accumulator
                                               // (overlapped kernel with 160-wide tiles)
};
static_assert(offsetof(LargeShared, masks) % 16 == 0, "mask scratch must take 16-byte stores");

// Tile shape: 128 output spins x BN replicas.  BN = 256 halves the coupling-operand
// traffic per output against BN = 128; BN = 128 keeps more tiles when replicas are few;
// the overlapped kernel may also take BN = 224 to even out the tiles per CTA, or BN = 160
// (with three accumulators) to stream fewer operand bytes per tile.
// With the two-chunk x/v ring in shared memory the 256-wide tile has room for three
// operand stages, the 128-wide one for four; with x/v prefetched into registers instead,
// four and six.
template <int BN, bool RING>
struct Tile {
    static constexpr int kStages = RING ? (BN >= 224 ? 3 : 4) : (BN >= 224 ? 4 : 6);
    static constexpr uint32_t kTmemCols = 2 * BN <= 256 ? 256 : 512;   // two accumulators, a power of 2
    static constexpr uint32_t kStageB = BN * kBKB;
    static constexpr int kColsPerWarp = BN / (kEpiWarps / 4);
    static constexpr int kChunksPerTile = kColsPerWarp / kChunk;
    static constexpr size_t kSmemBytes =
        1024 + kStages * (kStageA + kStageB) + (RING ? 2 * kRingBytes : 0) + sizeof(LargeShared);
    static_assert(kStages <= kMaxStages && BN <= kMaxBN, "tile over the shared bookkeeping");
    static_assert(kSmemBytes <= 232448, "shared memory over the per-CTA limit");
    static_assert(kRing - 1 <= kChunksPerTile, "prefetch reaches at most into the next tile");
};

struct LargeArgs {
    RunArgs a;
    uint8_t *S;         // [4][Rpad][Kbytes] spin operand buffers
    int64_t *Epart;     // [2][Rpad] sums of s (I + h) over output tiles, by iteration parity
    int8_t *flags;      // [2][Rpad] improved at an iteration, by parity
    float *X, *V;       // [Rpad/4][Mp][4] state: replica r, spin i at ((r/4) Mp + i) 4 + r%4
    int32_t Kbytes, Rpad, mtiles, ntiles, Mp;
    int32_t rtiles;     // replica tiles (ntiles = mtiles * rtiles)
    IterCtl *ctl;       // iteration of the launch and range of the run
    uint32_t *ready;    // overlapped variant: [rtiles] output tiles finished per replica tile,
                        // then [rtiles] iterations settled per replica tile (null otherwise)
    uint32_t *sbits;    // overlapped variant: [4][Mp/32][Rpad] packed spins by iteration slot,
                        // word-major (a word's replicas are consecutive)
    int64_t f0, f1;     // overlapped variant: this launch's iterations [f0, f1) of the call's
    int32_t xv_keep;    // overlapped variant: x and v stores ask L2 to keep their lines
                        // (evict_last), set when the state exceeds half of L2
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

// Bit k set when spin k of the 32 encoded spins at p (16-byte aligned) is +1.
template <int OP>
__device__ __forceinline__ uint32_t plus_bits32(const uint8_t *p) {
    const uint4 *q = reinterpret_cast<const uint4 *>(p);
    uint32_t bits = 0;
    if constexpr (OP == kOpE4M3) {
        // One byte per spin, sign in bit 7: gather the four inverted sign bits of a word
        // into bits 24..27 of one product (the other partial products land below bit 20).
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint4 w = q[h];
            const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t b = ((~ws[k] & 0x80808080u) >> 7) * 0x01020408u;
                bits |= ((b >> 24) & 0xFu) << (16 * h + 4 * k);
            }
        }
    } else {
        // Two bytes per spin, sign in bit 15 of each half-word.
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const uint4 w = q[h];
            const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t nw = ~ws[k];
                bits |= (((nw >> 15) & 1u) | ((nw >> 30) & 2u)) << (8 * h + 2 * k);
            }
        }
    }
    return bits;
}

// The encoded spins of 8 consecutive spins (e4m3: 8 bytes) or 4 (bf16: 8 bytes) taken
// from bits [b0, b0 + 8 / ESZ) of a sign mask (bit set: +1), as a 64-bit word.
// e4m3 +1 / -1 = 0x38 / 0xB8, bf16 +1 / -1 = 0x3F80 / 0xBF80: a set bit clears the sign.
template <int OP>
__device__ __forceinline__ uint64_t spin_word(uint32_t mask, int b0) {
    if constexpr (OP == kOpE4M3) {
        const uint32_t lo = (mask >> b0) & 0xFu, hi = (mask >> (b0 + 4)) & 0xFu;
        // bit k of a 4-bit group to bit 8k (the four shifted copies never overlap)
        const uint32_t slo = (lo * 0x00204081u) & 0x01010101u, shi = (hi * 0x00204081u) & 0x01010101u;
        return ((uint64_t)(0xB8B8B8B8u ^ (shi << 7)) << 32) | (uint64_t)(0xB8B8B8B8u ^ (slo << 7));
    } else {
        const uint32_t b = (mask >> b0) & 0xFu;
        const uint32_t slo = (b & 1u) | ((b & 2u) << 15), shi = ((b >> 2) & 1u) | ((b & 8u) << 13);
        return ((uint64_t)(0xBF80BF80u ^ (shi << 15)) << 32) | (uint64_t)(0xBF80BF80u ^ (slo << 15));
    }
}

// One epilogue chunk of the accumulator: 32 lanes x kChunk consecutive columns.
template <int C>
__device__ __forceinline__ void tmem_ld_chunk(uint32_t taddr, float (&v)[C]) {
    static_assert(C == 4 || C == 8 || C == 16, "unsupported chunk");
    if constexpr (C == 16) tmem_ld_x16_sync(taddr, v);
    else if constexpr (C == 8) tmem_ld_x8_sync(taddr, v);
    else tmem_ld_x4_sync(taddr, v);
}

// Epilogue arithmetic of one chunk (one output spin i, kChunk replica columns): the field
// I = J s + h from the accumulator (Eq. 6; exact integers in FP32), the energy terms
// s (I + h) of the live columns (Eq. 2 through Eq. 6; 0 elsewhere) and the momentum
// update at the new position (Eqs. 5, 8, A7).  The energy terms are integers from the
// exact accumulator; the momentum takes I as acc + h in FP32, the same rounding of the
// exact integer as converting it (both operands are exact).  (A second, unmasked copy of
// this code for full chunks was measured slower: 26.2 against 24.3 us per iteration at
// N = 2000.)
__device__ __forceinline__ void chunk_field_momentum(const float (&acc)[kChunk], const float (&xs)[kChunk],
                                                     float (&vs)[kChunk], int32_t hki, float hkf, int nlive,
                                                     int deriv, float eps, float bgq, float gamma,
                                                     int32_t (&p)[kChunk]) {
    float If[kChunk];
#pragma unroll
    for (int j = 0; j < kChunk; ++j) {
        const int32_t e = __float2int_rn(acc[j]) + 2 * hki;    // I + h, exact
        p[j] = j < nlive ? (xs[j] >= 0.0f ? e : -e) : 0;
        If[j] = acc[j] + hkf;
    }
    if (deriv == 1) {
#pragma unroll
        for (int j = 0; j < kChunk; ++j) vs[j] = momentum_quad(vs[j], xs[j], If[j], eps, bgq, gamma);
    } else {
#pragma unroll
        for (int j = 0; j < kChunk; ++j) vs[j] = momentum_exact(vs[j], xs[j], If[j], eps, bgq, gamma);
    }
}

// Next iteration's spins of one chunk into the B operand: one sign mask per replica
// column over the warp's 32 spins (rows row0 .. row0 + 31); lane l writes replica l / 4,
// spins 8 (l % 4) .. (e4m3: 8 bytes) or 4 (l % 4) .. (bf16: 8 bytes) of them.  `col` is
// the chunk's first replica row, `live` its live columns.  Spins past N land in K
// padding, which meets zero couplings; words wholly past N stay out (for bf16 they could
// pass the row's end).  The eight masks reach their lanes through `scratch` (8 words of
// this warp's shared memory).  With `bits` (the overlapped variant) lane j < live also
// stores column j's mask, the packed spins of rows row0 .. row0 + 31, at bits[j]
// (consecutive replicas: one sector).
template <int OP>
__device__ __forceinline__ void chunk_store_spins(const float (&xn)[kChunk], int lane, int live, uint8_t *col,
                                                  int Kbytes, int row0, int N, uint32_t *scratch,
                                                  uint32_t *bits = nullptr) {
    constexpr int ESZ = OP == kOpE4M3 ? 1 : 2;
    uint32_t m[kChunk];
#pragma unroll
    for (int j = 0; j < kChunk; ++j) m[j] = __ballot_sync(0xffffffffu, xn[j] >= 0.0f);
    __syncwarp();                      // the previous chunk's reads of scratch are done
    if (lane == 0) {
        reinterpret_cast<uint4 *>(scratch)[0] = make_uint4(m[0], m[1], m[2], m[3]);
        reinterpret_cast<uint4 *>(scratch)[1] = make_uint4(m[4], m[5], m[6], m[7]);
    }
    __syncwarp();
    const uint32_t msk = scratch[lane >> 2];
    if (bits && lane < live && lane < kChunk && row0 < N) bits[lane] = scratch[lane];
    const int jr = lane >> 2, part = lane & 3;
    if (jr < live) {
        constexpr int kPer = OP == kOpE4M3 ? 8 : 4;   // spins per 8-byte store
#pragma unroll
        for (int h = 0; h < 8 / kPer; ++h) {
            const int sp = part * kPer + h * 4 * kPer;     // first spin (of the warp's 32)
            if (row0 + sp >= N) continue;
            uint8_t *dst = col + (size_t)jr * Kbytes + (size_t)sp * ESZ;
            *reinterpret_cast<uint64_t *>(dst) = spin_word<OP>(msk, sp);
        }
    }
}

// Record step for replica r at iteration tt (Table 3, state 5): E from the sum the
// output tiles accumulated, best/target records, improved flag; the sum slot is cleared
// for iteration tt + 2.
__device__ __forceinline__ void settle_replica(const LargeArgs &L, int r, int64_t tt, int flag_mask = 1) {
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
    if (a.has_target && a.hit_step[r] < 0 && E <= a.target) {
        a.hit_step[r] = tt;
        if (a.hit_ns) a.hit_ns[r] = globaltimer_ns();
    }
    L.flags[(size_t)(tt & flag_mask) * L.Rpad + r] = (int8_t)imp;
}

// The record step of settle_replica for the replicas r0 + 32 k (k < K) of one lane, with
// every load issued before any store so that the K replicas' round trips overlap.
template <int K>
__device__ __forceinline__ void settle_lane(const LargeArgs &L, int r0, int64_t tt, int flag_mask) {
    const RunArgs &a = L.a;
    unsigned long long *slots = reinterpret_cast<unsigned long long *>(L.Epart) + (size_t)(tt & 1) * L.Rpad;
    long long tw[K], be[K], hs[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int r = r0 + 32 * k;
        const bool live = r < a.R;
        tw[k] = live ? (long long)slots[r] : 0;
        be[k] = live ? (long long)a.best_e[r] : 0;
        hs[k] = live ? (long long)a.hit_step[r] : 0;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int r = r0 + 32 * k;
        if (r >= a.R) continue;
        slots[r] = 0ull;
        const long long E = -tw[k] / 2;
        int imp = 0;
        if (!(a.stop_at_target && hs[k] >= 0) && E < be[k]) {
            a.best_e[r] = E;
            a.best_step[r] = tt;
            imp = 1;
        }
        if (a.has_target && hs[k] < 0 && E <= a.target) {
            a.hit_step[r] = tt;
            if (a.hit_ns) a.hit_ns[r] = globaltimer_ns();
        }
        L.flags[(size_t)(tt & flag_mask) * L.Rpad + r] = (int8_t)imp;
    }
}

// Best spins of iteration tt, output rows m*128 .. m*128+127, for the replicas r0 + 32 k
// (k < K) of one lane that improved at tt (flags slot tt & 3), from the packed spins the
// epilogue wrote (slot tt & 3, word-major): flags first, then per improved replica its
// four words (each load coalesced across the warp's consecutive replicas).
template <int K>
__device__ __forceinline__ void copy_best_lane(const LargeArgs &L, int r0, int m, int64_t tt) {
    const RunArgs &a = L.a;
    const int8_t *F = L.flags + (size_t)(tt & 3) * L.Rpad;
    const int Wp = L.Mp / 32;
    const uint32_t *B = L.sbits + (size_t)(tt & 3) * Wp * L.Rpad;
    int8_t f[K];
#pragma unroll
    for (int k = 0; k < K; ++k) f[k] = r0 + 32 * k < a.R ? F[r0 + 32 * k] : (int8_t)0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if (!f[k]) continue;
        const int r = r0 + 32 * k;
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) w[q] = B[(size_t)(m * 4 + q) * L.Rpad + r];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i0 = m * kBM + q * 32;
            if (i0 >= a.N) break;
            const uint32_t valid = a.N - i0 >= 32 ? 0xffffffffu : ((1u << (a.N - i0)) - 1u);
            a.best_bits[(size_t)r * a.W + (i0 >> 5)] = w[q] & valid;
        }
    }
}

template <int OP, int BN, int CL, bool RING>
__global__ void __launch_bounds__(kThreads, 1)
    tc_large_step(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                  const LargeArgs L) {
    constexpr int ESZ = OP == kOpE4M3 ? 1 : 2;
    constexpr uint32_t IDESC = make_idesc(OP == kOpE4M3 ? 0u : 1u, kBM, BN);
    constexpr int kStages = Tile<BN, RING>::kStages;
    constexpr uint32_t kStageB = Tile<BN, RING>::kStageB;
    constexpr int kColsPerWarp = Tile<BN, RING>::kColsPerWarp;
    constexpr int kChunksPerTile = Tile<BN, RING>::kChunksPerTile;
    constexpr uint16_t kMask = (uint16_t)((1u << CL) - 1u);
    static_assert(CL == 1 || CL == 2 || CL == 4, "cluster of 1, 2 or 4 CTAs");
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sA = smem;
    uint8_t *sB = smem + kStages * kStageA;
    float *ring_x = reinterpret_cast<float *>(sB + kStages * kStageB);
    float *ring_v = ring_x + kRingBytes / 4;
    LargeShared *sh = reinterpret_cast<LargeShared *>(RING ? reinterpret_cast<uint8_t *>(ring_v + kRingBytes / 4)
                                                           : reinterpret_cast<uint8_t *>(ring_x));
    volatile int32_t *tout = &sh->timed_out;

    const RunArgs &a = L.a;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // Cluster tiles: CL consecutive spin tiles of one replica tile; CTA `crank` of the
    // cluster takes the crank-th.  With CL = 1 a cluster tile is one output tile.
    const int crank = CL > 1 ? (int)cluster_ctarank() : 0;
    const int Gc = (int)gridDim.x / CL;             // clusters (the grid is a multiple of CL)
    const int cid = (int)blockIdx.x / CL;
    const int mgroups = L.mtiles / CL;
    const int ctiles = mgroups * L.rtiles;
    const int my_tiles = cid < ctiles ? (ctiles - 1 - cid) / Gc + 1 : 0;
    auto tile_m = [&](int lt) { return ((cid + lt * Gc) % mgroups) * CL + crank; };
    auto tile_n = [&](int lt) { return (cid + lt * Gc) / mgroups; };
    const int KB = L.Kbytes / kBKB;
    const int N = a.N, R = a.R;
    const uint64_t kWaitNs = a.wait_ns > 0 ? (uint64_t)a.wait_ns : kWaitTimeoutNs;

    if (warp == 0) {
        tmem_alloc(&sh->tmem_base, Tile<BN, RING>::kTmemCols);
        tmem_relinquish();
    }
    if (tid == 32) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&sh->full[s], 1);
            mbar_init(&sh->empty[s], CL);   // freed by the MMAs of every CTA of the cluster
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&sh->accf[b], 1);
            mbar_init(&sh->acce[b], kEpiWarps);
        }
        mbar_init(&sh->drain, 1);
        sh->timed_out = 0;
        fence_mbarrier_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if constexpr (CL > 1) cluster_sync_all();   // every CTA's barriers exist before any multicast
    const uint32_t tmem = sh->tmem_base;
    const int64_t t = L.ctl->t, t_first = L.ctl->t_first, t_end = L.ctl->t_end;

    if (warp == 0) {
        // TMA producer: the k-blocks of every tile of this CTA through one ring.  With
        // stall_producer (a testing aid) it issues nothing, so every wait below on a full
        // stage or a finished accumulator runs out after kWaitNs and the launch reports it.
        if (lane == 0 && !a.stall_producer) {
            int64_t kg = 0;
            bool ok = true;
            for (int lt = 0; lt < my_tiles && ok; ++lt) {
                const int m = tile_m(lt), n = tile_n(lt);
                const int ybuf = (int)(t & 3) * L.Rpad + n * BN;
                for (int kb = 0; kb < KB; ++kb, ++kg) {
                    const int s = (int)(kg % kStages);
                    if (kg >= kStages &&
                        (*tout || !mbar_wait_bounded(&sh->empty[s], (uint32_t)((kg / kStages) - 1) & 1u, kWaitNs))) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&sh->full[s], kStageA + kStageB);
                    tma_load_2d(sA + s * kStageA, &tmA, &sh->full[s], kb * (kBKB / ESZ), m * kBM);
                    if constexpr (CL == 1) {
                        tma_load_2d(sB + s * kStageB, &tmB, &sh->full[s], kb * (kBKB / ESZ), ybuf);
                    } else {
                        // this CTA's 1/CL of the spin tile, to the same place in every CTA
                        tma_load_2d_mc(sB + s * kStageB + crank * (BN / CL) * kBKB, &tmB, &sh->full[s],
                                       kb * (kBKB / ESZ), ybuf + crank * (BN / CL), kMask);
                    }
                }
            }
            if (!ok) *tout = 1;
            // Copies still in flight (only after a timeout) land before the CTA exits.
            for (int64_t k = kg > kStages ? kg - kStages : 0; k < kg; ++k)
                mbar_wait_bounded(&sh->full[k % kStages], (uint32_t)(k / kStages) & 1u, kWaitNs);
        }
    } else if (warp == 1) {
        // MMA issuer: 4 K-steps of 32 bytes per stage, accumulators alternating per tile.
        if (lane == 0) {
            int64_t kg = 0;
            bool ok = true;
            for (int lt = 0; lt < my_tiles && ok; ++lt) {
                const int b = lt & 1;
                if (lt >= 2 && (*tout || !mbar_wait_bounded(&sh->acce[b], (uint32_t)((lt >> 1) - 1) & 1u, kWaitNs))) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t dt = tmem + (uint32_t)(b * BN);
                for (int kb = 0; kb < KB; ++kb, ++kg) {
                    const int s = (int)(kg % kStages);
                    if (*tout || !mbar_wait_bounded(&sh->full[s], (uint32_t)(kg / kStages) & 1u, kWaitNs)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t ad = smem_desc_sw128(smem_u32(sA + s * kStageA));
                    const uint64_t bd = smem_desc_sw128(smem_u32(sB + s * kStageB));
#pragma unroll
                    for (int k = 0; k < kBKB / 32; ++k) {
                        if constexpr (OP == kOpE4M3) mma_e4m3(dt, ad + 2 * k, bd + 2 * k, IDESC, (kb | k) != 0);
                        else mma_bf16(dt, ad + 2 * k, bd + 2 * k, IDESC, (kb | k) != 0);
                    }
                    if constexpr (CL == 1) mma_commit(&sh->empty[s]);
                    else mma_commit_mc(&sh->empty[s], kMask);   // stage s free in every CTA of the cluster
                }
                if (ok) mma_commit(&sh->accf[b]);
            }
            if (!ok) *tout = 1;
            // Every MMA issued has completed before the accumulators are released.
            mma_commit(&sh->drain);
            mbar_wait_bounded(&sh->drain, 0, kWaitNs);
        }
    } else {
        // Epilogue warps: warp w reads TMEM lane quadrant w % 4 and column group (w - 2) / 4;
        // thread et owns spin i of its quadrant and 32 replica columns (4 chunks) per tile.
        const int ew = warp - 2;
        const int q4 = warp & 3;
        const int cg = ew >> 2;
        const int et = ew * 32 + lane;
        const int Mp = L.Mp;
        // Ring slot s holds a chunk's x (and v) as two 16-byte halves per thread at
        // float4 index (2 s + h) * kEpiThreads + et.
        float4 *rx4 = reinterpret_cast<float4 *>(ring_x) + et;
        float4 *rv4 = reinterpret_cast<float4 *>(ring_v) + et;
        // Float offset of this thread's first 4 values of chunk c of tile (m, n); the
        // other 4 (the next replica group) follow at + 4 Mp.
        const size_t grp_stride = (size_t)Mp * 4;
        auto xv_offset = [&](int m_, int n_, int c_) -> size_t {
            const int grp = (n_ * BN + cg * kColsPerWarp + c_ * kChunk) >> 2;
            return ((size_t)grp * Mp + (m_ * kBM + q4 * 32 + lane)) * 4;
        };
        auto issue = [&](size_t off, int slot) {
            cp_async_16(rx4 + (2 * slot) * kEpiThreads, L.X + off);
            cp_async_16(rx4 + (2 * slot + 1) * kEpiThreads, L.X + off + grp_stride);
            cp_async_16(rv4 + (2 * slot) * kEpiThreads, L.V + off);
            cp_async_16(rv4 + (2 * slot + 1) * kEpiThreads, L.V + off + grp_stride);
        };
        // Without the ring: the next chunk's x and v wait in registers (loaded one chunk ahead).
        float4 nx0 = make_float4(0.f, 0.f, 0.f, 0.f), nx1 = nx0, nv0 = nx0, nv1 = nx0;
        auto fetch = [&](size_t off) {
            nx0 = __ldcg(reinterpret_cast<const float4 *>(L.X + off));
            nx1 = __ldcg(reinterpret_cast<const float4 *>(L.X + off + grp_stride));
            nv0 = __ldcg(reinterpret_cast<const float4 *>(L.V + off));
            nv1 = __ldcg(reinterpret_cast<const float4 *>(L.V + off + grp_stride));
        };
        int m_cur = tile_m(0), n_cur = tile_n(0);
        if (!a.field_mode && my_tiles > 0) {
            if constexpr (RING) {
                for (int c0 = 0; c0 < kRing - 1; ++c0) {
                    issue(xv_offset(m_cur, n_cur, c0), c0);
                    cp_async_commit();
                }
            } else {
                fetch(xv_offset(m_cur, n_cur, 0));
            }
        }
        const float bgq = beta_at(t, inv_tm1_of(a.T_total), a.beta0, a.beta1) * (a.gamma * a.q);
        const float eps = a.eps, gamma = a.gamma;
        const bool more = t + 1 < t_end;
        const bool refresh_next = more && refresh_at(t + 1, a.refresh);
        uint8_t *Sn = L.S + (size_t)((t + 1) & 3) * L.Rpad * L.Kbytes;
        // Records of earlier iterations for every tile of this CTA, done while the first
        // tile's MMAs run (they read nothing this launch writes):
        // (a) records of iteration t-1 for each replica tile (output row 0 only);
        // (b) best spins of iteration t-2 for the replicas that improved then: lane l packs
        //     the 32 spins of this warp's quadrant for replica rb + l.
        for (int lt = 0; lt < my_tiles; ++lt) {
            const int m = tile_m(lt), n = tile_n(lt);
            if (m == 0 && t - 1 >= t_first && et < BN) {
                const int r = n * BN + et;
                if (r < R) settle_replica(L, r, t - 1);
            }
            if (t - 2 >= t_first) {
                const int rb = n * BN + cg * kColsPerWarp;
                const int8_t *F = L.flags + (size_t)((t - 2) & 1) * L.Rpad;
                const uint8_t *Sb = L.S + (size_t)((t - 2) & 3) * L.Rpad * L.Kbytes;
                const int i0 = m * kBM + q4 * 32;
                if (i0 < N) {
                    const uint32_t valid = N - i0 >= 32 ? 0xffffffffu : ((1u << (N - i0)) - 1u);
#pragma unroll
                    for (int u = 0; u < kColsPerWarp / 32; ++u) {
                        const int r = rb + u * 32 + lane;
                        if (r < R && F[r])
                            a.best_bits[(size_t)r * a.W + (i0 >> 5)] =
                                plus_bits32<OP>(Sb + (size_t)r * L.Kbytes + (size_t)i0 * ESZ) & valid;
                    }
                }
            }
        }
        int slot = 0;                                   // ring slot of the current chunk
        for (int lt = 0; lt < my_tiles; ++lt) {
            const int m = m_cur, n = n_cur;
            const int b = lt & 1;
            const bool has_nxt = lt + 1 < my_tiles;
            const int m_nxt = tile_m(lt + 1), n_nxt = tile_n(lt + 1);
            const int i = m * kBM + q4 * 32 + lane;
            const bool live_i = i < N;
            // (c) the field of this iteration and the update.
            const int32_t hki = live_i ? a.hk[i] : 0;
            const float hkf = (float)hki;
            const int rc0 = n * BN + cg * kColsPerWarp;          // first replica of this warp's columns
            const int ncol = max(0, min(kColsPerWarp, R - rc0));   // live replica columns of this warp
            // the warp's first spin of this tile, in row rc0 of the next spin buffer
            uint8_t *swarp = Sn + (size_t)rc0 * L.Kbytes + (size_t)(m * kBM + q4 * 32) * ESZ;
            // Warp-uniform, as the TMEM loads below are warp-collective.
            const bool ok = __all_sync(0xffffffffu, !*tout && mbar_wait_bounded(&sh->accf[b], (uint32_t)(lt >> 1) & 1u,
                                                                               kWaitNs));
            if (!ok) *tout = 1;
            tc_fence_after();
            const uint32_t tbase = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(b * BN + cg * kColsPerWarp);
            uint32_t accn[kChunk];                         // accumulators of the next chunk to compute
            if (ok && !a.field_mode) {
                tmem_ld_x8_issue(tbase, accn);
                tmem_ld_wait_x8(accn);
            }
#pragma unroll 1
            for (int c = 0; c < kChunksPerTile; ++c) {
                const int col0 = c * kChunk;               // first column of the chunk in this warp's group
                if (a.field_mode) {
                    float acc[kChunk];
                    if (ok) tmem_ld_chunk(tbase + col0, acc);
#pragma unroll
                    for (int j = 0; j < kChunk; ++j) {
                        const int r = rc0 + col0 + j;
                        int32_t part = 0;
                        if (live_i && r < R && ok) {
                            const size_t idx = (size_t)r * N + i;
                            const int32_t Ik = __float2int_rn(acc[j]) + hki;
                            part = (a.spins_in[idx] > 0 ? 1 : -1) * (Ik + hki);
                            if (a.field_out) a.field_out[idx] = Ik;
                        }
                        part = __reduce_add_sync(0xffffffffu, part);
                        if (lane == 0) sh->part[b][q4][cg * kColsPerWarp + col0 + j] = part;
                    }
                    continue;
                }
                float4 x0, x1, v0, v1;
                if constexpr (RING) {
                    // Keep kRing - 1 chunks in flight: this tile's later chunks, then the next tile's.
                    {
                        const int ca = c + kRing - 1;
                        const int sa = slot + kRing - 1 >= kRing ? slot - 1 : slot + kRing - 1;
                        if (ca < kChunksPerTile) issue(xv_offset(m, n, ca), sa);
                        else if (has_nxt) issue(xv_offset(m_nxt, n_nxt, ca - kChunksPerTile), sa);
                        cp_async_commit();
                    }
                    cp_async_wait<kRing - 1>();
                    const int sc = slot;
                    slot = slot + 1 == kRing ? 0 : slot + 1;
                    if (!ok) continue;
                    x0 = rx4[(2 * sc) * kEpiThreads]; x1 = rx4[(2 * sc + 1) * kEpiThreads];
                    v0 = rv4[(2 * sc) * kEpiThreads]; v1 = rv4[(2 * sc + 1) * kEpiThreads];
                } else {
                    x0 = nx0; x1 = nx1; v0 = nv0; v1 = nv1;
                    if (c + 1 < kChunksPerTile) fetch(xv_offset(m, n, c + 1));
                    else if (has_nxt) fetch(xv_offset(m_nxt, n_nxt, 0));
                    if (!ok) continue;
                }
                // This chunk's accumulators were loaded one chunk ahead; the next chunk's load
                // goes out now and completes while this one is computed.
                float acc[kChunk];
#pragma unroll
                for (int j = 0; j < kChunk; ++j) acc[j] = __uint_as_float(accn[j]);
                const bool ld_next = c + 1 < kChunksPerTile;
                if (ld_next) tmem_ld_x8_issue(tbase + col0 + kChunk, accn);
                const float xs[kChunk] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
                float vs[kChunk] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
                const int nlive = live_i ? ncol - col0 : 0;   // live columns of this chunk for this thread
                int32_t p[kChunk];
                chunk_field_momentum(acc, xs, vs, hki, hkf, nlive, a.deriv, eps, bgq, gamma, p);
#pragma unroll
                for (int j = 0; j < kChunk; ++j) {
                    const int32_t ps = __reduce_add_sync(0xffffffffu, p[j]);
                    if (lane == j) sh->part[b][q4][cg * kColsPerWarp + col0 + j] = ps;
                }
                if (refresh_next) {
#pragma unroll
                    for (int j = 0; j < kChunk; ++j)
                        vs[j] = draw_v(a.seed, a.inst, (uint32_t)(rc0 + col0 + j), (uint32_t)i, (uint32_t)(t + 1));
                }
                // Padding elements (i >= N or replica >= R) are stored too: they stay inside
                // the array and no record reads them.
                const size_t off = xv_offset(m, n, c);
                if (more) {
                    float xn[kChunk];
#pragma unroll
                    for (int j = 0; j < kChunk; ++j) xn[j] = xs[j] + eps * vs[j];
                    *reinterpret_cast<float4 *>(L.X + off) = make_float4(xn[0], xn[1], xn[2], xn[3]);
                    *reinterpret_cast<float4 *>(L.X + off + grp_stride) = make_float4(xn[4], xn[5], xn[6], xn[7]);
                    chunk_store_spins<OP>(xn, lane, ncol - col0, swarp + (size_t)col0 * L.Kbytes, L.Kbytes,
                                          m * kBM + q4 * 32, N, sh->masks[ew]);
                }
                *reinterpret_cast<float4 *>(L.V + off) = make_float4(vs[0], vs[1], vs[2], vs[3]);
                *reinterpret_cast<float4 *>(L.V + off + grp_stride) = make_float4(vs[4], vs[5], vs[6], vs[7]);
                if (ld_next) tmem_ld_wait_x8(accn);
            }
            // Accumulator b is free for the tile after next.
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&sh->acce[b]);
            named_barrier_sync(1, kEpiThreads);
            if (et < BN) {
                const int r = n * BN + et;
                const long long s4 =
                    (long long)sh->part[b][0][et] + sh->part[b][1][et] + sh->part[b][2][et] + sh->part[b][3][et];
                if (ok) atomicAdd(reinterpret_cast<unsigned long long *>(L.Epart) + (size_t)(t & 1) * L.Rpad + r,
                                  (unsigned long long)s4);
            }
            m_cur = m_nxt;
            n_cur = n_nxt;
        }
        if constexpr (RING) cp_async_wait<0>();
    }
    tc_fence_before();
    __syncthreads();
    // No CTA of a cluster leaves while another may still multicast into it or arrive on
    // its barriers.
    if constexpr (CL > 1) cluster_sync_all();
    if (tid == 0) {
        if (sh->timed_out) atomicExch(a.err, 1);
        iter_ctl_finish(L.ctl);
    }
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, Tile<BN, RING>::kTmemCols);
    }
}

// ---------------------------------------------------------------- overlapped variant
// All iterations of a run in one cooperative launch (variant 7).  Every CTA keeps the same
// output tiles for the whole run, so the state it updates never moves to another CTA;
// what crosses CTAs are the spins of a replica tile (the B operand of every output tile
// of that replica tile) and its energy sums.  Instead of a grid-wide step boundary, a
// per-replica-tile counter ready[n] counts the output tiles of replica tile n that have
// finished an iteration: the TMA producer of an output tile of n starts iteration t once
// ready[n] = mtiles (t - t0), so a replica tile whose spins are complete runs ahead
// while other tiles still finish the previous iteration, and the MMAs of a CTA's next
// tile overlap the epilogue of its current one across iteration boundaries too.
//
// Two more warps do the bookkeeping off the epilogue's path.  A signal warp waits until
// the epilogue warps finished a tile (an mbarrier), makes their stores visible to the GPU
// and counts the tile in ready[n].  A records warp settles the energies of iteration t of
// the replica tiles whose first output tile (m = 0) this CTA owns (after ready[n] counts
// iteration t complete), then publishes settled[n] = t - t0 + 1; every CTA copies the
// best spins of iteration t of its own tiles once settled[n] says the improved flags of
// t exist.  Reuse of the rotating buffers is guarded: the m = 0 tile is counted for
// iteration t only after its records warp settled t - 1 (the energy sums of t - 1 share a
// slot with t + 1), and a tile writes the spins of iteration t + 1 into the buffer of
// t - 3 only after its records warp copied t - 3; the improved flags rotate over four
// slots.  Every wait is bounded; a wait that runs out sets the run's error flag and the
// CTA winds down.
template <int OP, int BN, int CL, int NACC>
__global__ void __launch_bounds__(kThreads + 64, 1)
    tc_flow_run(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                const LargeArgs L) {
    constexpr int ESZ = OP == kOpE4M3 ? 1 : 2;
    constexpr uint32_t IDESC = make_idesc(OP == kOpE4M3 ? 0u : 1u, kBM, BN);
    constexpr int kStages = Tile<BN, true>::kStages;
    constexpr uint32_t kStageB = Tile<BN, true>::kStageB;
    constexpr int kColsPerWarp = Tile<BN, true>::kColsPerWarp;
    constexpr int kChunksPerTile = Tile<BN, true>::kChunksPerTile;
    constexpr uint16_t kMask = (uint16_t)((1u << CL) - 1u);
    static_assert(CL == 1 || CL == 2 || CL == 4, "cluster of 1, 2 or 4 CTAs");
    static_assert((NACC == 2 || NACC == 3) && NACC * BN <= (int)Tile<BN, true>::kTmemCols,
                  "accumulators beyond the tensor memory allocated");
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sA = smem;
    uint8_t *sB = smem + kStages * kStageA;
    float *ring_x = reinterpret_cast<float *>(sB + kStages * kStageB);
    float *ring_v = ring_x + kRingBytes / 4;
    LargeShared *sh = reinterpret_cast<LargeShared *>(ring_v + kRingBytes / 4);
    volatile int32_t *tout = &sh->timed_out;
    volatile int64_t *rec_settled = &sh->rec_settled, *rec_copied = &sh->rec_copied;

    const RunArgs &a = L.a;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // Cluster tiles: CL consecutive output tiles of one replica tile, CTA `crank` of the
    // cluster taking the crank-th; the cluster's CTAs load one CL-th of the spin tile each
    // and multicast it to all of them.
    const int crank = CL > 1 ? (int)cluster_ctarank() : 0;
    const int Gc = (int)gridDim.x / CL, cid = (int)blockIdx.x / CL;
    const int mt = L.mtiles;
    const int mgroups = mt / CL;
    const int ctiles = mgroups * L.rtiles;
    const int my_tiles = cid < ctiles ? (ctiles - 1 - cid) / Gc + 1 : 0;
    auto tile_m = [&](int lt) { return ((cid + lt * Gc) % mgroups) * CL + crank; };
    auto tile_n = [&](int lt) { return (cid + lt * Gc) / mgroups; };
    const int64_t t0 = L.f0, t_end = L.f1, t_call_end = a.t0 + a.nsteps;
    const int64_t total = (t_end - t0) * my_tiles;      // tiles this CTA processes, g = 0 .. total - 1
    const int KB = L.Kbytes / kBKB;
    const int N = a.N, R = a.R;
    const uint64_t kWaitNs = a.wait_ns > 0 ? (uint64_t)a.wait_ns : kWaitTimeoutNs;
    uint32_t *ready = L.ready, *settled = L.ready + L.rtiles;
    // Barriers of accumulator b (a third one sits after the first two's).
    auto accf_of = [&](int b) -> uint64_t * { return NACC > 2 && b == 2 ? &sh->accf2 : &sh->accf[b]; };
    auto acce_of = [&](int b) -> uint64_t * { return NACC > 2 && b == 2 ? &sh->acce2 : &sh->acce[b]; };
    auto tiledone_of = [&](int b) -> uint64_t * { return NACC > 2 && b == 2 ? &sh->tiledone2 : &sh->tiledone[b]; };

    if (warp == 0) {
        tmem_alloc(&sh->tmem_base, Tile<BN, true>::kTmemCols);
        tmem_relinquish();
    }
    if (tid == 32) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&sh->full[s], 1);
            mbar_init(&sh->empty[s], CL);   // freed by the MMAs of every CTA of the cluster
        }
        for (int b = 0; b < NACC; ++b) {
            mbar_init(accf_of(b), 1);
            mbar_init(acce_of(b), kEpiWarps + 1);   // + the signal warp
            mbar_init(tiledone_of(b), kEpiWarps);
        }
        mbar_init(&sh->drain, 1);
        sh->timed_out = 0;
        sh->rec_settled = t0 - 1;
        sh->rec_copied = t0 - 1;
        fence_mbarrier_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if constexpr (CL > 1) cluster_sync_all();   // every CTA's barriers exist before any multicast
    const uint32_t tmem = sh->tmem_base;

    if (warp == 0) {
        // TMA producer: tile g is iteration t0 + g / my_tiles of output tile g % my_tiles.
        if (lane == 0 && !a.stall_producer) {
            int64_t kg = 0;
            bool ok = true;
            for (int64_t g = 0; g < total && ok; ++g) {
                const int lt = (int)(g % my_tiles);
                const int64_t t = t0 + g / my_tiles;
                const int m = tile_m(lt), n = tile_n(lt);
                // the spins of iteration t of replica tile n: all its output tiles finished t - 1
                if (!wait_counter_at_least(ready + n, (uint32_t)(mt * (t - t0)), kWaitNs, tout)) {
                    ok = false;
                    break;
                }
                fence_proxy_async_global();
                const int ybuf = (int)(t & 3) * L.Rpad + n * BN;
                for (int kb = 0; kb < KB; ++kb, ++kg) {
                    const int s = (int)(kg % kStages);
                    if (kg >= kStages &&
                        (*tout || !mbar_wait_bounded(&sh->empty[s], (uint32_t)((kg / kStages) - 1) & 1u, kWaitNs))) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&sh->full[s], kStageA + kStageB);
                    tma_load_2d(sA + s * kStageA, &tmA, &sh->full[s], kb * (kBKB / ESZ), m * kBM);
                    if constexpr (CL == 1) {
                        tma_load_2d(sB + s * kStageB, &tmB, &sh->full[s], kb * (kBKB / ESZ), ybuf);
                    } else {
                        tma_load_2d_mc(sB + s * kStageB + crank * (BN / CL) * kBKB, &tmB, &sh->full[s],
                                       kb * (kBKB / ESZ), ybuf + crank * (BN / CL), kMask);
                    }
                }
            }
            if (!ok) *tout = 1;
            for (int64_t k = kg > kStages ? kg - kStages : 0; k < kg; ++k)
                mbar_wait_bounded(&sh->full[k % kStages], (uint32_t)(k / kStages) & 1u, kWaitNs);
        }
    } else if (warp == 1) {
        // MMA issuer: accumulators alternate per tile.
        if (lane == 0) {
            int64_t kg = 0;
            bool ok = true;
            for (int64_t g = 0; g < total && ok; ++g) {
                const int b = (int)((uint64_t)g % NACC);
                if (g >= NACC &&
                    (*tout || !mbar_wait_bounded(acce_of(b), (uint32_t)(((uint64_t)g / NACC) - 1) & 1u, kWaitNs))) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t dt = tmem + (uint32_t)(b * BN);
                for (int kb = 0; kb < KB; ++kb, ++kg) {
                    const int s = (int)(kg % kStages);
                    if (*tout || !mbar_wait_bounded(&sh->full[s], (uint32_t)(kg / kStages) & 1u, kWaitNs)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t ad = smem_desc_sw128(smem_u32(sA + s * kStageA));
                    const uint64_t bd = smem_desc_sw128(smem_u32(sB + s * kStageB));
#pragma unroll
                    for (int k = 0; k < kBKB / 32; ++k) {
                        if constexpr (OP == kOpE4M3) mma_e4m3(dt, ad + 2 * k, bd + 2 * k, IDESC, (kb | k) != 0);
                        else mma_bf16(dt, ad + 2 * k, bd + 2 * k, IDESC, (kb | k) != 0);
                    }
                    if constexpr (CL == 1) mma_commit(&sh->empty[s]);
                    else mma_commit_mc(&sh->empty[s], kMask);   // stage s free in every CTA of the cluster
                }
                if (ok) mma_commit(accf_of(b));
            }
            if (!ok) *tout = 1;
            mma_commit(&sh->drain);
            mbar_wait_bounded(&sh->drain, 0, kWaitNs);
        }
    } else if (warp < 2 + kEpiWarps) {
        // Epilogue warps, as in the per-iteration kernel; tiles follow each other across
        // iterations, and the x/v ring prefetches across both.
        const int ew = warp - 2;
        const int q4 = warp & 3;
        const int cg = ew >> 2;
        const int et = ew * 32 + lane;
        const int Mp = L.Mp;
        float4 *rx4 = reinterpret_cast<float4 *>(ring_x) + et;
        float4 *rv4 = reinterpret_cast<float4 *>(ring_v) + et;
        const size_t grp_stride = (size_t)Mp * 4;
        auto xv_offset = [&](int m_, int n_, int c_) -> size_t {
            const int grp = (n_ * BN + cg * kColsPerWarp + c_ * kChunk) >> 2;
            return ((size_t)grp * Mp + (m_ * kBM + q4 * 32 + lane)) * 4;
        };
        // Freshly written x and v are read again next iteration; with a state larger than
        // half of L2 their lines are kept ahead of the operand streams' (evict_last).  The
        // cluster variants keep plain stores (their registers are tighter).
        const bool keep = CL == 1 && L.xv_keep != 0;
        const uint64_t xvpol = l2_evict_last_policy();
        auto put4 = [&](float *p, float4 v) {
            if (keep) st_global_f4_policy(p, v, xvpol);
            else *reinterpret_cast<float4 *>(p) = v;
        };
        auto issue = [&](size_t off, int slot_) {
            cp_async_16(rx4 + (2 * slot_) * kEpiThreads, L.X + off);
            cp_async_16(rx4 + (2 * slot_ + 1) * kEpiThreads, L.X + off + grp_stride);
            cp_async_16(rv4 + (2 * slot_) * kEpiThreads, L.V + off);
            cp_async_16(rv4 + (2 * slot_ + 1) * kEpiThreads, L.V + off + grp_stride);
        };
        if (total > 0) {
            for (int c0 = 0; c0 < kRing - 1; ++c0) {
                issue(xv_offset(tile_m(0), tile_n(0), c0), c0);
                cp_async_commit();
            }
        }
        const float inv_tm1 = inv_tm1_of(a.T_total);
        int slot = 0;
        bool ok = true;
        for (int64_t g = 0; g < total; ++g) {
            const int lt = (int)(g % my_tiles);
            const int64_t t = t0 + g / my_tiles;
            const int m = tile_m(lt), n = tile_n(lt);
            const int b = (int)((uint64_t)g % NACC);
            const bool has_nxt = g + 1 < total;
            const int lt_nxt = (int)((g + 1) % my_tiles);
            const int m_nxt = tile_m(lt_nxt), n_nxt = tile_n(lt_nxt);
            const int i = m * kBM + q4 * 32 + lane;
            const bool live_i = i < N;
            const float bgq = beta_at(t, inv_tm1, a.beta0, a.beta1) * (a.gamma * a.q);
            const float eps = a.eps, gamma = a.gamma;
            const bool more = t + 1 < t_call_end;
            const bool refresh_next = more && refresh_at(t + 1, a.refresh);
            const int32_t hki = live_i ? a.hk[i] : 0;
            const float hkf = (float)hki;
            const int rc0 = n * BN + cg * kColsPerWarp;
            const int ncol = max(0, min(kColsPerWarp, R - rc0));
            uint8_t *swarp = L.S + (size_t)((t + 1) & 3) * L.Rpad * L.Kbytes + (size_t)rc0 * L.Kbytes +
                             (size_t)(m * kBM + q4 * 32) * ESZ;
            uint32_t *bwarp = L.sbits + ((size_t)((t + 1) & 3) * (Mp / 32) + m * 4 + q4) * L.Rpad + rc0;
            // The spins of t + 1 overwrite those of t - 3: their best copy must be done.
            if (ok && more && t - 3 >= t0) {
                const uint64_t ts = globaltimer_ns();
                while (*rec_copied < t - 3) {
                    if (*tout || globaltimer_ns() - ts > kWaitNs) {
                        ok = false;
                        break;
                    }
                    __nanosleep(64);
                }
            }
            ok = __all_sync(0xffffffffu, ok && !*tout &&
                                             mbar_wait_bounded(accf_of(b), (uint32_t)((uint64_t)g / NACC) & 1u, kWaitNs));
            if (!ok) *tout = 1;
            tc_fence_after();
            const uint32_t tbase = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(b * BN + cg * kColsPerWarp);
            uint32_t accn[kChunk];
            if (ok) {
                tmem_ld_x8_issue(tbase, accn);
                tmem_ld_wait_x8(accn);
            }
            unsigned long long *ep = reinterpret_cast<unsigned long long *>(L.Epart) + (size_t)(t & 1) * L.Rpad;
#pragma unroll 1
            for (int c = 0; c < kChunksPerTile; ++c) {
                const int col0 = c * kChunk;
                {
                    const int ca = c + kRing - 1;
                    const int sa = slot + kRing - 1 >= kRing ? slot - 1 : slot + kRing - 1;
                    if (ca < kChunksPerTile) issue(xv_offset(m, n, ca), sa);
                    else if (has_nxt) issue(xv_offset(m_nxt, n_nxt, ca - kChunksPerTile), sa);
                    cp_async_commit();
                }
                cp_async_wait<kRing - 1>();
                const int sc = slot;
                slot = slot + 1 == kRing ? 0 : slot + 1;
                if (!ok) continue;
                const float4 x0 = rx4[(2 * sc) * kEpiThreads], x1 = rx4[(2 * sc + 1) * kEpiThreads];
                const float4 v0 = rv4[(2 * sc) * kEpiThreads], v1 = rv4[(2 * sc + 1) * kEpiThreads];
                float acc[kChunk];
#pragma unroll
                for (int j = 0; j < kChunk; ++j) acc[j] = __uint_as_float(accn[j]);
                const bool ld_next = c + 1 < kChunksPerTile;
                if (ld_next) tmem_ld_x8_issue(tbase + col0 + kChunk, accn);
                const float xs[kChunk] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
                float vs[kChunk] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
                const int nlive = live_i ? ncol - col0 : 0;
                int32_t p[kChunk];
                chunk_field_momentum(acc, xs, vs, hki, hkf, nlive, a.deriv, eps, bgq, gamma, p);
                // the warp's sum of column j lands in lane j, which adds it to the replica's total
                int32_t mine = 0;
#pragma unroll
                for (int j = 0; j < kChunk; ++j) {
                    const int32_t ps = __reduce_add_sync(0xffffffffu, p[j]);
                    if (lane == j) mine = ps;
                }
                if (lane < kChunk && mine != 0) atomicAdd(ep + rc0 + col0 + lane, (unsigned long long)(long long)mine);
                if (refresh_next) {
#pragma unroll
                    for (int j = 0; j < kChunk; ++j)
                        vs[j] = draw_v(a.seed, a.inst, (uint32_t)(rc0 + col0 + j), (uint32_t)i, (uint32_t)(t + 1));
                }
                const size_t off = xv_offset(m, n, c);
                if (more) {
                    float xn[kChunk];
#pragma unroll
                    for (int j = 0; j < kChunk; ++j) xn[j] = xs[j] + eps * vs[j];
                    put4(L.X + off, make_float4(xn[0], xn[1], xn[2], xn[3]));
                    put4(L.X + off + grp_stride, make_float4(xn[4], xn[5], xn[6], xn[7]));
                    chunk_store_spins<OP>(xn, lane, ncol - col0, swarp + (size_t)col0 * L.Kbytes, L.Kbytes,
                                          m * kBM + q4 * 32, N, sh->masks[ew], bwarp + col0);
                }
                put4(L.V + off, make_float4(vs[0], vs[1], vs[2], vs[3]));
                put4(L.V + off + grp_stride, make_float4(vs[4], vs[5], vs[6], vs[7]));
                if (ld_next) tmem_ld_wait_x8(accn);
            }
            // The tile is done: the signal warp publishes it (its arrival on tiledone carries
            // this warp's stores), then the accumulator is released.
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tiledone_of(b));
            if (lane == 0) mbar_arrive(acce_of(b));
        }
        cp_async_wait<0>();
    } else if (warp == 2 + kEpiWarps) {
        // Records warp.
        constexpr int K = BN / 32;   // replicas per lane of a replica tile
        for (int64_t t = t0; t < t_end && !*tout; ++t) {
            bool ok = true;
            for (int lt = 0; lt < my_tiles && ok; ++lt) {
                const int n = tile_n(lt);
                if (tile_m(lt) != 0) continue;
                ok = wait_counter_at_least(ready + n, (uint32_t)(mt * (t - t0 + 1)), kWaitNs, tout);
                if (!ok) break;
                settle_lane<K>(L, n * BN + lane, t, 3);
                __syncwarp();
                if (lane == 0) {
                    __threadfence();
                    st_release_gpu(settled + n, (uint32_t)(t - t0 + 1));
                }
                __syncwarp();
            }
            if (lane == 0) *rec_settled = t;
            for (int lt = 0; lt < my_tiles && ok; ++lt) {
                const int m = tile_m(lt), n = tile_n(lt);
                ok = wait_counter_at_least(settled + n, (uint32_t)(t - t0 + 1), kWaitNs, tout);
                if (ok) copy_best_lane<K>(L, n * BN + lane, m, t);
            }
            if (!ok) {
                *tout = 1;
                break;
            }
            __syncwarp();
            if (lane == 0) *rec_copied = t;
        }
    } else if (lane == 0) {
        // Signal warp: once the epilogue warps finished tile g, make their spins and
        // energy terms visible to the GPU and count the tile in ready[n].  The m = 0 tile
        // of a replica tile is counted for iteration t only after its energy sums of t - 1
        // were read out (those of t + 1 go to the same slot).
        for (int64_t g = 0; g < total; ++g) {
            const int b = (int)((uint64_t)g % NACC);
            const int lt = (int)(g % my_tiles);
            const int64_t t = t0 + g / my_tiles;
            const int m = tile_m(lt), n = tile_n(lt);
            if (*tout || !mbar_wait_bounded(tiledone_of(b), (uint32_t)((uint64_t)g / NACC) & 1u, kWaitNs)) {
                *tout = 1;
                break;
            }
            mbar_arrive(acce_of(b));
            if (m == 0 && t - 1 >= t0) {
                const uint64_t ts = globaltimer_ns();
                bool go = true;
                while (*rec_settled < t - 1) {
                    if (*tout || globaltimer_ns() - ts > kWaitNs) {
                        go = false;
                        break;
                    }
                    __nanosleep(32);
                }
                if (!go) {
                    *tout = 1;
                    break;
                }
            }
            __threadfence();
            atomicAdd(ready + n, 1u);
        }
    }
    tc_fence_before();
    __syncthreads();
    // No CTA of a cluster leaves while another may still multicast into it or arrive on
    // its barriers.
    if constexpr (CL > 1) cluster_sync_all();
    if (tid == 0 && sh->timed_out) atomicExch(a.err, 1);
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, Tile<BN, true>::kTmemCols);
    }
}

// Initial state (or given), refresh at t0, first position update, spins of iteration t0;
// one thread per element of the padded interleaved x/v arrays (padding set to 0).
template <int OP>
__global__ void tc_large_prologue(const LargeArgs L) {
    const RunArgs &a = L.a;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx == 0) iter_ctl_start(L.ctl, a.t0, a.nsteps);
    if (idx >= (int64_t)L.Rpad * L.Mp) return;
    const int64_t gi = idx >> 2;                       // (group, spin)
    const int grp = (int)(gi / L.Mp), i = (int)(gi - (int64_t)grp * L.Mp);
    const int r = grp * 4 + (int)(idx & 3);
    float x = 0.0f, v = 0.0f;
    if (r < a.R && i < a.N) {
        const size_t src = (size_t)r * a.N + i;
        if (a.x_in) {
            x = a.x_in[src];
            v = a.v_in[src];
        } else {
            const U4 o = draw_raw(a.seed, a.inst, (uint32_t)r, (uint32_t)i, 0u);
            x = box_muller(o.x, o.y);
            v = box_muller(o.z, o.w);
        }
        if (refresh_at(a.t0, a.refresh)) v = draw_v(a.seed, a.inst, (uint32_t)r, (uint32_t)i, (uint32_t)a.t0);
        x = x + a.eps * v;
        put_spin_byte<OP>(L.S + ((size_t)(a.t0 & 3) * L.Rpad + r) * L.Kbytes, i, x >= 0.0f);
    }
    L.X[idx] = x;
    L.V[idx] = v;
}

// Final state back to the caller's [R][N] arrays.
__global__ void tc_large_export(const LargeArgs L) {
    const RunArgs &a = L.a;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)a.R * a.N) return;
    const int r = (int)(idx / a.N), i = (int)(idx - (int64_t)r * a.N);
    const size_t src = ((size_t)(r >> 2) * L.Mp + i) * 4 + (r & 3);
    if (a.x_out) a.x_out[idx] = L.X[src];
    if (a.v_out) a.v_out[idx] = L.V[src];
}

// Field-only mode: spins given, field and energy out (no records).
template <int OP>
__global__ void tc_large_field_prologue(const LargeArgs L) {
    const RunArgs &a = L.a;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx == 0) iter_ctl_start(L.ctl, 0, 1);
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

template <int OP, int BN, int CL, bool RING>
cudaError_t run_large(const LargeBuffers &B, const RunArgs &a, cudaStream_t st, int *launches, int sms) {
    constexpr size_t kSmem = Tile<BN, RING>::kSmemBytes;
    LargeArgs L;
    memset(&L, 0, sizeof L);   // the bytes key the graph cache
    L.a = a;
    L.ctl = B.ctl;
    L.S = B.S;
    L.Epart = B.Epart;
    L.flags = B.flags;
    L.Kbytes = B.Kbytes;
    L.Rpad = B.Rpad;
    L.mtiles = B.Mpad / kBM;
    L.rtiles = (a.R + BN - 1) / BN;
    L.ntiles = L.mtiles * L.rtiles;
    L.X = B.X;
    L.V = B.V;
    L.Mp = B.Mpad;
    CUtensorMap tmA, tmB;
    const int esz = OP == kOpE4M3 ? 1 : 2;
    if (!make_map(&tmA, B.Jop, OP, (uint64_t)B.Kbytes / esz, (uint64_t)B.Mpad, (uint64_t)B.Kbytes, kBM) ||
        !make_map(&tmB, B.S, OP, (uint64_t)B.Kbytes / esz, (uint64_t)4 * B.Rpad, (uint64_t)B.Kbytes, BN / CL))
        return cudaErrorInvalidValue;
    auto step = tc_large_step<OP, BN, CL, RING>;
    cudaError_t e = cudaFuncSetAttribute(step, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
    if (e != cudaSuccess) return e;
    // Persistent grid: one CTA per SM, or as many whole clusters as can be resident at once.
    const int ctiles = (L.mtiles / CL) * L.rtiles;
    int clusters = std::min(ctiles, std::max(sms, 1));
    if (CL > 1) {
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3((unsigned)(CL * std::max(sms / CL, 1)));
        cfg.blockDim = dim3(kThreads);
        cfg.dynamicSmemBytes = kSmem;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = CL;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int resident = 0;
        e = cudaOccupancyMaxActiveClusters(&resident, reinterpret_cast<const void *>(step), &cfg);
        if (e != cudaSuccess) return e;
        if (resident < 1) return cudaErrorInvalidConfiguration;
        clusters = std::min(ctiles, resident);
    }
    const dim3 grid((unsigned)(clusters * CL));
    e = cudaMemsetAsync(B.Epart, 0, 2 * (size_t)B.Rpad * sizeof(int64_t), st);   // energy sums start at 0
    if (e != cudaSuccess) return e;
    const int64_t RN = (int64_t)a.R * a.N;
    const unsigned eg = (unsigned)((RN + 255) / 256);
    int n = 0;
    if (a.field_mode) {
        L.a.nsteps = 1;
        L.a.T_total = 1;
        tc_large_field_prologue<OP><<<eg, 256, 0, st>>>(L);
        void *args[3] = {&tmA, &tmB, &L};
        e = launch_steps(nullptr, reinterpret_cast<const void *>(step), grid, dim3(kThreads), kSmem, args, nullptr, 0,
                         1, st, CL);
        if (e != cudaSuccess) return e;
        tc_large_field_out<<<(a.R + 255) / 256, 256, 0, st>>>(L);
        n += 3;
        if (launches) *launches += n;
        return cudaGetLastError();
    }
    const int64_t RMp = (int64_t)B.Rpad * B.Mpad;
    tc_large_prologue<OP><<<(unsigned)((RMp + 255) / 256), 256, 0, st>>>(L);
    ++n;
    {
        // The step kernel reads its iteration from L.ctl: every launch is the same, and
        // the arguments leave out what only the prologue and the export read.
        LargeArgs Ls = L;
        Ls.a.t0 = 0;
        Ls.a.nsteps = 0;
        Ls.a.x_in = Ls.a.v_in = nullptr;
        Ls.a.x_out = Ls.a.v_out = nullptr;
        void *args[3] = {&tmA, &tmB, &Ls};
        uint8_t key[2 * sizeof(CUtensorMap) + sizeof(LargeArgs)];
        memcpy(key, &tmA, sizeof tmA);
        memcpy(key + sizeof tmA, &tmB, sizeof tmB);
        memcpy(key + 2 * sizeof tmA, &Ls, sizeof Ls);
        e = launch_steps(B.graphs, reinterpret_cast<const void *>(step), grid, dim3(kThreads), kSmem, args, key,
                         sizeof key, a.nsteps, st, CL);
        if (e != cudaSuccess) return e;
        n += (int)a.nsteps;
    }
    const int64_t t_last = a.t0 + a.nsteps - 1;
    tc_large_settle<<<(a.R + 255) / 256, 256, 0, st>>>(L, t_last);
    const int64_t RW = (int64_t)a.R * a.W;
    tc_large_copy<OP><<<(unsigned)((RW + 255) / 256), 256, 0, st>>>(L, t_last - 1 >= a.t0 ? t_last - 1 : t_last,
                                                                     t_last);
    tc_large_count<<<1, 32, 0, st>>>(L);
    n += 3;
    if (a.x_out || a.v_out) {
        tc_large_export<<<eg, 256, 0, st>>>(L);
        ++n;
    }
    if (launches) *launches += n;
    return cudaGetLastError();
}

// Packed spins of the run's first iteration (the epilogue writes those of later ones).
template <int OP>
__global__ void tc_flow_pack0(const LargeArgs L) {
    constexpr int ESZ = OP == kOpE4M3 ? 1 : 2;
    const int Wp = L.Mp / 32, W = L.a.W;   // words past W are never read unmasked
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)L.a.R * W) return;
    const int w = (int)(idx / L.a.R), r = (int)(idx - (int64_t)w * L.a.R);
    const int64_t slot = L.a.t0 & 3;
    const uint8_t *row = L.S + ((size_t)slot * L.Rpad + r) * L.Kbytes;
    L.sbits[((size_t)slot * Wp + w) * L.Rpad + r] = plus_bits32<OP>(row + (size_t)w * 32 * ESZ);
}

// Variants 7-13: the whole run in cooperative launches of tc_flow_run (all CTAs resident
// at once, as CTAs wait on each other's tiles), with NACC TMEM accumulators.  Runs whose tile counters could pass 2^31 go
// out in several launches; every launch settles and copies all of its iterations.
template <int OP, int BN, int CL, int NACC = 2>
cudaError_t run_flow(const LargeBuffers &B, const RunArgs &a, cudaStream_t st, int *launches, int sms) {
    constexpr size_t kSmem = Tile<BN, true>::kSmemBytes;
    constexpr int kFlowThreads = kThreads + 64;
    LargeArgs L;
    memset(&L, 0, sizeof L);
    L.a = a;
    L.ctl = B.ctl;
    L.S = B.S;
    L.Epart = B.Epart;
    L.flags = B.flags;
    L.Kbytes = B.Kbytes;
    L.Rpad = B.Rpad;
    L.mtiles = B.Mpad / kBM;
    L.rtiles = (a.R + BN - 1) / BN;
    L.ntiles = L.mtiles * L.rtiles;
    L.X = B.X;
    L.V = B.V;
    L.Mp = B.Mpad;
    L.ready = B.ready;
    L.sbits = B.sbits;
    {
        int dev = 0, l2 = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) == cudaSuccess)
            L.xv_keep = (size_t)B.Rpad * (size_t)B.Mpad * 8 * 2 > (size_t)l2 ? 1 : 0;
    }
    CUtensorMap tmA, tmB;
    const int esz = OP == kOpE4M3 ? 1 : 2;
    if (!make_map(&tmA, B.Jop, OP, (uint64_t)B.Kbytes / esz, (uint64_t)B.Mpad, (uint64_t)B.Kbytes, kBM) ||
        !make_map(&tmB, B.S, OP, (uint64_t)B.Kbytes / esz, (uint64_t)4 * B.Rpad, (uint64_t)B.Kbytes, BN / CL))
        return cudaErrorInvalidValue;
    auto k = tc_flow_run<OP, BN, CL, NACC>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
    if (e != cudaSuccess) return e;
    // All CTAs (whole clusters) resident at once: the launch is cooperative.
    cudaLaunchConfig_t cfg{};
    cfg.blockDim = dim3(kFlowThreads);
    cfg.dynamicSmemBytes = kSmem;
    cfg.stream = st;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    at[1].id = cudaLaunchAttributeClusterDimension;
    at[1].val.clusterDim.x = CL;
    at[1].val.clusterDim.y = 1;
    at[1].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = CL > 1 ? 2 : 1;
    const int ctiles = (L.mtiles / CL) * L.rtiles;
    int resident = 0;
    if (CL > 1) {
        cudaLaunchConfig_t q = cfg;
        q.gridDim = dim3((unsigned)(CL * std::max(sms / CL, 1)));
        q.attrs = at + 1;
        q.numAttrs = 1;
        e = cudaOccupancyMaxActiveClusters(&resident, reinterpret_cast<const void *>(k), &q);
    } else {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k, kFlowThreads, kSmem);
        resident *= std::max(sms, 1);
    }
    if (e != cudaSuccess) return e;
    if (resident < 1) return cudaErrorInvalidConfiguration;
    cfg.gridDim = dim3((unsigned)(CL * std::min(ctiles, resident)));
    e = cudaMemsetAsync(B.Epart, 0, 2 * (size_t)B.Rpad * sizeof(int64_t), st);
    if (e != cudaSuccess) return e;
    int n = 0;
    const int64_t RMp = (int64_t)B.Rpad * B.Mpad;
    tc_large_prologue<OP><<<(unsigned)((RMp + 255) / 256), 256, 0, st>>>(L);
    const int64_t RW = (int64_t)a.R * a.W;
    tc_flow_pack0<OP><<<(unsigned)((RW + 255) / 256), 256, 0, st>>>(L);
    n += 2;
    const int64_t chunk = std::max<int64_t>(1, ((int64_t)1 << 31) / L.mtiles - 1);
    for (int64_t t = a.t0; t < a.t0 + a.nsteps; t += chunk) {
        LargeArgs Lc = L;
        Lc.f0 = t;
        Lc.f1 = t + std::min(chunk, a.t0 + a.nsteps - t);
        Lc.a.x_in = Lc.a.v_in = nullptr;
        Lc.a.x_out = Lc.a.v_out = nullptr;
        e = cudaMemsetAsync(B.ready, 0, 2 * (size_t)L.rtiles * sizeof(uint32_t), st);
        if (e != cudaSuccess) return e;
        void *args[3] = {&tmA, &tmB, &Lc};
        e = cudaLaunchKernelExC(&cfg, reinterpret_cast<const void *>(k), args);
        if (e != cudaSuccess && CL > 1 && t == a.t0) {
            // a cooperative launch in clusters refused: the whole call without clusters (the
            // prologue reads only the caller's arrays, so it runs again unchanged)
            cudaGetLastError();
            return run_flow<OP, BN, 1, NACC>(B, a, st, launches, sms);
        }
        if (e != cudaSuccess) return e;
        ++n;
    }
    tc_large_count<<<1, 32, 0, st>>>(L);
    ++n;
    if (a.x_out || a.v_out) {
        const int64_t RN = (int64_t)a.R * a.N;
        tc_large_export<<<(unsigned)((RN + 255) / 256), 256, 0, st>>>(L);
        ++n;
    }
    if (launches) *launches += n;
    return cudaGetLastError();
}

template <int OP, int BN>
cudaError_t run_variant(const LargeBuffers &B, const RunArgs &a, cudaStream_t st, int *launches, int sms) {
    const int mtiles = B.Mpad / kBM;
    int v = a.large_variant;
    if (v == 0) v = kDefaultLargeVariant;
    // The overlapped variants need their tile counters (absent from the allocation-free
    // entry); clusters need the output tiles to split evenly among their CTAs.
    if (v >= 7 && (!B.ready || !B.sbits || a.field_mode)) v = 1;
    if (v >= 10) v = 7;
    if (v == 9 && mtiles % 4 != 0) v = 8;
    if (v == 8 && mtiles % 2 != 0) v = 7;
    if (v == 9) return run_flow<OP, BN, 4>(B, a, st, launches, sms);
    if (v == 8) return run_flow<OP, BN, 2>(B, a, st, launches, sms);
    if (v == 7) return run_flow<OP, BN, 1>(B, a, st, launches, sms);
    // A cluster needs the spin tiles to split evenly among its CTAs.
    if (v == 6 && mtiles % 4 != 0) v = 5;
    if (v == 5 && mtiles % 2 != 0) v = 1;
    if (v == 4 && mtiles % 4 != 0) v = 3;
    if (v == 3 && mtiles % 2 != 0) v = 2;
    if (v == 6) return run_large<OP, BN, 4, true>(B, a, st, launches, sms);
    if (v == 5) return run_large<OP, BN, 2, true>(B, a, st, launches, sms);
    if (v == 4) return run_large<OP, BN, 4, false>(B, a, st, launches, sms);
    if (v == 3) return run_large<OP, BN, 2, false>(B, a, st, launches, sms);
    if (v == 2) return run_large<OP, BN, 1, false>(B, a, st, launches, sms);
    return run_large<OP, BN, 1, true>(B, a, st, launches, sms);
}

}  // namespace

cudaError_t launch_tc_large(const LargeBuffers &B, const RunArgs &a, int op, cudaStream_t st, int *launches) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (a.large_variant < 0 || a.large_variant > 13) return cudaErrorInvalidValue;
    // The overlapped kernel's tile width: variants 10 / 11 / 12 / 13 fix it at 256 / 224 /
    // 128 / 160 replicas; variant 7 takes the width whose estimated iteration time is least.
    // With w tiles on the busiest CTA, an epilogue of E = 0.045 us per replica column of a
    // tile and a TMA + MMA mainloop of M = Kbytes x (128 + BN) / (90 bytes per ns) per tile
    // (both fitted to timings at N = 1024 / 2000 / 4000), an iteration takes about
    // max(w E, w M, E + 1.5 us + M): the epilogues or the mainloops of a CTA back to back,
    // or, with one tile, its own epilogue, the counter round trip and its next mainloop
    // in series (no other tile to hide them behind).  160-wide tiles leave room in tensor
    // memory for three accumulators; where the mainloops set the pace they cut the bytes
    // per tile at the same tiles per CTA (N = 4000, 1200 replicas: 26.2 against 30.8 us
    // with 224-wide tiles, as the estimate has it).
    const int lv = a.large_variant;
    if ((lv == 7 || lv >= 10) && B.ready && B.sbits && !a.field_mode) {
        const int mt = B.Mpad / kBM;
        const int want = lv == 10 ? 256 : lv == 11 ? 224 : lv == 12 ? 128 : lv == 13 ? 160 : 0;
        int best_bn = 0;
        double best_us = 0.0;
        for (int bn : {256, 224, 160, 128}) {
            if (want && bn != want) continue;
            const int rt = (a.R + bn - 1) / bn;
            if ((int64_t)rt * bn > B.Rpad) continue;
            const double w = (double)(((int64_t)mt * rt + sms - 1) / sms);
            const double E = 0.045 * bn;
            const double M = (double)B.Kbytes * (128 + bn) / 90.0 / 1000.0;
            const double us = std::max(std::max(w * E, w * M), E + 1.5 + M);
            if (!best_bn || us < best_us) {
                best_bn = bn;
                best_us = us;
            }
        }
        if (!best_bn) best_bn = 256;   // a fixed width the padding cannot hold: the standard one
        if (op == kOpE4M3) {
            if (best_bn == 224) return run_flow<kOpE4M3, 224, 1>(B, a, st, launches, sms);
            if (best_bn == 160) return run_flow<kOpE4M3, 160, 1, 3>(B, a, st, launches, sms);
            if (best_bn == 128) return run_flow<kOpE4M3, 128, 1>(B, a, st, launches, sms);
            return run_flow<kOpE4M3, 256, 1>(B, a, st, launches, sms);
        }
        if (best_bn == 224) return run_flow<kOpBF16, 224, 1>(B, a, st, launches, sms);
        if (best_bn == 160) return run_flow<kOpBF16, 160, 1, 3>(B, a, st, launches, sms);
        if (best_bn == 128) return run_flow<kOpBF16, 128, 1>(B, a, st, launches, sms);
        return run_flow<kOpBF16, 256, 1>(B, a, st, launches, sms);
    }
    // 256-replica tiles when they still give every SM one, else 128-replica tiles.
    const bool wide = (int64_t)(B.Mpad / kBM) * ((a.R + 255) / 256) >= sms;
    if (op == kOpE4M3)
        return wide ? run_variant<kOpE4M3, 256>(B, a, st, launches, sms) : run_variant<kOpE4M3, 128>(B, a, st, launches, sms);
    return wide ? run_variant<kOpBF16, 256>(B, a, st, launches, sms) : run_variant<kOpBF16, 128>(B, a, st, launches, sms);
}

}  // namespace phia
