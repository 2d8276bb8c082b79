// phia_internal.h -- declarations shared by the library's translation units (not part
// of the public ABI; see include/phia.h for that).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace phia {

// One CTA's instance in a batched run of small dense instances (the resident tcgen05
// kernel with an instance table): where its couplings and field are, its size, Philox
// instance id and fixed-point scale, its first replica, and where its records start.
struct SmallCta {
    const int8_t *Jk;       // [N][N]
    const int32_t *hk;      // [N]
    int32_t N, W;           // spins, ceil(N / 32)
    uint32_t inst;
    float q;
    int32_t rbase;          // first replica of this CTA (within the instance)
    int64_t rec_off;        // into the per-replica record arrays
    int64_t bits_off;       // into the bit-packed best states
    int64_t target;         // target energy (units of q)
};

// Everything one run of the hot path needs.  Replica-state arrays are [R][N]
// row-major FP32; per-replica records persist across resumable calls.
struct RunArgs {
    // instance
    int32_t N;
    int32_t frac_bits;
    const int8_t *Jk;      // dense k, [N][N] int8 (exact storage)
    const int32_t *hk;     // [N]
    const float *Jf;       // FP32 copy of J = k q (FP32 path)
    const int32_t *row_ptr; const int32_t *col; const int8_t *val;  // CSR
    // run
    int32_t R;
    int64_t t0, nsteps, T_total;
    float beta0, beta1, eps, gamma, q;
    int32_t refresh;
    int32_t deriv;              // derivative factor of Eq. 8: 0 exact, 1 quadratic stand-in
    uint64_t seed;
    uint32_t inst;
    const float *x_in, *v_in;   // initial state, or null -> Philox draw d = 0
    float *x_out, *v_out;       // final state, or null
    // field-only mode (no dynamics): spins in, field/energy out
    int32_t field_mode;
    const int8_t *spins_in;     // [R][N]
    int32_t *field_out;         // [R][N]
    int64_t *energy_out;        // [R]
    // per-replica records
    int64_t *best_e, *best_step, *hit_step;
    uint64_t *hit_ns;           // %globaltimer when hit_step was recorded (null: not kept)
    uint32_t *best_bits;        // [R][W]
    int32_t W;
    int32_t has_target, stop_at_target;
    int64_t target;
    unsigned long long *min_hit;         // earliest hit over replicas (stop-at-target)
    unsigned long long *replica_iters;   // sum over replicas of iterations run
    int32_t *err;                        // nonzero: a bounded device wait expired
    int32_t tile_rl;                     // tensor-core small path: live replicas per CTA (0 = auto)
    int32_t coupling_mem;                // tensor-core small path: 1 = J in shared, 2 = in tensor memory
    int64_t wait_ns;                     // per-iteration kernel: bound of each device wait (0 = kWaitTimeoutNs)
    int32_t stall_producer;              // per-iteration kernel, testing: the TMA producer issues nothing
    int32_t large_variant;               // per-iteration kernel: 0 auto, 1 x/v ring, 2 x/v in registers,
                                         // 3 / 4 registers + spin tiles multicast over 2 / 4 CTAs, 5 / 6
                                         // ring + multicast, 7-13 overlapped (phia_opts.large_variant)
    int32_t accept_test;                 // Table 3 state 4: 1 = Metropolis test on H at trajectory ends
    int64_t *proposed, *accepted;        // [R] per-replica counts of the test (accept_test = 1)
    const SmallCta *small_cta;           // batched small dense runs: one entry per CTA
    int32_t small_ctas;                  // its length
};

constexpr uint64_t kWaitTimeoutNs = 2000000000ull;  // 2 s bound on every device-side wait

// Iteration control of a per-iteration path, in device memory.  The run's prologue
// kernel sets it; every step launch reads t (and the run's range) at its start and the
// last CTA of the launch to finish advances t.  Step launches therefore have identical
// arguments, so a chunk of them can be replayed as one instantiated CUDA graph.
struct IterCtl {
    int64_t t;          // iteration of the next step launch
    int64_t t_first;    // first iteration of the run
    int64_t t_end;      // one past the run's last iteration
    uint32_t done;      // CTAs of the current launch that have finished
    uint32_t pad;
};

#ifdef __CUDACC__
// End of a step launch, called by one thread per CTA after the CTA's last read of the
// control block: the last CTA to arrive advances the iteration for the next launch.
__device__ __forceinline__ void iter_ctl_finish(IterCtl *c) {
    __threadfence();
    const unsigned total = gridDim.x * gridDim.y * gridDim.z;
    if (atomicAdd(&c->done, 1u) == total - 1) {
        c->done = 0;
        c->t = c->t + 1;
        __threadfence();
    }
}
// The prologue of a run (one thread).
__device__ __forceinline__ void iter_ctl_start(IterCtl *c, int64_t t0, int64_t nsteps) {
    c->t = t0;
    c->t_first = t0;
    c->t_end = t0 + nsteps;
    c->done = 0;
}
#endif

// Instantiated graphs of step launches, owned by a handle or a batch.
struct StepGraphCache;
StepGraphCache *step_graphs_new();
void step_graphs_free(StepGraphCache *c);
// `steps` launches of `func` with the argument list `args` (each launch identical): full
// chunks replay one cached graph of up to 100 launches, the rest launch directly.  With
// no cache every launch is direct.  The cache key is the kernel, its launch shape and
// the argument bytes `key` (`key_bytes` of them).  cluster > 1: thread-block clusters of
// that many CTAs along x.
cudaError_t launch_steps(StepGraphCache *cache, const void *func, dim3 grid, dim3 block, size_t smem, void **args,
                         const void *key, size_t key_bytes, int64_t steps, cudaStream_t st, unsigned cluster = 1);
constexpr int kOpE4M3 = 1;
constexpr int kOpBF16 = 2;

// tcgen05 persistent kernel for small dense instances (J resident in shared memory).
int tc_small_max_n(int op);
int tc_small_tile_replicas(int R, int requested);
cudaError_t launch_tc_small(const RunArgs &a, int op, cudaStream_t st, int *launches);
// The same kernel over a table of CTAs (a.small_cta, a.small_ctas entries, 8 live replicas
// each) of small dense instances of one operand and one number of 128-spin tiles (mt):
// all iterations of every instance in one launch; no early stop at a target.
cudaError_t launch_tc_small_batch(const RunArgs &a, int op, int mt, int kpad, cudaStream_t st);

// tcgen05 per-iteration kernel for dense instances of any size (TMA-staged J and spins).
struct LargeBuffers {
    const void *Jop;      // [Mpad][Kbytes] couplings in the operand encoding
    uint8_t *S;           // [4][Rpad][Kbytes] spin operand buffers (zero padding)
    int64_t *Epart;       // [2][Rpad], zero between uses
    int8_t *flags;        // [2][Rpad] ([4][Rpad] with the tile counters below)
    float *X, *V;         // [Rpad/4][Mpad][4] working state (replica groups of 4 interleaved per spin)
    IterCtl *ctl;         // iteration control
    StepGraphCache *graphs;   // or null: step launches go out one by one
    uint32_t *ready;      // [2][Rpad/128] tile counters of the overlapped variant, or null
                          // (then flags has [2][Rpad]; with counters [4][Rpad])
    uint32_t *sbits;      // [4][Rpad][Mpad/32] packed spins of the overlapped variant, or null
    int32_t Kbytes, Mpad, Rpad;
};
cudaError_t launch_tc_large(const LargeBuffers &B, const RunArgs &a, int op, cudaStream_t st, int *launches);
cudaError_t launch_convert_operand(const int8_t *Jk, int N, void *Jop, int Mpad, int Kbytes, int op, cudaStream_t st);
// Device checks of a dense instance into res[4] (initialised by the caller to
// {ULLONG_MAX, ULLONG_MAX, ULLONG_MAX, 0}): res[0] lowest i*N+j with k_ij != k_ji (i < j),
// res[1] lowest i with k_ii != 0, res[2] lowest i with |kh_i| >= 2^24, res[3] max |k_ij|.
cudaError_t launch_check_dense(const int8_t *J, const int32_t *h, int N, unsigned long long *res, unsigned blocks,
                               cudaStream_t st);
inline int large_kbytes(int N, int op) { return ((N * (op == kOpE4M3 ? 1 : 2)) + 127) / 128 * 128; }
inline int round_up(int x, int m) { return (x + m - 1) / m * m; }
// Replica padding of the per-iteration dense path (its widest tile is 256 replicas).
inline int large_rpad(int R) { return round_up(R, 256); }
// Handles pad by one more 256-replica group, so that the overlapped kernel may cut the
// replicas into 224-wide tiles (ceil(R / 224) * 224 <= this).
inline int large_rpad_handle(int R) { return round_up(R, 256) + 256; }

// Sparse batched path: many CSR instances, one launch per iteration over all of them.
struct CsrInst {
    int32_t N;
    uint32_t inst_id;       // fourth Philox counter word
    float q;                // 2^-frac_bits
    int32_t pad;
    int64_t rp_off;         // into row_ptr (N + 1 entries, values relative to nz_off)
    int64_t nz_off;         // into col / val
    int64_t h_off;          // into hk
    int64_t row_base;       // global index of row 0 (rows are stored instance after instance)
    int64_t x_off;          // into X, V ([N][R] per instance)
    int64_t xin_off;        // into caller arrays ([R][N] per instance)
    int64_t s_off;          // into each spin buffer, in uint32 words ([N][R/32] per instance)
    int64_t rec_off;        // into per-replica records (R per instance)
    int64_t bits_off;       // into best_bits (R * ceil(N/32) per instance)
};
struct CsrBlock {
    int32_t inst;
    int32_t i0;             // first of up to 64 rows
};
struct CsrArgs {
    RunArgs a;              // run parameters; record pointers indexed by rec_off + r
    const CsrInst *inst;
    int32_t count;
    const CsrBlock *blocks;
    int32_t nblocks;
    const int32_t *row_ptr; const int32_t *col; const int8_t *val; const int32_t *hk;
    float *X, *V;
    const float *x_in, *v_in;
    float *x_out, *v_out;
    uint32_t *S;            // 4 rotating spin buffers of total_swords words each
    int64_t total_swords;
    int64_t *Esum;          // [2][total_reps]
    int8_t *flags;          // [2][total_reps]
    int64_t total_reps;
    uint32_t *best_bits;
    const long long *targets;   // per instance, or null (then a.target)
    int32_t R;              // replicas per instance as run (multiple of 256)
    int32_t R_real;         // replicas the caller asked for (<= R); the rest pad the groups
    int32_t max_words;      // max ceil(N/32)
    int64_t total_rows;
    IterCtl *ctl;           // iteration control
    int32_t persistent;     // 1: every iteration in one cooperative launch (grid barrier per iteration)
    int32_t pad1;
    unsigned *sync;         // 4 words of device memory for that launch's barrier and work counters
};
cudaError_t launch_csr(const CsrArgs &C, StepGraphCache *graphs, cudaStream_t st, int *launches);

}  // namespace phia
struct phia_batch_s;
struct phia_instance_desc;
struct phia_opts;
struct phia_schedule;
struct phia_stats;
namespace phia {
int batch_create(phia_batch_s **out, int32_t count, const phia_instance_desc *d, const phia_opts *opts);
int batch_run(phia_batch_s *b, const phia_schedule *sched, int32_t R_real, int64_t t0, int64_t steps, int64_t total,
              uint64_t seed, const float *x_in, float *x_out, const float *v_in, float *v_out, int reset,
              const int8_t *spins_in, int32_t *field_out, int64_t *energy_out);
int batch_best(phia_batch_s *b, int inst, int64_t *energy_k, int8_t *spins);
int batch_replica_results(phia_batch_s *b, int inst, int32_t R, int64_t *be, int64_t *bs, int64_t *hs, uint32_t *bits);
int batch_stats(phia_batch_s *b, int inst, phia_stats *out);

// Thread-local error message of the C ABI.
int set_last_error(int code, const char *msg);

// int8 tensor-core resident kernel (mma.sync s8 x s8 -> s32) for small dense instances.
int imma_small_max_n();
cudaError_t launch_imma_small(const RunArgs &a, cudaStream_t st, int *launches);

// Incremental-field resident kernel for small dense instances (CUDA cores, exact
// integer field updated by the columns whose spin changed sign; no field mode).
int inc_small_max_n();
int inc_small_tile_replicas(int N, int requested);
cudaError_t launch_inc_small(const RunArgs &a, cudaStream_t st, int *launches);

// Plain FP32 per-step path (the comparator).  `metro` holds the acceptance test's
// per-replica state (used when a.accept_test = 1): the trajectory's start position
// [R][N], the last iteration's energy, the start's energy and x.x, v.v sums, whether a
// start is known.
struct Fp32Metro {
    float *x_start;
    int64_t *e_last, *e_start;
    float *xx_start, *vv_start;
    int32_t *has_start;
};
cudaError_t launch_fp32_run(const RunArgs &a, float *x, float *v, int8_t *s0, int8_t *s1,
                            int64_t *e_acc, const Fp32Metro &metro, cudaStream_t st, int *launches);

// Vanilla GAHMC (exact zero crossings), one warp per replica; records into a's arrays.
int gahmc_max_n();
cudaError_t launch_gahmc(const RunArgs &a, float travel, int64_t K, int64_t *counts, int32_t *events,
                         int32_t events_cap, cudaStream_t st);

// Philox draws for testing.
cudaError_t launch_philox_draws(uint64_t seed, uint32_t inst, uint32_t d, int R, int N, uint32_t *raw,
                                float *x, float *v, cudaStream_t st);

// Initial state (Philox d = 0) into x, v.
cudaError_t launch_init_state(int R, int N, uint64_t seed, uint32_t inst, float *x, float *v,
                              cudaStream_t st);

}  // namespace phia
