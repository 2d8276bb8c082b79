/*
 * phia.h -- C ABI of the GB300 PHIA library (Parallel Hamiltonian Monte Carlo
 * Ising Annealer, arXiv 2407.10205).
 *
 * Problem (Sec. 2.1, Eq. 2): minimise E(s) = -sum_{i<j} J_ij s_i s_j - sum_i h_i s_i
 * over s in {-1,+1}^N.  Couplings are fixed point (Sec. 2.2: J and h held as
 * fixed-point constants): J_ij = k_ij * 2^-f with int8 k (symmetric, zero
 * diagonal) and h_i = kh_i * 2^-f with int32 kh.  All energies and fields cross
 * this boundary as exact integers in units of q = 2^-f.
 *
 * Method (Eqs. 4-8, A7-A8): every replica carries a continuous position x and
 * momentum v (FP32 on the device) and iterates
 *     x <- x + eps v ;  s = sgn x (sgn 0 = +1) ;  I = J s + h           (Eq. 6)
 *     v <- v + eps (beta_t gamma (1 - tanh^2(gamma x)) I - x)           (Eqs. 5, 8, A7)
 * with beta_t linear from beta0 to beta1 over the run (Table 3, state 4), the
 * momentum redrawn at trajectory starts (Sec. 2.1, Fig. 1b) and the lowest-
 * energy state kept per replica (Table 3, state 5).
 *
 * Random numbers: Philox4x32-10 keyed by the 64-bit seed, counter
 * (spin j, replica r, draw d, instance id); words 0-1 give the initial position,
 * words 2-3 the momentum, each through the Box-Muller cosine branch on 24-bit
 * uniforms.  d = 0 is the initial draw, d = t the refresh before iteration t.
 *
 * Conventions for every call:
 *  - Return value: PHIA_OK (0) or a negative PHIA_E* code; no exception or
 *    abort crosses this boundary.  phia_last_error() returns a thread-local
 *    message for the last failing call of the calling thread.
 *  - "host" pointers are ordinary CPU memory owned by the caller; the library
 *    copies from / to them and keeps no reference after the call returns.
 *    "device" pointers are CUDA global memory on the handle's device, owned by
 *    the caller, and must stay valid until the work enqueued on the handle's
 *    stream has finished (phia_sync).
 *  - A handle owns all device memory it allocates; phia_destroy frees it.  A
 *    dense handle's buffers come from a stream-ordered memory pool per device that
 *    the library keeps for the process: freed blocks serve later handles without
 *    new allocations, so the process keeps its peak handle memory reserved.
 *    Handles are not thread-safe: one thread at a time per handle.
 *  - Work is enqueued on the stream given in phia_opts (NULL = the CUDA legacy
 *    default stream).  Calls that return results to host memory synchronise
 *    that stream.
 */
#ifndef PHIA_H
#define PHIA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PHIA_OK 0
#define PHIA_EINVAL (-1)   /* bad argument: N < 1, asymmetric J, nonzero diagonal, bad CSR */
#define PHIA_ERANGE (-2)   /* a value out of range for the chosen path or operand format */
#define PHIA_ENOMEM (-3)   /* device or host allocation failed */
#define PHIA_ETIMEOUT (-4) /* a bounded device-side wait expired; the context stays usable */
#define PHIA_ECUDA (-5)    /* a CUDA runtime call failed */
#define PHIA_ESTATE (-6)   /* call out of order (e.g. phia_best before any run) */
#define PHIA_ENOTSUP (-7)  /* the requested path does not handle this instance */

/* Field path (how I = J s + h is computed; every path gives the same exact integers). */
#define PHIA_PATH_AUTO 0   /* dense -> PHIA_PATH_TC, CSR -> PHIA_PATH_CSR */
#define PHIA_PATH_TC 1     /* tcgen05 tensor-core MMA, FP32 accumulation of integer products */
#define PHIA_PATH_FP32 2   /* plain FP32 CUDA-core mat-vec, one launch per step (comparator) */
#define PHIA_PATH_CSR 3    /* warp-per-row CSR gather over bit-packed spins */

/* Tensor-core operand encoding of the int8 couplings (exact re-encodings of k). */
#define PHIA_OP_AUTO 0     /* E4M3 when every |k| <= 16, else BF16 */
#define PHIA_OP_E4M3 1     /* FP8 e4m3, exact for |k| <= 16 */
#define PHIA_OP_BF16 2     /* BF16, exact for every int8 k */
#define PHIA_PEAK_S8_MMA_SYNC 3   /* phia_mma_peak only: warp-level int8 mma.sync (the int8 kernel's route) */

typedef struct phia_opts {
    int32_t path;          /* PHIA_PATH_* */
    int32_t operand;       /* PHIA_OP_* (tensor-core path only) */
    int32_t device;        /* CUDA device ordinal */
    uint32_t instance_id;  /* fourth Philox counter word: separates instances sharing a seed */
    void *stream;          /* cudaStream_t to enqueue on; NULL = legacy default stream */
    int32_t tile_replicas; /* tensor-core path: replicas per CTA, 4, 8 or 16; 0 = automatic */
    int32_t coupling_mem;  /* tensor-core path, where J stays during a run: 1 = shared memory,
                              2 = tensor memory; 0 = automatic */
    int32_t tc_kernel;     /* tensor-core path: 1 = resident tcgen05 kernel (all iterations in one
                              launch, J on chip; N <= 384 e4m3 / 256 bf16), 2 = one launch per
                              iteration (J streamed by TMA; any N), 3 = resident int8 kernel
                              (warp-level mma.sync s8 x s8 -> s32, J in registers; N <= 256;
                              tile_replicas 8 or 16), 4 = resident incremental-field kernel
                              (CUDA cores: the exact integer field is updated by the columns of
                              the spins that changed sign, Eq. 6 being linear in s; N <= 384
                              e4m3 / 256 bf16; tile_replicas 4, 8 or 16); 0 = automatic */
    int32_t large_variant; /* per-iteration kernel (tc_kernel 2): 1 = x, v staged through a shared-
                              memory ring (3 operand stages at 256-wide tiles); 2 = x, v
                              prefetched into registers (4 stages); 3 / 4 = as 2, with the CTAs of
                              a cluster of 2 / 4 sharing each replica tile and multicasting the
                              spin operand to one another (TMA multicast); 5 / 6 = as 1 with the
                              multicast over 2 / 4 CTAs; 7 = overlapped: the whole run in one
                              cooperative launch whose CTAs keep their output tiles for every
                              iteration and start a replica tile's next iteration as soon as
                              all of its spins are written (per-replica-tile counters instead
                              of a launch boundary; a records warp settles the energies); its
                              CTAs wait on each other, so it wants the GPU's SMs to itself;
                              its tile width (256, 224, 160 or 128 replicas; 160-wide tiles
                              with three tensor-memory accumulators) is the one whose
                              estimated iteration time is least; 8 / 9 = as 7 with 256- or
                              128-wide tiles and the spin-operand multicast over clusters of
                              2 / 4 CTAs; 10 / 11 / 12 / 13 = as 7 with 256- / 224- / 128- /
                              160-wide tiles; 0 = automatic (the autotuner's choice where it
                              has one; a choice of 7..13 is kept by the tuned handle only,
                              other handles take the fastest of 1..6) */
} phia_opts;

/* Annealing schedule.  No values are given in the paper; every field is explicit. */
typedef struct phia_schedule {
    float beta0;           /* inverse temperature at iteration 0 */
    float beta1;           /* inverse temperature at the last iteration (linear in between) */
    float eps;             /* step size of Eq. A7 */
    float gamma;           /* tanh sharpness of Eqs. 7-8 */
    int32_t refresh;       /* momentum redrawn before iteration t when t % refresh == 0, t > 0;
                              0 = drawn only at the start */
    int32_t has_target;    /* 1: record the first iteration with E <= target_k */
    int32_t stop_at_target;/* 1: freeze a replica's result at its first hit; the resident
                              kernels also end the run once every replica has passed the
                              earliest hit, the per-iteration paths run all their iterations */
    int32_t deriv;         /* derivative factor of Eq. 8 in the momentum update: 0 = exact,
                              1 - tanh^2(gamma x); 1 = quadratic stand-in max(0, 1 - (gamma x /
                              1.5)^2), after the FPGA's quadratic fit (Sec. 2.2), coefficients
                              chosen here (value 1 at 0 and integral 2, as the exact factor);
                              anything else is PHIA_EINVAL */
    int64_t target_k;      /* target energy in units of q */
    int32_t accept_test;   /* Table 3 state 4: 0 = every trajectory kept (App. A: exact HMC
                              accepts with probability 1); 1 = Metropolis test on the
                              Hamiltonian H = beta E(sgn x) + x.x/2 + v.v/2 (Eq. 4, Eq. A6)
                              at each trajectory end: just before the momentum draw of
                              iteration t (t % refresh == 0, t > 0), the trajectory
                              [t - refresh, t) is accepted when u <= exp(-(H_end - H_start)),
                              both H under beta_{t-1}, u the uniform of Philox counter
                              (0xFFFFFFFF, replica, t, instance id) word 0; a rejected end
                              point puts x back to the trajectory's start (the states it
                              visited still count for the best state).  A call's first
                              trajectory starts from a state whose energy no iteration of the
                              call evaluated and is kept untested; the last has no test (no
                              draw follows it).  Needs refresh > 0 to have any effect.
                              Resident tcgen05 kernel (tc_kernel 1, J in shared memory) and
                              the FP32 path only; elsewhere PHIA_ENOTSUP.  Counts:
                              phia_acceptance. */
    int32_t reserved;      /* must be 0 */
} phia_schedule;

typedef struct phia_stats {
    int64_t replicas;      /* replicas of the last run */
    int64_t steps;         /* iterations requested (field evaluations per replica) */
    int64_t spin_updates;  /* replicas * N * iterations actually run */
    int64_t best_energy_k; /* lowest energy over replicas (units of q) */
    int64_t best_replica;  /* replica holding it (ties: earliest step, then lowest index) */
    int64_t best_step;     /* iteration at which it was first seen */
    int64_t hit_step;      /* earliest iteration with E <= target over replicas, or -1 */
    int64_t hit_replica;   /* lowest replica index hitting at hit_step, or -1 */
    float device_ms;       /* device time of the last run, CUDA events on the handle's stream */
    int32_t path;          /* path actually used (PHIA_PATH_TC / _FP32 / _CSR) */
    int32_t operand;       /* operand actually used (PHIA_OP_E4M3 / _BF16), 0 for other paths */
    int32_t kernel_launches; /* kernels launched by the last run */
    int32_t tc_kernel;     /* dense kernel used (1 resident tcgen05, 2 per iteration, 3 resident
                              int8 mma.sync, 4 resident incremental field), 0 for other paths */
    int32_t reserved0;     /* 0 */
    int64_t hit_ns;        /* device time to target: %globaltimer nanoseconds from the start of
                              the run (its record reset, the first call of a resumed run) to
                              the recording of hit_step for hit_replica, or -1.  The resident
                              kernels record a hit in the iteration itself; the per-iteration
                              paths settle records one launch later (Table 3, state 5). */
} phia_stats;

typedef struct phia_s phia_t;

/* Create a dense instance (Eq. 2).  J_k: host, N*N int8 row-major, must be
 * symmetric with a zero diagonal (Eq. 2 sums i<j; a diagonal term has no place in
 * Eq. 6) -> PHIA_EINVAL otherwise.  h_k: host, N int32 with |h_k| < 2^24.
 * frac_bits f in [0, 30].  opts may be NULL (all defaults = 0).  Copies J and h to
 * the device; the caller keeps its buffers. */
int phia_create(phia_t **out, const int8_t *J_k, const int32_t *h_k, int32_t N,
                int32_t frac_bits, const phia_opts *opts);

/* Create a dense instance from device memory (for example PyTorch tensors): J_k, N*N
 * int8 row-major, and h_k, N int32, both on opts->device (device or managed memory).
 * Same requirements, errors, options and ownership as phia_create: the checks
 * (symmetry, zero diagonal, |h_k| < 2^24, max |k| for the operand) run on the device,
 * ordered after the caller's work on opts->stream; J and h are copied device to device
 * into the handle's buffers; the caller keeps its buffers.  Host pointers, or buffers on
 * another device -> PHIA_EINVAL. */
int phia_create_from_device(phia_t **out, const int8_t *J_k, const int32_t *h_k, int32_t N,
                            int32_t frac_bits, const phia_opts *opts);

/* Create a sparse instance in CSR form (host arrays): row_ptr[N+1], col[nnz]
 * (0 <= col < N, no self loops), val_k[nnz] int8; the pattern and values must be
 * symmetric.  Stored zeros are allowed.  Runs on the CSR path (a batch of one); its
 * replicas run in groups of 256, smaller counts padded with unreported replicas.  One
 * launch per iteration (opts->tc_kernel = 1: one persistent launch for the run instead;
 * that cooperative launch assumes no other persistent launch runs on the device at the
 * same time, and reports PHIA_ETIMEOUT rather than waiting without end if one does). */
int phia_create_csr(phia_t **out, const int32_t *row_ptr, const int32_t *col,
                    const int8_t *val_k, const int32_t *h_k, int32_t N, int32_t frac_bits,
                    const phia_opts *opts);

/* Run `replicas` independent replicas for `steps` iterations (Eqs. A7-A8) from the
 * Philox initial draw (positions ~ g(x) of Eq. A3, momenta ~ N(0,1)), keeping the
 * best state per replica.  Enqueued on the handle's stream; returns before the
 * device finishes.  replicas >= 1, steps >= 1. */
int phia_anneal(phia_t *p, const phia_schedule *sched, int32_t replicas, int64_t steps,
                uint64_t seed);

/* Autotuner.  Times short probe runs (probe_iters iterations of `replicas` replicas) of
 * every tensor-core kernel variant that applies to this handle -- the resident tcgen05
 * kernel with 4, 8 or 16 replicas per CTA and J in shared or tensor memory, the
 * resident int8 mma.sync kernel with 8 or 16 replicas per CTA (N small enough), the
 * resident incremental-field kernel with 4, 8 or 16 replicas per CTA (N small enough),
 * and the per-iteration kernel in its thirteen variants (phia_opts.large_variant) -- keeps
 * the fastest for the handle and caches it,
 * process-wide, for (N, replicas, operand): handles created with all variant options
 * automatic use the cached choice for runs with that replica count.  The probes
 * overwrite the handle's last-run records.  Tensor-core path only (else PHIA_ENOTSUP). */
typedef struct phia_tune_result {
    int32_t tc_kernel;         /* 1 resident tcgen05, 2 per iteration, 3 resident int8 mma.sync,
                                  4 resident incremental field; the per-iteration kernel's variant
                                  (phia_opts.large_variant) is reported in large_variant */
    int32_t tile_replicas;     /* resident kernel: replicas per CTA */
    int32_t coupling_mem;      /* resident kernel: 1 shared, 2 tensor memory */
    int32_t candidates;        /* variants timed */
    float best_us_per_iter;    /* device time per iteration of the chosen variant */
    float worst_us_per_iter;   /* of the slowest variant */
    int32_t large_variant;     /* per-iteration kernel: the variant chosen (1..13), 0 otherwise */
    int32_t reserved;          /* 0 */
} phia_tune_result;

int phia_autotune(phia_t *p, const phia_schedule *sched, int32_t replicas, int32_t probe_iters,
                  phia_tune_result *out);

/* Lowest energy found by the last run (ties: earliest step, then lowest replica)
 * and its spins.  energy_k: host int64 (units of q).  spins: host, N int8 in
 * {-1,+1}, may be NULL.  Synchronises the stream.  PHIA_ETIMEOUT if a bounded
 * device wait expired during the run. */
int phia_best(phia_t *p, int64_t *energy_k, int8_t *spins);

/* Statistics of the last run (synchronises the stream). */
int phia_stats_get(phia_t *p, phia_stats *out);

/* Per-replica results of the last run, host arrays of `replicas` entries (any may
 * be NULL): best energy (units of q), iteration of the best, first iteration with
 * E <= target (-1 if none), and the best spins bit-packed: replicas x ceil(N/32)
 * uint32 words, bit (i % 32) of word (i / 32) set when s_i = +1. */
int phia_replica_results(phia_t *p, int32_t replicas, int64_t *best_energy_k,
                         int64_t *best_step, int64_t *hit_step, uint32_t *best_bits);

/* ---------------------------------------------------------------- vanilla GAHMC
 * The exact dynamics of H(x, v) = beta E(sgn x) + x.x/2 + v.v/2 (Eq. 4, App. A) solved by
 * zero crossings -- the Gaussian-augmented HMC of the paper's reference [Pakman &
 * Paninski 2013] that Sec. 2.1 names as the exact alternative to PHIA's approximate
 * gradient and Sec. 3.2 uses as an ablation.  Inside an orthant every coordinate rotates
 * on the unit circle (x cos t + v sin t); where x_j reaches 0 the spin flips if the
 * kinetic energy of that coordinate pays the energy step beta q dE, dE = 2 s_j I_j
 * (speed reduced to sqrt(A^2 - 2 beta q dE)), else it is reflected.  With a travel time
 * <= pi each spin meets its wall at most once per trajectory; events are taken in time
 * order (ties: lower spin index first).  Replicas are independent (one warp each).
 * Random numbers as phia_anneal: the initial draw d = 0, the momentum of trajectory
 * k > 0 from draw d = k. */
typedef struct phia_gahmc_schedule {
    float beta0;           /* inverse temperature of the first trajectory */
    float beta1;           /* of the last (linear in between) */
    float travel;          /* time per trajectory, 0 < travel <= pi */
    int32_t has_target;    /* 1: record the first trajectory whose states reach E <= target_k */
    int64_t target_k;      /* units of q */
} phia_gahmc_schedule;

/* Run `trajectories` GAHMC trajectories for `replicas` replicas of a dense handle
 * (N <= 1024; any dense path -- it reads the stored int8 couplings).  x, v: device
 * [replicas][N] float32 or NULL: on entry the initial state (NULL: the Philox draw d = 0),
 * on return the final state.  counts: device [replicas][2] int64 (crossings, reflections)
 * or NULL.  events: device [replicas][events_cap] int32 or NULL: the first events_cap wall
 * events of each replica in order, j for a crossing of spin j and -(j + 1) for a
 * reflection; entries past a replica's events are left untouched.  The per-replica
 * records (phia_best, phia_replica_results, phia_stats_get) hold the best energy over
 * every visited state (the initial one and one per crossing), with best_step and
 * hit_step counted in trajectories (0 = already in the initial state or trajectory 0);
 * spin_updates counts N per replica and trajectory.  Asynchronous.  PHIA_ENOTSUP for a
 * CSR handle or N > 1024; PHIA_EINVAL for travel outside (0, pi], negative beta or
 * trajectories < 1. */
int phia_gahmc(phia_t *p, const phia_gahmc_schedule *sched, int32_t replicas, int64_t trajectories,
               uint64_t seed, float *x, float *v, int64_t *counts, int32_t *events, int32_t events_cap);

/* Acceptance counts of the last run with accept_test = 1 (Table 3, state 4: the
 * acceptance rate is accepted / proposed), host arrays of `replicas` entries (either may
 * be NULL): trajectories put to the test and accepted, per replica.  Zero after a run
 * without the test.  Synchronises the stream. */
int phia_acceptance(phia_t *p, int32_t replicas, int64_t *proposed, int64_t *accepted);

/* Resumable form of phia_anneal.  Runs iterations t0 .. t0+steps-1 of a run of
 * total_steps iterations (beta_t and the refresh draws depend on the absolute t)
 * from the state in x, v (device, replicas x N float32 row-major, updated in place
 * to the state after the last iteration).  reset_best = 1 starts the per-replica
 * best/target record afresh; 0 continues the record of the previous call with the
 * same replica count.  Running [0,a) then [a,b) gives bit-identical states and
 * records to running [0,b) at once. */
int phia_run(phia_t *p, const phia_schedule *sched, int32_t replicas, int64_t t0,
             int64_t steps, int64_t total_steps, uint64_t seed, float *x, float *v,
             int32_t reset_best);

/* The initial draw of phia_anneal written to device arrays x, v (replicas x N). */
int phia_init_state(phia_t *p, int32_t replicas, uint64_t seed, float *x, float *v);

/* Field (Eq. 6) and energy (Eq. 2, through E = -1/2 sum s (I + h)) of given spins on
 * the handle's field path.  spins: device, replicas x N int8 in {-1,+1};
 * field_k: device, replicas x N int32 (units of q); energy_k: device, replicas
 * int64 (units of q).  Either output may be NULL. */
int phia_field(phia_t *p, const int8_t *spins, int32_t replicas, int32_t *field_k,
               int64_t *energy_k);

/* The library's device Philox draws, for testing: for replica r < replicas,
 * spin j < N: raw[(r*N + j)*4 + w] = Philox4x32-10 word w of counter
 * (j, r, d, instance_id) and key (seed lo, seed hi); x[r*N+j], v[r*N+j] the two
 * Box-Muller normals.  All device pointers (any may be NULL); stream may be NULL. */
int phia_philox_draws(uint64_t seed, uint32_t instance_id, uint32_t d, int32_t replicas,
                      int32_t N, uint32_t *raw, float *x, float *v, void *stream);

/* Run without allocating: the paper has no counterpart to this entry point; it exists
 * for callers that cannot allocate device memory.  Some programs hand the whole device
 * to their own memory pool at start-up, so a cudaMalloc from a library would fail or
 * break the pool's accounting; others run a latency-critical loop in which cudaMalloc
 * and cudaFree are forbidden because they can synchronise the device and take unbounded
 * time.  Such callers own every input and output buffer, and this call takes its
 * scratch (the operand copy of J, the spin buffers, the energy sums, a working copy of
 * x and v, its counters) from one array of 64 MiB compiled into the library.
 *
 * When that array is reserved: with CUDA's lazy module loading (the default), a device
 * reserves the array's 64 MiB when the library's code is first used on it -- in practice
 * at the first call of this entry point on that device, which also looks up the array's
 * device address (cudaGetSymbolAddress) -- and holds it until the process exits.  Make
 * that first call at start-up, before the caller's own pool claims the device's memory
 * and before any stream capture begins on that device.  Later calls reserve nothing
 * more.
 *
 * It runs the tensor-core path with one launch per iteration, exactly as phia_run does
 * on a handle created with tc_kernel = 2, and gives the same results.  All pointers are
 * device memory on the current CUDA device except sched (host): J_k N*N int8, h_k N
 * int32, x and v replicas*N float32 updated in place, and the records best_energy_k,
 * best_step, hit_step (replicas each) and best_bits (replicas * ceil(N/32)), which
 * reset_best = 1 initialises.  J_k and h_k are checked on the device as phia_create
 * checks them: asymmetric J or a nonzero diagonal -> PHIA_EINVAL, |h_k| >= 2^24 ->
 * PHIA_ERANGE.  operand: PHIA_OP_E4M3 (needs every |k| <= 16, else PHIA_ERANGE),
 * PHIA_OP_BF16, or PHIA_OP_AUTO (e4m3 when every |k| <= 16, else bf16, as phia_create).
 * stream: cudaStream_t or NULL.  Sizes that need more scratch than the array holds
 * return PHIA_ERANGE with the largest replica count that fits for that N and operand
 * (for example N = 2000 with e4m3 fits at most 2304 replicas).  The call allocates
 * nothing: no cudaMalloc, cudaFree or allocating library routine.  It synchronises the
 * stream (once after the instance checks, once at the end) and returns after the work
 * has finished, with PHIA_ETIMEOUT if a bounded device wait expired.  All calls share the
 * one array, whose contents the next call overwrites (the call clears what must start at
 * zero): calls that overlap on the GPU (other threads, other streams) race and must be
 * serialised by the caller. */
int phia_run_noalloc(const int8_t *J_k, const int32_t *h_k, int32_t N, int32_t frac_bits, int32_t operand,
                     const phia_schedule *sched, int32_t replicas, int64_t t0, int64_t steps,
                     int64_t total_steps, uint64_t seed, uint32_t instance_id, float *x, float *v,
                     int64_t *best_energy_k, int64_t *best_step, int64_t *hit_step, uint32_t *best_bits,
                     int32_t reset_best, void *stream);

/* ---------------------------------------------------------------- batches
 * Many independent instances of uneven N annealed together.  Dense descriptors with
 * N <= 384 and every |k| <= 16, or N <= 256, run on the resident tcgen05 kernel over a
 * table of CTAs (8 replicas each): every such instance, all iterations, one launch per
 * (operand, number of 128-spin tiles) group.  The other instances run on the sparse CSR
 * path (larger dense descriptors converted to CSR): by default one persistent cooperative
 * launch covers every iteration of every CSR instance (blocks take 64-row x 256-replica
 * work units from a counter, the grid meets at a bounded barrier between iterations);
 * phia_opts.tc_kernel = 2 at creation gives one launch per iteration instead (replayed as
 * CUDA graphs), and phia_batch_autotune picks the faster.  Each instance keeps its own
 * couplings, replicas, records and Philox instance id, so its result does not depend on
 * the rest of the batch or on the path, and equals the same instance run alone on that
 * path. */
typedef struct phia_instance_desc {
    int32_t N;                 /* spins */
    int32_t frac_bits;         /* J = k 2^-f, h = kh 2^-f */
    const int8_t *J_k;         /* host, dense N*N (symmetric, zero diagonal), or NULL for CSR */
    const int32_t *row_ptr;    /* host CSR (used when J_k is NULL): row_ptr[N+1], col, val_k */
    const int32_t *col;
    const int8_t *val_k;
    const int32_t *h_k;        /* host, N int32, |h_k| < 2^24 */
    uint32_t instance_id;      /* Philox counter word of this instance */
    int32_t has_target;        /* 1: this instance's own target energy (units of q) */
    int64_t target_k;
} phia_instance_desc;

typedef struct phia_batch_s phia_batch_t;

/* Validate and upload `count` instances (copied; the caller keeps its arrays).  opts
 * may be NULL; opts->path must be PHIA_PATH_AUTO or PHIA_PATH_CSR; opts->tc_kernel: 0 or
 * 1 = the CSR instances in one persistent launch, 2 = one launch per iteration. */
int phia_batch_create(phia_batch_t **out, int32_t count, const phia_instance_desc *descs,
                      const phia_opts *opts);

/* Anneal `replicas` replicas of every instance for `steps` iterations (as phia_anneal
 * per instance).  The sparse path runs replicas in groups of 256; other counts are
 * padded with extra replicas that are run but never reported.  Asynchronous. */
int phia_batch_anneal(phia_batch_t *b, const phia_schedule *sched, int32_t replicas, int64_t steps,
                      uint64_t seed);

/* Best state of one instance (as phia_best). */
int phia_batch_best(phia_batch_t *b, int32_t instance, int64_t *energy_k, int8_t *spins);

/* Per-replica records of one instance (as phia_replica_results). */
int phia_batch_replica_results(phia_batch_t *b, int32_t instance, int32_t replicas,
                               int64_t *best_energy_k, int64_t *best_step, int64_t *hit_step,
                               uint32_t *best_bits);

/* Autotuner of a batch: times probe runs (probe_iters iterations, `replicas` replicas per
 * instance) of the CSR instances in one persistent launch and in one launch per
 * iteration, keeps the faster for the batch; out->tc_kernel reports it (1 persistent,
 * 2 per iteration) with the times per iteration.  The probes overwrite the records. */
int phia_batch_autotune(phia_batch_t *b, const phia_schedule *sched, int32_t replicas, int32_t probe_iters,
                        phia_tune_result *out);

/* Statistics of the last batch run: spin_updates counts every instance; the best and
 * hit fields describe instance 0. */
int phia_batch_stats_get(phia_batch_t *b, phia_stats *out);

int phia_batch_sync(phia_batch_t *b);
void phia_batch_destroy(phia_batch_t *b);

/* ---------------------------------------------------------------- serving
 * A request loop with continuous batching.  Requests (an instance, a schedule, a replica
 * count, a step cap, a seed, a target energy) are queued on submission and admitted in
 * arrival order as soon as one of max_inflight slots and enough of the device-memory
 * budget are free; while some run, later arrivals are admitted into freed slots.  Each
 * admitted request keeps its couplings and replica state on the device and runs in
 * chunks of chunk_iters iterations on its slot's own stream, so requests overlap on the
 * GPU; it ends when a chunk shows its target reached (stop at target) or the step cap
 * spent.  A request's result depends only on the request, not on the slot or the mix.
 * Dense instances run on the tensor-core path, CSR instances on the CSR path.  The
 * server is thread-safe: submit and poll from any thread. */
typedef struct phia_server_opts {
    int32_t device;
    int32_t max_inflight;      /* slots (1..256), one CUDA stream each */
    int64_t hbm_budget_bytes;  /* device memory the admitted requests may hold together */
    int32_t chunk_iters;       /* iterations per launch chunk (target checked in between) */
    int32_t path;              /* PHIA_PATH_AUTO (dense: tensor core, CSR: CSR path) or
                                  PHIA_PATH_FP32 (every request on the plain FP32 path) */
} phia_server_opts;

typedef struct phia_request_status {
    int32_t state;             /* 0 queued, 1 running, 2 done, < 0 a PHIA_E* code */
    int32_t hit;               /* 1: the target was reached */
    int64_t energy_k;          /* best energy (the earliest hit when the target was reached) */
    int64_t hit_step;          /* first iteration reaching the target, or -1 */
    int64_t steps_run;         /* iterations run */
    double t_submit_s;         /* times since server creation (steady clock), -1 if not yet */
    double t_admit_s;
    double t_done_s;
    int32_t path;              /* path that ran it */
    int32_t reserved;
} phia_request_status;

typedef struct phia_server_stats {
    int64_t completed;         /* requests done */
    int64_t hits;              /* requests that reached their target */
    int64_t spin_updates;      /* replicas * N * iterations over completed requests */
    double ttt_p50_s;          /* time to target from arrival (submit), over hits */
    double ttt_p99_s;
    double ttt_admit_p50_s;    /* time to target from admission, over hits */
    double ttt_admit_p99_s;
    double elapsed_s;          /* since server creation */
    int64_t used_bytes;        /* device memory currently held by admitted requests */
} phia_server_stats;

typedef struct phia_server_s phia_server_t;

int phia_server_create(phia_server_t **out, const phia_server_opts *opts);

/* Queue a request (the instance is copied; the caller keeps its arrays).  The
 * instance's has_target/target_k, when set, override the schedule's target; stop at
 * target is always on.  Returns its id in *request_id.  PHIA_ENOMEM if the request
 * alone needs more than the whole budget. */
int phia_server_submit(phia_server_t *s, const phia_instance_desc *inst, const phia_schedule *sched,
                       int32_t replicas, int64_t step_cap, uint64_t seed, int64_t *request_id);

/* Status of a request; spins (host, N int8, may be NULL) receive the best state once done. */
int phia_server_poll(phia_server_t *s, int64_t request_id, phia_request_status *status, int8_t *spins);

/* Block until every submitted request is done (PHIA_ETIMEOUT after timeout_ms). */
int phia_server_wait_all(phia_server_t *s, int64_t timeout_ms);

int phia_server_stats_get(phia_server_t *s, phia_server_stats *out);

/* Stop the loop, free every request's device memory and the streams. */
void phia_server_destroy(phia_server_t *s);

/* Measurement aid (no counterpart in the paper): dense tensor-core throughput of the
 * current device for the operand encodings of the field (Eq. 6), so that its roofline
 * has a denominator measured for its own operand type.  One CTA per SM issues
 * rounds x 4 tcgen05 MMAs of shape M = 128, N = n (16..256, a multiple of 16), K = one
 * 128-byte swizzle row split in four (e4m3: K = 32 per MMA, kind::f8f6f4; bf16: K = 16,
 * kind::f16) from shared memory into one FP32 tensor-memory accumulator.  operand:
 * PHIA_OP_E4M3 or PHIA_OP_BF16; or PHIA_PEAK_S8_MMA_SYNC: 32 warps per SM, each issuing
 * rounds x 8 warp-level mma.sync m16n8k32 s8 x s8 -> s32 into eight independent register
 * accumulators (n is then ignored; 2 * 16 * 8 * 32 integer ops per MMA).  stream:
 * cudaStream_t or NULL.  Writes the device time of the timed launch (after one warm-up
 * launch; CUDA events) to *ms and the achieved dense rate (flops or integer ops per
 * second, x 1e-12) to *tflops (host pointers, either may be NULL).  Allocates a 4-byte
 * status word; synchronises the stream. */
int phia_mma_peak(int32_t operand, int32_t n, int64_t rounds, void *stream, float *ms, double *tflops);

/* Testing aid for the error path of bounded device waits (Sec. 2.2 gives the FPGA's
 * fixed schedule and no error handling; this entry point has no counterpart in the
 * paper).  Every device-side wait of the library's kernels gives up after a time bound,
 * records the fact and lets the kernel return, so that a lost arrival cannot hang the
 * GPU; later calls that return results then fail with PHIA_ETIMEOUT and the CUDA context
 * stays usable.  wait_budget_ns sets that bound for the per-iteration tensor-core kernel
 * of this handle (0 = the library default of 2 s).  stall_producer = 1, allowed only on a
 * handle created with tc_kernel = 2, makes that kernel's TMA producer issue no copy at all:
 * no tensor-core or copy operation is then ever in flight, every wait for a full operand
 * stage or a finished accumulator runs out after the bound, and the run reports
 * PHIA_ETIMEOUT.  stall_producer = 0 restores normal runs.  Settings stay on the handle
 * until changed.  PHIA_EINVAL for a negative bound or a stall flag other than 0/1,
 * PHIA_ENOTSUP for a stall on any other kernel. */
int phia_debug_wait(phia_t *p, int64_t wait_budget_ns, int32_t stall_producer);

/* Wait for all work enqueued on the handle's stream. */
int phia_sync(phia_t *p);

/* Free every resource of the handle (NULL is allowed). */
void phia_destroy(phia_t *p);

/* Message for the last failing call on this thread ("" if none). */
const char *phia_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PHIA_H */
