// phia_internal.h -- declarations shared by the library's translation units (not part
// of the public ABI; see include/phia.h for that).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace phia {

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
    uint32_t *best_bits;        // [R][W]
    int32_t W;
    int32_t has_target, stop_at_target;
    int64_t target;
    unsigned long long *min_hit;         // earliest hit over replicas (stop-at-target)
    unsigned long long *replica_iters;   // sum over replicas of iterations run
    int32_t *err;                        // nonzero: a bounded device wait expired
    int32_t tile_rl;                     // tensor-core small path: live replicas per CTA (0 = auto)
    int32_t coupling_mem;                // tensor-core small path: 1 = J in shared, 2 = in tensor memory
};

constexpr uint64_t kWaitTimeoutNs = 2000000000ull;  // 2 s bound on every device-side wait
constexpr int kOpE4M3 = 1;
constexpr int kOpBF16 = 2;

// tcgen05 persistent kernel for small dense instances (J resident in shared memory).
int tc_small_max_n(int op);
int tc_small_tile_replicas(int R, int requested);
cudaError_t launch_tc_small(const RunArgs &a, int op, cudaStream_t st, int *launches);

// tcgen05 per-iteration kernel for dense instances of any size (TMA-staged J and spins).
struct LargeBuffers {
    const void *Jop;      // [Mpad][Kbytes] couplings in the operand encoding
    uint8_t *S;           // [4][Rpad][Kbytes] spin operand buffers (zero padding)
    int64_t *Epart;       // [2][Rpad], zero between uses
    int8_t *flags;        // [2][Rpad]
    float *X, *V;         // [R][N] state when the caller gives none
    int32_t Kbytes, Mpad, Rpad;
};
cudaError_t launch_tc_large(const LargeBuffers &B, const RunArgs &a, int op, cudaStream_t st, int *launches);
cudaError_t launch_convert_operand(const int8_t *Jk, int N, void *Jop, int Mpad, int Kbytes, int op, cudaStream_t st);
inline int large_kbytes(int N, int op) { return ((N * (op == kOpE4M3 ? 1 : 2)) + 127) / 128 * 128; }
inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Thread-local error message of the C ABI.
int set_last_error(int code, const char *msg);

// Plain FP32 per-step path (the comparator).
cudaError_t launch_fp32_run(const RunArgs &a, float *x, float *v, int8_t *s0, int8_t *s1,
                            int64_t *e_acc, cudaStream_t st, int *launches);

// Philox draws for testing.
cudaError_t launch_philox_draws(uint64_t seed, uint32_t inst, uint32_t d, int R, int N, uint32_t *raw,
                                float *x, float *v, cudaStream_t st);

// Initial state (Philox d = 0) into x, v.
cudaError_t launch_init_state(int R, int N, uint64_t seed, uint32_t inst, float *x, float *v,
                              cudaStream_t st);

}  // namespace phia
