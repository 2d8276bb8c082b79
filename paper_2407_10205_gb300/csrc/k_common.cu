// k_common.cu -- small kernels shared by every path: the Philox draws exposed for
// testing and the initial state (position and momentum draws, Sec. 2.1 and Eq. A3).
#include "device_common.cuh"
#include "phia_internal.h"

namespace phia {

namespace {

__global__ void philox_draws_kernel(uint64_t seed, uint32_t inst, uint32_t d, int R, int N, uint32_t *raw,
                                    float *x, float *v) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)R * N) return;
    const int r = (int)(idx / N), j = (int)(idx - (int64_t)r * N);
    const U4 o = draw_raw(seed, inst, (uint32_t)r, (uint32_t)j, d);
    if (raw) reinterpret_cast<uint4 *>(raw)[idx] = make_uint4(o.x, o.y, o.z, o.w);
    if (x) x[idx] = box_muller(o.x, o.y);
    if (v) v[idx] = box_muller(o.z, o.w);
}

}  // namespace

cudaError_t launch_philox_draws(uint64_t seed, uint32_t inst, uint32_t d, int R, int N, uint32_t *raw, float *x,
                                float *v, cudaStream_t st) {
    const int64_t n = (int64_t)R * N;
    if (n == 0) return cudaSuccess;
    philox_draws_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(seed, inst, d, R, N, raw, x, v);
    return cudaGetLastError();
}

cudaError_t launch_init_state(int R, int N, uint64_t seed, uint32_t inst, float *x, float *v, cudaStream_t st) {
    return launch_philox_draws(seed, inst, 0u, R, N, nullptr, x, v, st);
}

}  // namespace phia
