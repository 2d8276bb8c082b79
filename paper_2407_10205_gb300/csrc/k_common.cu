// k_common.cu -- small kernels shared by every path: the Philox draws exposed for
// testing and the initial state (position and momentum draws, Sec. 2.1 and Eq. A3).
#include <cuda_bf16.h>
#include <cuda_fp8.h>

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

// Couplings k -> exact operand encoding (e4m3 byte or bf16), zero-padded to
// [Mpad rows][Kbytes], row-major (K contiguous).
__global__ void convert_operand_kernel(const int8_t *Jk, int N, uint8_t *Jop, int Mpad, int Kbytes, int op) {
    const int esz = op == kOpE4M3 ? 1 : 2;
    const int Kel = Kbytes / esz;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)Mpad * Kel) return;
    const int row = (int)(idx / Kel), col = (int)(idx - (int64_t)row * Kel);
    const float v = (row < N && col < N) ? (float)Jk[(size_t)row * N + col] : 0.0f;
    if (op == kOpE4M3) Jop[idx] = __nv_fp8_e4m3(v).__x;
    else reinterpret_cast<uint16_t *>(Jop)[idx] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
}

// Instance checks on the device: res[0] = lowest linear index i*N + j (i < j) with
// k_ij != k_ji, res[1] = lowest i with k_ii != 0, res[2] = lowest i with |kh_i| >= 2^24
// (each left untouched where there is none), res[3] = max |k_ij| over i < j (atomic max).
__global__ void check_dense_kernel(const int8_t *J, const int32_t *h, int N, unsigned long long *res) {
    const int64_t total = (int64_t)N * N;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t first = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned int mx = 0;
    for (int64_t e = first; e < total; e += stride) {
        const int i = (int)(e / N), j = (int)(e - (int64_t)i * N);
        const int k = J[e];
        if (j > i) {
            if (k != J[(int64_t)j * N + i]) atomicMin(&res[0], (unsigned long long)e);
            mx = max(mx, (unsigned int)abs(k));
        } else if (j == i && k != 0) {
            atomicMin(&res[1], (unsigned long long)i);
        }
    }
    mx = __reduce_max_sync(0xffffffffu, mx);
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(&res[3], (unsigned long long)mx);
    for (int64_t i = first; i < N; i += stride)
        if (h[i] >= (1 << 24) || h[i] <= -(1 << 24)) atomicMin(&res[2], (unsigned long long)i);
}

}  // namespace

cudaError_t launch_check_dense(const int8_t *J, const int32_t *h, int N, unsigned long long *res, unsigned blocks,
                               cudaStream_t st) {
    check_dense_kernel<<<blocks, 256, 0, st>>>(J, h, N, res);
    return cudaGetLastError();
}

cudaError_t launch_convert_operand(const int8_t *Jk, int N, void *Jop, int Mpad, int Kbytes, int op, cudaStream_t st) {
    const int esz = op == kOpE4M3 ? 1 : 2;
    const int64_t n = (int64_t)Mpad * (Kbytes / esz);
    convert_operand_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(Jk, N, (uint8_t *)Jop, Mpad, Kbytes, op);
    return cudaGetLastError();
}

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
