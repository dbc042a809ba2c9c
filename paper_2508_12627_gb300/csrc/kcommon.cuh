// Device helpers shared by the engine's kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ustat {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum of v over the block, returned by thread 0 (blockDim.x * blockDim.y <= 1024).
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[32];
    const int tid = threadIdx.x + threadIdx.y * blockDim.x + threadIdx.z * blockDim.x * blockDim.y;
    const int nthr = blockDim.x * blockDim.y * blockDim.z;
    v = warp_sum(v);
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    double r = 0.0;
    if (tid < 32) {
        r = (tid < (nthr + 31) / 32) ? red[tid] : 0.0;
        r = warp_sum(r);
    }
    return r;
}

template <typename T>
__device__ __forceinline__ T ld_term(const T *M, int trans, int64_t n, int64_t i, int64_t j) {
    return trans ? M[j * n + i] : M[i * n + j];
}

}  // namespace ustat
