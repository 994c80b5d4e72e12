// Deterministic block reductions shared by the FGMRES kernels.
#pragma once

#include "common.cuh"

namespace abilu {

constexpr int RED_THREADS = 256;
constexpr int RED_WARPS = RED_THREADS / 32;

// block-wide sum of K values per thread; result in sh_out[k] (valid after sync)
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double *sh_w, double *sh_out, int kn) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; k++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; k++) sh_w[warp * K + k] = v[k];
    __syncthreads();
    if (threadIdx.x < kn) {
        double s = 0.0;
        for (int w = 0; w < RED_WARPS; w++) s += sh_w[w * K + threadIdx.x];
        sh_out[threadIdx.x] = s;
    }
    __syncthreads();
}

}  // namespace abilu
