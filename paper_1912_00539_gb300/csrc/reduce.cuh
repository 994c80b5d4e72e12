// Deterministic block reductions shared by the FGMRES kernels.
#pragma once

#include "common.cuh"

namespace abilu {

constexpr int RED_THREADS = 256;
constexpr int RED_WARPS = RED_THREADS / 32;

// block-wide sum of K values per thread; result in sh_out[k], k < kn (valid after sync)
// TREE: the cross-warp stage as a shuffle tree (default for one or two values)
template <int K, bool TREE = (K <= 2)>
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
    if constexpr (TREE) {
        // warp k sums value k over the warps by a shuffle tree (log2 of the
        // warp count dependent adds, not one per warp: an FP64 add takes 64
        // cycles on this GPU)
        if (warp < kn) {
            double s = lane < RED_WARPS ? sh_w[lane * K + warp] : 0.0;
#pragma unroll
            for (int o = RED_WARPS / 2; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            if (lane == 0) sh_out[warp] = s;
        }
    } else {   // thread k adds the warps' sums in order (fewer registers)
        if (threadIdx.x < kn) {
            double s = 0.0;
            for (int w = 0; w < RED_WARPS; w++) s += sh_w[w * K + threadIdx.x];
            sh_out[threadIdx.x] = s;
        }
    }
    __syncthreads();
}

}  // namespace abilu
