// Deterministic block reductions shared by the FGMRES kernels.
#pragma once

#include "common.cuh"

namespace abilu {

constexpr int RED_THREADS = 256;
constexpr int RED_WARPS = RED_THREADS / 32;

// Block-wide sum of K values per thread; result in sh_out[k], k < kn (valid
// after the call's final barrier).  sh_w holds K * RED_THREADS doubles.  The
// values are staged in shared memory and warp k sums value k: each lane adds
// its 8 values (threads lane, lane + 32, ...) in order, then a 5-level
// shuffle tree.  A fixed order, so deterministic.  This GPU has two FP64 lanes
// per SM, so a warp-wide FP64 add occupies its FP64 pipe for 16 cycles
// whatever the lanes do: per value this form issues 12 warp-wide FP64 adds
// where a shuffle tree in every warp and a cross-warp stage issued 43-48,
// which was most of the gap between the dot kernels and their FMA floor.
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double *sh_w, double *sh_out, int kn) {
#pragma unroll
    for (int k = 0; k < K; k++) sh_w[k * RED_THREADS + threadIdx.x] = v[k];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int k = threadIdx.x >> 5; k < kn; k += RED_WARPS) {
        const double *p = sh_w + k * RED_THREADS + lane;
        double s = p[0];
#pragma unroll
        for (int r = 1; r < RED_WARPS; r++) s += p[32 * r];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) sh_out[k] = s;
    }
    __syncthreads();
}

}  // namespace abilu
