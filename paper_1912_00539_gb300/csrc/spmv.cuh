// Row q of block row i of A times x, FP64: the SpMV's inner product, shared by
// the product kernel and the residual kernels so that every FP64 product of A
// runs the same FMA chain (blocks in order; within a block x_j[0..3]).  The
// first four blocks' loads are issued before any arithmetic, so each thread
// keeps up to 8 independent 16-byte loads in flight.
#pragma once
#include "common.cuh"

namespace abilu {

__device__ __forceinline__ double row_dot_blocks(const PatternView &P, const double *__restrict__ A,
                                                 const double *__restrict__ x, int i, int q) {
    const int p0 = P.rowptr[i], p1 = P.rowptr[i + 1];
    double2 a0[4], a1[4];
    int jj[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const int p = p0 + k;
        if (p < p1) {
            jj[k] = __ldg(P.colind + p);
            const double2 *ap = reinterpret_cast<const double2 *>(A + (size_t)p * BB + q * BS);
            a0[k] = __ldg(ap);
            a1[k] = __ldg(ap + 1);
        } else {
            jj[k] = -1;
        }
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        if (jj[k] >= 0) {
            const double2 *xp = reinterpret_cast<const double2 *>(x + (size_t)jj[k] * BS);
            double2 x0 = __ldg(xp), x1 = __ldg(xp + 1);
            s = fma(a0[k].x, x0.x, s);
            s = fma(a0[k].y, x0.y, s);
            s = fma(a1[k].x, x1.x, s);
            s = fma(a1[k].y, x1.y, s);
        }
    }
    for (int p = p0 + 4; p < p1; p++) {  // rows longer than four blocks
        const int j = __ldg(P.colind + p);
        const double2 *ap = reinterpret_cast<const double2 *>(A + (size_t)p * BB + q * BS);
        const double2 *xp = reinterpret_cast<const double2 *>(x + (size_t)j * BS);
        double2 b0 = __ldg(ap), b1 = __ldg(ap + 1), x0 = __ldg(xp), x1 = __ldg(xp + 1);
        s = fma(b0.x, x0.x, s);
        s = fma(b0.y, x0.y, s);
        s = fma(b1.x, x1.x, s);
        s = fma(b1.y, x1.y, s);
    }
    return s;
}

}  // namespace abilu
