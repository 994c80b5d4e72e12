// Diagnostics of a factorisation (Sec. 6.2): the ILU fixed-point residual
// ||x - h(x)||_1 (the paper plots its ratio to the initial one), the defect
// max |(LU)_ij - A_ij| over S_B, and the max-norms of the block-Jacobi iteration
// matrices of the triangular solves, ||L - I||_inf and
// ||D_U^{-1}(U - D_U)||_inf (the "diagonal dominance" of L and U).
//
// Evaluated in FP64 from the stored factors (whatever their dtype): one quad
// per block row, h(x) formed exactly as a synchronous sweep forms it, with
// inv(U_jj) recomputed from the stored U_jj.  A diagnostic, run once: the
// inverses are recomputed per use and the sums use atomics.
#include <string.h>

#include "common.cuh"

namespace abilu {

// inverse of the 4x4 block a (FP64 adjugate); singular -> identity
__device__ static void inv4_full(const double *a, double *r) {
    double s0 = a[0] * a[5] - a[4] * a[1], s1 = a[0] * a[6] - a[4] * a[2];
    double s2 = a[0] * a[7] - a[4] * a[3], s3 = a[1] * a[6] - a[5] * a[2];
    double s4 = a[1] * a[7] - a[5] * a[3], s5 = a[2] * a[7] - a[6] * a[3];
    double c5 = a[10] * a[15] - a[14] * a[11], c4 = a[9] * a[15] - a[13] * a[11];
    double c3 = a[9] * a[14] - a[13] * a[10], c2 = a[8] * a[15] - a[12] * a[11];
    double c1 = a[8] * a[14] - a[12] * a[10], c0 = a[8] * a[13] - a[12] * a[9];
    double det = s0 * c5 - s1 * c4 + s2 * c3 + s3 * c2 - s4 * c1 + s5 * c0;
    if (det == 0.0 || !isfinite(det)) {
        for (int k = 0; k < 16; k++) r[k] = (k % 5 == 0) ? 1.0 : 0.0;
        return;
    }
    double id = 1.0 / det;
    r[0] = (a[5] * c5 - a[6] * c4 + a[7] * c3) * id;
    r[1] = (-a[1] * c5 + a[2] * c4 - a[3] * c3) * id;
    r[2] = (a[13] * s5 - a[14] * s4 + a[15] * s3) * id;
    r[3] = (-a[9] * s5 + a[10] * s4 - a[11] * s3) * id;
    r[4] = (-a[4] * c5 + a[6] * c2 - a[7] * c1) * id;
    r[5] = (a[0] * c5 - a[2] * c2 + a[3] * c1) * id;
    r[6] = (-a[12] * s5 + a[14] * s2 - a[15] * s1) * id;
    r[7] = (a[8] * s5 - a[10] * s2 + a[11] * s1) * id;
    r[8] = (a[4] * c4 - a[5] * c2 + a[7] * c0) * id;
    r[9] = (-a[0] * c4 + a[1] * c2 - a[3] * c0) * id;
    r[10] = (a[12] * s4 - a[13] * s2 + a[15] * s0) * id;
    r[11] = (-a[8] * s4 + a[9] * s2 - a[11] * s0) * id;
    r[12] = (-a[4] * c3 + a[5] * c1 - a[6] * c0) * id;
    r[13] = (a[0] * c3 - a[1] * c1 + a[2] * c0) * id;
    r[14] = (-a[12] * s3 + a[13] * s1 - a[14] * s0) * id;
    r[15] = (a[8] * s3 - a[9] * s1 + a[10] * s0) * id;
}

template <typename T>
__device__ __forceinline__ void ld_block(const T *p, double b[16]) {
#pragma unroll
    for (int r = 0; r < 4; r++) ld_row(p + r * BS, b + r * BS);
}

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long *a, double v) {
    // for non-negative doubles the bit patterns order like the values
    atomicMax(a, (unsigned long long)__double_as_longlong(v));
}

// out: [0] sum |x - h(x)| (double), [1] defect max, [2] ||L - I||_inf, [3] U norm
template <typename T>
__global__ void k_diagnostics(PatternView P, const double *__restrict__ A, const T *__restrict__ L,
                              const T *__restrict__ U, const T *__restrict__ D,
                              const T *__restrict__ Ud, double *sum, unsigned long long *mx) {
    const int i = blockIdx.x * (blockDim.x >> 2) + (threadIdx.x >> 2), q = threadIdx.x & 3;
    if (i >= P.n) return;
    const int p0 = P.rowptr[i], p1 = P.rowptr[i + 1], dp = P.diagpos[i];
    const int lb = P.lrow[i], ub = P.urow[i];
    double res = 0.0, defect = 0.0, lrow = 0.0, urow = 0.0;
    double dinv_i[4];
    ld_row(D + (size_t)i * BB + q * BS, dinv_i);
    for (int p = p0; p < p1; p++) {
        const int j = P.colind[p];
        double s[4];
        ld_row(A + (size_t)p * BB + q * BS, s);
        for (int t = P.pair_ptr[p]; t < P.pair_ptr[p + 1]; t++) {
            const int2 pr = P.pairs[t];
            double l[4], u[16];
            ld_row(L + (size_t)pr.x * BB + q * BS, l);
            ld_block(U + (size_t)pr.y * BB, u);
            for (int c = 0; c < 4; c++) {
                double acc = 0.0;
                for (int k = 0; k < 4; k++) acc += l[k] * u[k * 4 + c];
                s[c] -= acc;
            }
        }
        // stored value x (row q) and h(x) (row q)
        double x[4], h[4];
        if (j < i) {
            ld_row(L + (size_t)(lb + p - p0) * BB + q * BS, x);
            double ujj[16], inv[16];
            ld_block(Ud + (size_t)j * BB, ujj);
            inv4_full(ujj, inv);
            for (int c = 0; c < 4; c++) {
                h[c] = 0.0;
                for (int k = 0; k < 4; k++) h[c] += s[k] * inv[k * 4 + c];
            }
            // (LU)_ij - A_ij = L_ij U_jj - S
            for (int c = 0; c < 4; c++) {
                double lu = 0.0;
                for (int k = 0; k < 4; k++) lu += x[k] * ujj[k * 4 + c];
                defect = fmax(defect, fabs(lu - s[c]));
                lrow += fabs(x[c]);
            }
        } else {
            if (j == i) ld_row(Ud + (size_t)i * BB + q * BS, x);
            else ld_row(U + (size_t)(ub + p - dp - 1) * BB + q * BS, x);
            for (int c = 0; c < 4; c++) {
                h[c] = s[c];
                defect = fmax(defect, fabs(x[c] - s[c]));
            }
            if (j > i) {  // row q of Dinv_i U_ij
                double u[16];
                ld_block(U + (size_t)(ub + p - dp - 1) * BB, u);
                for (int c = 0; c < 4; c++) {
                    double acc = 0.0;
                    for (int k = 0; k < 4; k++) acc += dinv_i[k] * u[k * 4 + c];
                    urow += fabs(acc);
                }
            }
        }
        for (int c = 0; c < 4; c++) res += fabs(x[c] - h[c]);
    }
    atomicAdd(sum, res);
    atomic_max_nonneg(mx + 0, defect);
    atomic_max_nonneg(mx + 1, lrow);
    atomic_max_nonneg(mx + 2, urow);
}

template <typename T>
static abilu_status diag_t(abilu_factors f, const double *A, double *out, cudaStream_t st) {
    const PatternView &P = f->p->v;
    const int c = f->cur;
    double *dsum = nullptr;
    unsigned long long *dmx = nullptr;
    void *buf = nullptr;
    ABILU_CUDA(cudaMallocAsync(&buf, 64, st));
    dsum = reinterpret_cast<double *>(buf);
    dmx = reinterpret_cast<unsigned long long *>(dsum + 1);
    ABILU_CUDA(cudaMemsetAsync(buf, 0, 64, st));
    k_diagnostics<T><<<counted((P.n + 63) / 64), 256, 0, st>>>(
        P, A, reinterpret_cast<const T *>(f->L[c]), reinterpret_cast<const T *>(f->U[c]),
        reinterpret_cast<const T *>(f->D[c]), reinterpret_cast<const T *>(f->Udiag), dsum, dmx);
    cudaError_t e = cudaGetLastError();
    unsigned long long h[4] = {0, 0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, buf, 32, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFreeAsync(buf, st);
    if (e != cudaSuccess) return cuda_fail(e, "factors_diagnostics");
    double v[4];
    memcpy(v, h, sizeof v);
    out[0] = v[0];
    out[1] = v[1];
    out[2] = v[2];
    out[3] = v[3];
    return ABILU_OK;
}

}  // namespace abilu

using namespace abilu;

extern "C" abilu_status abilu_factors_diagnostics(abilu_factors f, const double *A_vals,
                                                  double *out, abilu_stream stream) {
    if (!f || !A_vals || !out) return fail(ABILU_EINVAL, "factors_diagnostics: NULL argument");
    if (f->scalar) return fail(ABILU_EINVAL, "factors_diagnostics: block factors only");
    switch (f->dtype) {
    case ABILU_F64: return diag_t<double>(f, A_vals, out, S(stream));
    case ABILU_F32: return diag_t<float>(f, A_vals, out, S(stream));
    case ABILU_BF16: return diag_t<__nv_bfloat16>(f, A_vals, out, S(stream));
    }
    return fail(ABILU_EINVAL, "factors_diagnostics: bad dtype");
}
