// Block ILU(0) by fixed-point sweeps (Sec. 4.2).
//
// One sweep evaluates, for every block (i,j) of S_B,
//   S_ij = A_ij - sum_{k<min(i,j)} L_ik U_kj            (Eq. bilu)
//   U_ij = S_ij (i <= j),  L_ij = S_ij U_jj^{-1} (i > j),
// and refreshes Dinv_i = U_ii^{-1}.  Work item = one block row (the paper's
// work item, Sec. 3.3), blocks of the row in ascending column order with a
// local accumulator and one write per block.
//
// Thread mapping: 4 threads ("a quad") per block row; thread q of the quad
// owns row q of every 4x4 block, so a block is read with four 16/32-byte row
// loads that are contiguous across the quad (fully used sectors), and the 4x4
// products exchange rows through quad shuffles.  The inversion of U_ii is done
// by one thread per block out of shared memory (FP64 adjugate), because FP64
// throughput is scarce on this GPU: no FP64 work is duplicated across lanes.
//
// Precision: A is FP64.  In FP64 factor mode everything is FP64.  In FP32/BF16
// factor mode the products and the L update run in FP32 and only the U_ii
// inversion is FP64; the factors are stored in the narrow type.
//
// Modes: SYNC reads iterate n (L[cur], U[cur], D[cur]) and writes n+1 into the
// other buffer (Jacobi-type, Eq. seq_blockilu_fp); ASYNC updates one buffer in
// place, reading whatever is current through volatile loads, with the rows cut
// into chunks handed out by a ticket counter across all sweeps, so no barrier
// separates sweeps (Algorithm 4 with blocks, Eq. async_blockilu_fp).
#include "common.cuh"

namespace abilu {

template <typename T> struct BuildArith { using C = float; };
template <> struct BuildArith<double> { using C = double; };

constexpr int BUILD_THREADS = 256;
constexpr int BUILD_ROWS = BUILD_THREADS / 4;  // rows per CTA (= chunk of the async queue)

// Inverse of a 4x4 block by the adjugate: Laplace expansion by the 2x2 minors
// of rows {0,1} and {2,3}; inverse = adj / det.  det == 0 or non-finite marks
// the block singular and it is replaced by the identity (the modified
// iteration of Sec. 4.2).  FP64 throughout.
__device__ __forceinline__ bool inv4_adj(const double *a, double *r) {
    double s0 = a[0] * a[5] - a[4] * a[1], s1 = a[0] * a[6] - a[4] * a[2];
    double s2 = a[0] * a[7] - a[4] * a[3], s3 = a[1] * a[6] - a[5] * a[2];
    double s4 = a[1] * a[7] - a[5] * a[3], s5 = a[2] * a[7] - a[6] * a[3];
    double c5 = a[10] * a[15] - a[14] * a[11], c4 = a[9] * a[15] - a[13] * a[11];
    double c3 = a[9] * a[14] - a[13] * a[10], c2 = a[8] * a[15] - a[12] * a[11];
    double c1 = a[8] * a[14] - a[12] * a[10], c0 = a[8] * a[13] - a[12] * a[9];
    double det = s0 * c5 - s1 * c4 + s2 * c3 + s3 * c2 - s4 * c1 + s5 * c0;
    if (det == 0.0 || !isfinite(det)) {
#pragma unroll
        for (int k = 0; k < 16; k++) r[k] = (k % 5 == 0) ? 1.0 : 0.0;
        return true;
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
    return false;
}

template <bool VOL, typename T, typename C>
__device__ __forceinline__ void st_row_sel(T *p, const C v[4]) {
    if constexpr (VOL) {
        // whole 16/32-byte vector stores from registers: another thread never
        // sees a partial sum (Sec. 3.3); a torn block mixes complete old and
        // new rows, which the block-asynchronous model allows.
        if constexpr (sizeof(T) == 8) {
            double w0 = (double)v[0], w1 = (double)v[1], w2 = (double)v[2], w3 = (double)v[3];
            asm volatile("st.volatile.global.v2.f64 [%0], {%1,%2};" ::"l"(p), "d"(w0), "d"(w1) : "memory");
            asm volatile("st.volatile.global.v2.f64 [%0], {%1,%2};" ::"l"(p + 2), "d"(w2), "d"(w3) : "memory");
        } else if constexpr (sizeof(T) == 4) {
            asm volatile("st.volatile.global.v4.f32 [%0], {%1,%2,%3,%4};" ::"l"(p), "f"((float)v[0]),
                         "f"((float)v[1]), "f"((float)v[2]), "f"((float)v[3]) : "memory");
        } else {
            __nv_bfloat162 a = __floats2bfloat162_rn((float)v[0], (float)v[1]);
            __nv_bfloat162 b = __floats2bfloat162_rn((float)v[2], (float)v[3]);
            unsigned ua = *reinterpret_cast<unsigned *>(&a), ub = *reinterpret_cast<unsigned *>(&b);
            asm volatile("st.volatile.global.v2.u32 [%0], {%1,%2};" ::"l"(p), "r"(ua), "r"(ub) : "memory");
        }
    } else {
        double w[4] = {(double)v[0], (double)v[1], (double)v[2], (double)v[3]};
        st_row(p, w);
    }
}

// One block row i handled by one quad.  Writes the row's L and U blocks,
// leaves U_ii (row q) in sh_u[(row in CTA)*16 + q*4 ..].
template <typename T, bool VOL>
__device__ __forceinline__ void build_row_products(const PatternView &P, int i,
                                                   const double *__restrict__ A, const T *Lin,
                                                   const T *Uin, const T *Din, T *Lout, T *Uout,
                                                   double *sh_u) {
    using C = typename BuildArith<T>::C;
    const int q = threadIdx.x & 3;
    const int p0 = P.rowptr[i], p1 = P.rowptr[i + 1], dp = P.diagpos[i];
    const int lb = P.lrow[i], ub = P.urow[i];
    for (int p = p0; p < p1; p++) {
        const int j = P.colind[p];
        C s[4];
        {
            double a[4];
            ld_row(A + (size_t)p * BB + q * BS, a);
            s[0] = (C)a[0]; s[1] = (C)a[1]; s[2] = (C)a[2]; s[3] = (C)a[3];
        }
        const int t1 = P.pair_ptr[p + 1];
        for (int t = P.pair_ptr[p]; t < t1; t++) {
            const int2 pr = P.pairs[t];
            C l[4], u[4];
            ld_row_sel<VOL>(Lin + (size_t)pr.x * BB + q * BS, l);  // row q of L_ik
            ld_row_sel<VOL>(Uin + (size_t)pr.y * BB + q * BS, u);  // row q of U_kj
            C acc[4] = {0, 0, 0, 0};
#pragma unroll
            for (int k = 0; k < 4; k++)
#pragma unroll
                for (int c = 0; c < 4; c++) acc[c] += l[k] * qshfl(u[c], k);
#pragma unroll
            for (int c = 0; c < 4; c++) s[c] -= acc[c];
        }
        if (j < i) {  // L_ij = S Dinv_j
            C d[4];
            ld_row_sel<VOL>(Din + (size_t)j * BB + q * BS, d);
            C o[4];
#pragma unroll
            for (int c = 0; c < 4; c++) {
                // o[c] = sum_k s[k] * Dinv_j[k][c]; row k of Dinv_j lives in thread k
                C d0 = qshfl(d[c], 0), d1 = qshfl(d[c], 1), d2 = qshfl(d[c], 2), d3 = qshfl(d[c], 3);
                o[c] = s[0] * d0 + s[1] * d1 + s[2] * d2 + s[3] * d3;
            }
            st_row_sel<VOL>(Lout + (size_t)(lb + (p - p0)) * BB + q * BS, o);
        } else if (j == i) {
            double *u = sh_u + (threadIdx.x >> 2) * BB + q * BS;
            u[0] = (double)s[0]; u[1] = (double)s[1]; u[2] = (double)s[2]; u[3] = (double)s[3];
        } else {
            st_row_sel<VOL>(Uout + (size_t)(ub + (p - dp - 1)) * BB + q * BS, s);
        }
    }
}

// Inversion phase: one thread per row of the CTA inverts its U_ii from shared
// memory and writes Dinv_i (and U_ii if requested) with coalesced row stores
// done by the quads afterwards.
template <typename T, bool VOL>
__device__ __forceinline__ void build_cta_invert(int row0, int n, T *Dout, T *Udiag,
                                                 double *sh_u, double *sh_d,
                                                 unsigned long long *nsing) {
    __syncthreads();
    const int r = threadIdx.x;
    if (r < BUILD_ROWS && row0 + r < n) {
        double a[16], inv[16];
#pragma unroll
        for (int k = 0; k < 16; k++) a[k] = sh_u[r * BB + k];
        if (inv4_adj(a, inv)) atomicAdd(nsing, 1ull);
#pragma unroll
        for (int k = 0; k < 16; k++) sh_d[r * BB + k] = inv[k];
    }
    __syncthreads();
    const int i = row0 + (threadIdx.x >> 2), q = threadIdx.x & 3;
    if (i < n) {
        const double *d = sh_d + (threadIdx.x >> 2) * BB + q * BS;
        st_row_sel<VOL>(Dout + (size_t)i * BB + q * BS, d);
        if (Udiag) {
            const double *u = sh_u + (threadIdx.x >> 2) * BB + q * BS;
            st_row_sel<false>(Udiag + (size_t)i * BB + q * BS, u);
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(BUILD_THREADS)
k_build_sync(PatternView P, const double *__restrict__ A, const T *__restrict__ Lin,
             const T *__restrict__ Uin, const T *__restrict__ Din, T *__restrict__ Lout,
             T *__restrict__ Uout, T *__restrict__ Dout, T *__restrict__ Udiag,
             unsigned long long *nsing) {
    __shared__ double sh_u[BUILD_ROWS * BB];
    __shared__ double sh_d[BUILD_ROWS * BB];
    const int row0 = blockIdx.x * BUILD_ROWS;
    const int i = row0 + (threadIdx.x >> 2);
    if (i < P.n) build_row_products<T, false>(P, i, A, Lin, Uin, Din, Lout, Uout, sh_u);
    build_cta_invert<T, false>(row0, P.n, Dout, Udiag, sh_u, sh_d, nsing);
}

// Persistent in-place kernel: tickets t = 0 .. nsweeps*nchunks-1 taken in
// order from ctr; ticket t is chunk (t mod nchunks) in sweep (t / nchunks).
template <typename T>
__global__ void __launch_bounds__(BUILD_THREADS)
k_build_async(PatternView P, const double *__restrict__ A, T *L, T *U, T *D, T *Udiag,
              int nsweeps, unsigned long long *nsing, unsigned long long *ticket) {
    __shared__ double sh_u[BUILD_ROWS * BB];
    __shared__ double sh_d[BUILD_ROWS * BB];
    __shared__ unsigned long long s_t;
    const long long nchunks = (P.n + BUILD_ROWS - 1) / BUILD_ROWS;
    const long long total = nchunks * nsweeps;
    for (;;) {
        if (threadIdx.x == 0) s_t = atomicAdd(ticket, 1ull);
        __syncthreads();
        const long long t = (long long)s_t;
        __syncthreads();
        if (t >= total) break;
        const int sweep = (int)(t / nchunks);
        const int row0 = (int)(t % nchunks) * BUILD_ROWS;
        const int i = row0 + (threadIdx.x >> 2);
        if (i < P.n) build_row_products<T, true>(P, i, A, L, U, D, L, U, sh_u);
        build_cta_invert<T, true>(row0, P.n, D, sweep == nsweeps - 1 ? Udiag : nullptr, sh_u,
                                  sh_d, nsing);
    }
}

// X^0 = A: L^0 = strictly lower blocks of A (unscaled), U^0 = upper blocks,
// Dinv^0 = inv(A_ii) (Sec. 6 setup: the initial guess is the matrix itself).
template <typename T>
__global__ void __launch_bounds__(BUILD_THREADS)
k_build_init(PatternView P, const double *__restrict__ A, T *__restrict__ L, T *__restrict__ U,
             T *__restrict__ D, T *__restrict__ Udiag, unsigned long long *nsing) {
    __shared__ double sh_u[BUILD_ROWS * BB];
    __shared__ double sh_d[BUILD_ROWS * BB];
    const int row0 = blockIdx.x * BUILD_ROWS;
    const int i = row0 + (threadIdx.x >> 2), q = threadIdx.x & 3;
    if (i < P.n) {
        const int p0 = P.rowptr[i], p1 = P.rowptr[i + 1], dp = P.diagpos[i];
        const int lb = P.lrow[i], ub = P.urow[i];
        for (int p = p0; p < p1; p++) {
            double a[4];
            ld_row(A + (size_t)p * BB + q * BS, a);
            if (p < dp) st_row(L + (size_t)(lb + p - p0) * BB + q * BS, a);
            else if (p > dp) st_row(U + (size_t)(ub + p - dp - 1) * BB + q * BS, a);
            else {
                double *u = sh_u + (threadIdx.x >> 2) * BB + q * BS;
                u[0] = a[0]; u[1] = a[1]; u[2] = a[2]; u[3] = a[3];
            }
        }
    }
    build_cta_invert<T, false>(row0, P.n, D, Udiag, sh_u, sh_d, nsing);
}

// Export to A's layout in FP64: X[p] = L or U block, U_ii on the diagonal.
template <typename T>
__global__ void k_export(PatternView P, const T *__restrict__ L, const T *__restrict__ U,
                         const T *__restrict__ D, const T *__restrict__ Udiag, double *X,
                         double *Dinv) {
    const int i = blockIdx.x * (blockDim.x >> 2) + (threadIdx.x >> 2), q = threadIdx.x & 3;
    if (i >= P.n) return;
    if (X) {
        const int p0 = P.rowptr[i], p1 = P.rowptr[i + 1], dp = P.diagpos[i];
        const int lb = P.lrow[i], ub = P.urow[i];
        for (int p = p0; p < p1; p++) {
            double v[4];
            if (p < dp) ld_row(L + (size_t)(lb + p - p0) * BB + q * BS, v);
            else if (p > dp) ld_row(U + (size_t)(ub + p - dp - 1) * BB + q * BS, v);
            else ld_row(Udiag + (size_t)i * BB + q * BS, v);
            st_row(X + (size_t)p * BB + q * BS, v);
        }
    }
    if (Dinv) {
        double v[4];
        ld_row(D + (size_t)i * BB + q * BS, v);
        st_row(Dinv + (size_t)i * BB + q * BS, v);
    }
}

template <typename T>
static abilu_status build_t(abilu_factors f, const double *A, int nsweeps, abilu_mode mode,
                            abilu_init init, cudaStream_t st) {
    const PatternView &P = f->p->v;
    const int grid = (P.n + BUILD_ROWS - 1) / BUILD_ROWS;
    T **L = reinterpret_cast<T **>(f->L), **U = reinterpret_cast<T **>(f->U);
    T **D = reinterpret_cast<T **>(f->D);
    T *Ud = reinterpret_cast<T *>(f->Udiag);
    if (init == ABILU_INIT_FROM_A) {
        k_build_init<T><<<counted(grid), BUILD_THREADS, 0, st>>>(P, A, L[f->cur], U[f->cur], D[f->cur], Ud,
                                                        f->ctr);
        ABILU_LAUNCH_CHECK("k_build_init");
    }
    if (nsweeps == 0) return ABILU_OK;
    if (mode == ABILU_SYNC) {
        for (int s = 0; s < nsweeps; s++) {
            const int c = f->cur, o = 1 - f->cur;
            k_build_sync<T><<<counted(grid), BUILD_THREADS, 0, st>>>(
                P, A, L[c], U[c], D[c], L[o], U[o], D[o], s == nsweeps - 1 ? Ud : nullptr, f->ctr);
            ABILU_LAUNCH_CHECK("k_build_sync");
            f->cur = o;
        }
    } else {
        int dev;
        cudaGetDevice(&dev);
        int per_sm = 0, sms = 0;
        ABILU_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_build_async<T>,
                                                                 BUILD_THREADS, 0));
        ABILU_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        // at most one CTA per chunk: more would sweep the same rows at once
        int ctas = per_sm * sms;
        if (ctas > grid) ctas = grid;
        if (ctas < 1) ctas = 1;
        ABILU_CUDA(cudaMemsetAsync(f->ctr + 1, 0, sizeof(unsigned long long), st));
        const int c = f->cur;
        k_build_async<T><<<counted(ctas), BUILD_THREADS, 0, st>>>(P, A, L[c], U[c], D[c], Ud, nsweeps,
                                                         f->ctr, f->ctr + 1);
        ABILU_LAUNCH_CHECK("k_build_async");
    }
    return ABILU_OK;
}

template <typename T>
static abilu_status export_t(abilu_factors f, double *X, double *Dinv, cudaStream_t st) {
    const PatternView &P = f->p->v;
    const int c = f->cur;
    k_export<T><<<counted((P.n + 63) / 64), 256, 0, st>>>(
        P, reinterpret_cast<const T *>(f->L[c]), reinterpret_cast<const T *>(f->U[c]),
        reinterpret_cast<const T *>(f->D[c]), reinterpret_cast<const T *>(f->Udiag), X, Dinv);
    ABILU_LAUNCH_CHECK("k_export");
    return ABILU_OK;
}

abilu_status build_dispatch(abilu_factors f, const double *A, int nsweeps, abilu_mode mode,
                            abilu_init init, cudaStream_t st) {
    switch (f->dtype) {
    case ABILU_F64: return build_t<double>(f, A, nsweeps, mode, init, st);
    case ABILU_F32: return build_t<float>(f, A, nsweeps, mode, init, st);
    case ABILU_BF16: return build_t<__nv_bfloat16>(f, A, nsweeps, mode, init, st);
    }
    return fail(ABILU_EINVAL, "build: bad dtype");
}

abilu_status export_dispatch(abilu_factors f, double *X, double *Dinv, cudaStream_t st) {
    switch (f->dtype) {
    case ABILU_F64: return export_t<double>(f, X, Dinv, st);
    case ABILU_F32: return export_t<float>(f, X, Dinv, st);
    case ABILU_BF16: return export_t<__nv_bfloat16>(f, X, Dinv, st);
    }
    return fail(ABILU_EINVAL, "export: bad dtype");
}

}  // namespace abilu
