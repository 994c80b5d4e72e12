// The scalar ILU(0) preconditioner of Chow and Patel (Sec. 3.2, Eq.
// scalarilu_fp_detail, Algorithm 3) and its scalar triangular sweeps
// (Algorithm 2): the variant the paper compares the block method against, on
// the same 4x4-block matrices.  FP64.
//
// The scalar pattern is every entry of every block of S_B, so the factors keep
// A's block layout: the compact L blocks hold L entries, the U blocks U
// entries, and the diagonal block of row I (the D array) holds its strictly
// lower L entries (unit diagonal implied) and the rest of U.  For entry (a, b)
// of block (I, J), with i = 4I + a, j = 4J + b:
//   s = A_ij - sum over block pairs (L_IK U_KJ)[a][b]       (K < min(I, J))
//            - [J < I]  sum_{c<b} L_IJ[a][c] U_JJ[c][b]       (K = J)
//            - [J > I]  sum_{c<a} L_II[a][c] U_IJ[c][b]       (K = I)
//            - [J = I]  sum_{c<min(a,b)} D_I[a][c] D_I[c][b]
//   L entries (J < I, or J = I and a > b): s / U_jj, U entries: s.
// The block-pair sum is the block method's product sum over the same pair
// lists; the within-block terms and the scalar pivot are what make it scalar.
// A zero or non-finite pivot is replaced by 1 and counted (Chow and Patel's
// modified iteration).  One quad per block row: thread a owns row a of every
// block of the row; other rows of a block come by quad shuffles.
//
// Sweeps: SYNC reads iterate n and writes n+1 (double buffered); ASYNC updates
// in place (volatile reads, whole-row vector stores), chunks of 64 block rows
// (256 scalar rows) handed out by a ticket counter, no barrier between sweeps.
// The triangular sweeps: y_i = r_i - sum_{j<i} L_ij y_j and
// x_i = (y_i - sum_{j>i} U_ij x_j) / U_ii, from zero guesses; the first update
// of each (y = r, x = y_i / U_ii) is formed directly.
#include <math.h>

#include <atomic>

#include "common.cuh"

namespace abilu {

constexpr int S_THREADS = 256;
constexpr int S_ROWS = S_THREADS / 4;

__device__ __forceinline__ double spivot(double u, unsigned long long *nsing) {
    if (u == 0.0 || !isfinite(u)) {
        atomicAdd(nsing, 1ull);
        return 1.0;
    }
    return u;
}

template <bool VOL>
__device__ __forceinline__ void srow(const double *p, double v[4]) {
    if constexpr (VOL) ld_row_volatile(p, v);
    else ld_row(p, v);
}

// one block row of the scalar build (thread q = row q of each block)
template <bool VOL>
__device__ __forceinline__ void sbuild_row(const PatternView &P, int i, const double *__restrict__ A,
                                           const double *Lin, const double *Uin, const double *Din,
                                           double *Lout, double *Uout, double *Dout,
                                           unsigned long long *nsing) {
    const int q = threadIdx.x & 3;
    const int p0 = P.rowptr[i], p1 = P.rowptr[i + 1], dp = P.diagpos[i];
    const int lb = P.lrow[i], ub = P.urow[i];
    double di[4];                                   // row q of D_I (iterate n)
    srow<VOL>(Din + (size_t)i * BB + q * BS, di);
    for (int p = p0; p < p1; p++) {
        const int j = P.colind[p];
        double s[4];
        ld_row(A + (size_t)p * BB + q * BS, s);
        for (int t = P.pair_ptr[p]; t < P.pair_ptr[p + 1]; t++) {   // K < min(I, J)
            const int2 pr = P.pairs[t];
            double l[4], u[4];
            srow<VOL>(Lin + (size_t)pr.x * BB + q * BS, l);
            srow<VOL>(Uin + (size_t)pr.y * BB + q * BS, u);
#pragma unroll
            for (int c = 0; c < 4; c++) {
                double acc = 0.0;
#pragma unroll
                for (int k = 0; k < 4; k++) acc += l[k] * qshfl(u[c], k);
                s[c] -= acc;
            }
        }
        double out[4];
        if (j < i) {          // L block: K = J term, then / U_JJ[b][b]
            const int lpos = lb + (p - p0);
            double f[4], dj[4];
            srow<VOL>(Lin + (size_t)lpos * BB + q * BS, f);   // row q of L_IJ
            srow<VOL>(Din + (size_t)j * BB + q * BS, dj);     // row q of D_J
#pragma unroll
            for (int b = 0; b < 4; b++) {
                double v = s[b];
#pragma unroll
                for (int c = 0; c < 4; c++)
                    if (c < b) v -= f[c] * qshfl(dj[b], c);    // U_JJ[c][b] from thread c
                out[b] = v / spivot(qshfl(dj[b], b), nsing);
            }
            st_row(Lout + (size_t)lpos * BB + q * BS, out);
        } else if (j > i) {   // U block: K = I term
            const int upos = ub + (p - dp - 1);
            double f[4];
            srow<VOL>(Uin + (size_t)upos * BB + q * BS, f);   // row q of U_IJ
#pragma unroll
            for (int b = 0; b < 4; b++) {
                double v = s[b];
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    const double ucb = qshfl(f[b], c);            // U_IJ[c][b]
                    if (c < q) v -= di[c] * ucb;                  // L_II[q][c]
                }
                out[b] = v;
            }
            st_row(Uout + (size_t)upos * BB + q * BS, out);
        } else {              // diagonal block
#pragma unroll
            for (int b = 0; b < 4; b++) {
                double v = s[b];
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    const double dcb = qshfl(di[b], c);           // D_I[c][b]
                    if (c < q && c < b) v -= di[c] * dcb;
                }
                const double piv = qshfl(di[b], b);               // U_II[b][b]
                out[b] = q > b ? v / spivot(piv, nsing) : v;
            }
            st_row(Dout + (size_t)i * BB + q * BS, out);
        }
    }
}

__global__ void __launch_bounds__(S_THREADS)
k_sbuild_sync(PatternView P, const double *__restrict__ A, const double *Lin, const double *Uin,
              const double *Din, double *Lout, double *Uout, double *Dout,
              unsigned long long *nsing) {
    const int i = blockIdx.x * S_ROWS + (threadIdx.x >> 2);
    if (i >= P.n) return;
    sbuild_row<false>(P, i, A, Lin, Uin, Din, Lout, Uout, Dout, nsing);
}

// in place; ticket t = chunk (t mod nchunks) of sweep t / nchunks
__global__ void __launch_bounds__(S_THREADS)
k_sbuild_async(PatternView P, const double *__restrict__ A, double *L, double *U, double *D,
               int nsweeps, unsigned long long *nsing, unsigned long long *ticket) {
    __shared__ unsigned long long s_t;
    const long long nchunks = (P.n + S_ROWS - 1) / S_ROWS;
    const long long total = nchunks * nsweeps;
    for (;;) {
        if (threadIdx.x == 0) s_t = atomicAdd(ticket, 1ull);
        __syncthreads();
        const long long t = (long long)s_t;
        __syncthreads();
        if (t >= total) break;
        const int i = (int)(t % nchunks) * S_ROWS + (threadIdx.x >> 2);
        if (i < P.n) sbuild_row<true>(P, i, A, L, U, D, L, U, D, nsing);
    }
}

// X^0 = A: L, U and D blocks copied from A (the current buffer)
__global__ void k_sprepare(PatternView P, const double *__restrict__ A, double *L, double *U,
                           double *D) {
    const int i = blockIdx.x * S_ROWS + (threadIdx.x >> 2), q = threadIdx.x & 3;
    if (i >= P.n) return;
    const int p0 = P.rowptr[i], p1 = P.rowptr[i + 1], dp = P.diagpos[i];
    for (int p = p0; p < p1; p++) {
        double a[4];
        ld_row(A + (size_t)p * BB + q * BS, a);
        double *dst = p < dp ? L + (size_t)(P.lrow[i] + p - p0) * BB
                             : (p > dp ? U + (size_t)(P.urow[i] + p - dp - 1) * BB : D + (size_t)i * BB);
        st_row(dst + q * BS, a);
    }
}

// ---------------------------------------------------------------- sweeps
// lower: y_i = r_i - sum_{J<I} L_IJ y_J - sum_{c<a} D_I[a][c] y_I[c]
// upper: x_i = (y_i - sum_{J>I} U_IJ x_J - sum_{c>a} D_I[a][c] x_I[c]) / D_I[a][a]
template <bool UPPER, bool VOL>
__device__ __forceinline__ double ssweep_row(const PatternView &P, int i, const double *F,
                                             const double *D, const double *rhs,
                                             const double *vin) {
    const int q = threadIdx.x & 3;
    const int l0 = UPPER ? P.urow[i] : P.lrow[i], l1 = UPPER ? P.urow[i + 1] : P.lrow[i + 1];
    const int32_t *col = UPPER ? P.ucol : P.lcol;
    double acc = rhs[(size_t)i * BS + q];
    for (int l = l0; l < l1; l++) {
        double f[4], v[4];
        ld_row(F + (size_t)l * BB + q * BS, f);
        srow<VOL>(vin + (size_t)col[l] * BS, v);
        acc -= f[0] * v[0] + f[1] * v[1] + f[2] * v[2] + f[3] * v[3];
    }
    double d[4], vi[4];
    ld_row(D + (size_t)i * BB + q * BS, d);
    srow<VOL>(vin + (size_t)i * BS, vi);
#pragma unroll
    for (int c = 0; c < 4; c++)
        if (UPPER ? c > q : c < q) acc -= d[c] * vi[c];
    if constexpr (UPPER) {
        double u = d[q];
        if (u == 0.0 || !isfinite(u)) u = 1.0;
        acc /= u;
    }
    return acc;
}

template <bool UPPER>
__global__ void __launch_bounds__(S_THREADS)
k_ssweep_sync(PatternView P, const double *__restrict__ F, const double *__restrict__ D,
              const double *__restrict__ rhs, const double *__restrict__ vin, double *__restrict__ vout,
              Skip skip) {
    if (skip_all(skip)) return;
    const int i = blockIdx.x * S_ROWS + (threadIdx.x >> 2), q = threadIdx.x & 3;
    if (i >= P.n) return;
    vout[(size_t)i * BS + q] = ssweep_row<UPPER, false>(P, i, F, D, rhs, vin);
}

// in place; UPPER runs the chunks backwards; the last sweep also writes z
template <bool UPPER>
__global__ void __launch_bounds__(S_THREADS)
k_ssweep_async(PatternView P, const double *__restrict__ F, const double *__restrict__ D,
               const double *__restrict__ rhs, double *v, double *__restrict__ z, int nsweeps,
               unsigned long long *ticket, Skip skip) {
    if (skip_all(skip)) return;
    __shared__ unsigned long long s_t;
    const long long nchunks = (P.n + S_ROWS - 1) / S_ROWS;
    const long long total = nchunks * nsweeps;
    const int q = threadIdx.x & 3;
    for (;;) {
        if (threadIdx.x == 0) s_t = atomicAdd(ticket, 1ull);
        __syncthreads();
        const long long t = (long long)s_t;
        __syncthreads();
        if (t >= total) break;
        const long long c = t % nchunks;
        const int chunk = UPPER ? (int)(nchunks - 1 - c) : (int)c;
        const int i = chunk * S_ROWS + (threadIdx.x >> 2);
        if (i < P.n) {
            const double x = ssweep_row<UPPER, true>(P, i, F, D, rhs, v);
            __syncwarp(quad_mask());   // the quad's reads of its own row precede its writes
            reinterpret_cast<volatile double *>(v)[(size_t)i * BS + q] = x;
            if (z && t / nchunks == nsweeps - 1) z[(size_t)i * BS + q] = x;
        }
    }
}

// first updates: y = r (lower), x = y_i / U_ii (upper); either may go to z
__global__ void k_sfirst(PatternView P, const double *__restrict__ D, const double *__restrict__ in,
                         double *__restrict__ out, int upper, Skip skip) {
    if (skip_all(skip)) return;
    const int i = blockIdx.x * S_ROWS + (threadIdx.x >> 2), q = threadIdx.x & 3;
    if (i >= P.n) return;
    double v = in[(size_t)i * BS + q];
    if (upper) {
        double u = D[(size_t)i * BB + q * BS + q];
        if (u == 0.0 || !isfinite(u)) u = 1.0;
        v /= u;
    }
    out[(size_t)i * BS + q] = v;
}

abilu_status scalar_build(abilu_factors f, const double *A, int nsweeps, abilu_mode mode,
                          abilu_init init, cudaStream_t st) {
    const PatternView &P = f->p->v;
    const int grid = (P.n + S_ROWS - 1) / S_ROWS;
    double **L = reinterpret_cast<double **>(f->L), **U = reinterpret_cast<double **>(f->U);
    double **D = reinterpret_cast<double **>(f->D);
    if (init == ABILU_INIT_FROM_A) {
        k_sprepare<<<counted(grid), S_THREADS, 0, st>>>(P, A, L[f->cur], U[f->cur], D[f->cur]);
        ABILU_LAUNCH_CHECK("k_sprepare");
    }
    if (nsweeps == 0) return ABILU_OK;
    if (mode == ABILU_SYNC) {
        for (int s = 0; s < nsweeps; s++) {
            const int c = f->cur, o = 1 - c;
            k_sbuild_sync<<<counted(grid), S_THREADS, 0, st>>>(P, A, L[c], U[c], D[c], L[o], U[o], D[o],
                                                               f->ctr);
            ABILU_LAUNCH_CHECK("k_sbuild_sync");
            f->cur = o;
        }
        return ABILU_OK;
    }
    static std::atomic<int> per_sm_cache{-1};
    int dev = 0, sms = 0, per_sm = per_sm_cache.load(std::memory_order_relaxed);
    cudaGetDevice(&dev);
    if (per_sm < 0) {
        ABILU_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sbuild_async, S_THREADS, 0));
        per_sm_cache.store(per_sm, std::memory_order_relaxed);
    }
    ABILU_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int ctas = per_sm * sms;
    if (ctas > grid) ctas = grid;   // at most one CTA per chunk
    if (ctas < 1) ctas = 1;
    ABILU_CUDA(cudaMemsetAsync(f->ctr + 1, 0, sizeof(unsigned long long), st));
    const int c = f->cur;
    k_sbuild_async<<<counted(ctas), S_THREADS, 0, st>>>(P, A, L[c], U[c], D[c], nsweeps, f->ctr,
                                                        f->ctr + 1);
    ABILU_LAUNCH_CHECK("k_sbuild_async");
    return ABILU_OK;
}

template <bool UPPER> static int sweep_ctas() {
    static std::atomic<int> cache{-1};
    int c = cache.load(std::memory_order_relaxed);
    if (c < 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ssweep_async<UPPER>, S_THREADS, 0);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        c = per_sm * sms > 0 ? per_sm * sms : 1;
        cache.store(c, std::memory_order_relaxed);
    }
    return c;
}

void scalar_apply_warm() {
    sweep_ctas<false>();
    sweep_ctas<true>();
}

abilu_status scalar_apply(abilu_factors f, const double *r, double *z, int nl, int nu,
                          abilu_mode mode, cudaStream_t st, Skip skip) {
    const PatternView &P = f->p->v;
    const int c = f->cur;
    const double *L = reinterpret_cast<const double *>(f->L[c]);
    const double *U = reinterpret_cast<const double *>(f->U[c]);
    const double *D = reinterpret_cast<const double *>(f->D[c]);
    double *y[2] = {reinterpret_cast<double *>(f->y[0]), reinterpret_cast<double *>(f->y[1])};
    double *x[2] = {reinterpret_cast<double *>(f->x[0]), reinterpret_cast<double *>(f->x[1])};
    const int grid = (P.n + S_ROWS - 1) / S_ROWS;
    const long long nchunks = grid;
    if (nl == 0 || nu == 0) {  // y = 0, or no upper update: z = 0
        ABILU_CUDA(cudaMemsetAsync(z, 0, sizeof(double) * (size_t)P.n * BS, st));
        return ABILU_OK;
    }
    // lower: y^1 = r, then nl - 1 sweeps
    const double *yfin;
    if (mode == ABILU_SYNC) {
        const double *yprev = r;
        for (int s = 2; s <= nl; s++) {
            k_ssweep_sync<false><<<counted(grid), S_THREADS, 0, st>>>(P, L, D, r, yprev, y[s & 1], skip);
            yprev = y[s & 1];
        }
        yfin = yprev;
    } else {
        k_sfirst<<<counted(grid), S_THREADS, 0, st>>>(P, D, r, y[0], 0, skip);
        if (nl >= 2) {
            ABILU_CUDA(cudaMemsetAsync(f->ctr + 2, 0, sizeof(unsigned long long), st));
            const int g = (int)(sweep_ctas<false>() < nchunks ? sweep_ctas<false>() : nchunks);
            k_ssweep_async<false><<<counted(g), S_THREADS, 0, st>>>(P, L, D, r, y[0], nullptr, nl - 1,
                                                                  f->ctr + 2, skip);
        }
        yfin = y[0];
    }
    ABILU_LAUNCH_CHECK("scalar lower");
    // upper: x^1 = y_i / U_ii, then nu - 1 sweeps, the last into z
    if (mode == ABILU_SYNC) {
        k_sfirst<<<counted(grid), S_THREADS, 0, st>>>(P, D, yfin, nu == 1 ? z : x[1], 1, skip);
        const double *xprev = x[1];
        for (int s = 2; s <= nu; s++) {
            double *xo = s == nu ? z : x[s & 1];
            k_ssweep_sync<true><<<counted(grid), S_THREADS, 0, st>>>(P, U, D, yfin, xprev, xo, skip);
            xprev = xo;
        }
    } else {
        k_sfirst<<<counted(grid), S_THREADS, 0, st>>>(P, D, yfin, nu == 1 ? z : x[0], 1, skip);
        if (nu >= 2) {
            ABILU_CUDA(cudaMemsetAsync(f->ctr + 3, 0, sizeof(unsigned long long), st));
            const int g = (int)(sweep_ctas<true>() < nchunks ? sweep_ctas<true>() : nchunks);
            k_ssweep_async<true><<<counted(g), S_THREADS, 0, st>>>(P, U, D, yfin, x[0], z, nu - 1,
                                                                 f->ctr + 3, skip);
        }
    }
    ABILU_LAUNCH_CHECK("scalar upper");
    return ABILU_OK;
}

// export: X in A's layout (the diagonal block from D, holding both parts)
__global__ void k_sexport(PatternView P, const double *__restrict__ L, const double *__restrict__ U,
                          const double *__restrict__ D, double *X) {
    const int i = blockIdx.x * S_ROWS + (threadIdx.x >> 2), q = threadIdx.x & 3;
    if (i >= P.n) return;
    const int p0 = P.rowptr[i], p1 = P.rowptr[i + 1], dp = P.diagpos[i];
    for (int p = p0; p < p1; p++) {
        const double *src = p < dp ? L + (size_t)(P.lrow[i] + p - p0) * BB
                                   : (p > dp ? U + (size_t)(P.urow[i] + p - dp - 1) * BB : D + (size_t)i * BB);
        double v[4];
        ld_row(src + q * BS, v);
        st_row(X + (size_t)p * BB + q * BS, v);
    }
}

abilu_status scalar_export(abilu_factors f, double *X, cudaStream_t st) {
    const PatternView &P = f->p->v;
    const int c = f->cur;
    if (!X) return ABILU_OK;
    k_sexport<<<counted((P.n + S_ROWS - 1) / S_ROWS), S_THREADS, 0, st>>>(
        P, reinterpret_cast<const double *>(f->L[c]), reinterpret_cast<const double *>(f->U[c]),
        reinterpret_cast<const double *>(f->D[c]), X);
    ABILU_LAUNCH_CHECK("k_sexport");
    return ABILU_OK;
}

}  // namespace abilu
