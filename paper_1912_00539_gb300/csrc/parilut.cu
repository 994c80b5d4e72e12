// Threshold block ILU by fixed-point sweeps.
//
// The paper's closing section names a parallel threshold ILU (ParILUT) as the
// next extension of its sweeps, without an algorithm.  This is the library's:
//   start   X = A on A's pattern S, `sweeps` synchronous sweeps of Eq. (bilu);
//   repeat `iters` times:
//     fill  S' = the block pattern of L U (L unit lower, U upper on S; it
//           contains S), new blocks start at zero, A is zero outside its own
//           pattern, `sweeps` synchronous sweeps on S';
//     drop  of the strictly lower blocks keep those whose squared Frobenius
//           norm exceeds the (budget+1)-th largest (every one if there are at
//           most budget), likewise the strictly upper blocks; diagonal blocks
//           stay.  Budgets: floor(fill * count) with the counts of A's
//           pattern.  `sweeps` synchronous sweeps on the kept pattern.
// Every sweep is the FP64 synchronous build of build.cu on an analysed
// pattern (abilu_pattern_create), so the pair lists of the fill blocks come
// from the same analysis as A's.  Pattern work on the device: a thread per row
// merges the upper parts of the rows its L blocks name (sorted, at most
// PLU_MAX_ROW blocks per row); values move between patterns by a per-row merge
// of the sorted columns; the selection threshold is found by bisection on the
// bit patterns of the non-negative keys (integer counts, exact).
#include <string.h>

#include <utility>
#include <vector>

#include "common.cuh"

namespace abilu {

abilu_status build_dispatch(abilu_factors f, const double *A, int nsweeps, abilu_mode mode,
                            abilu_init init, cudaStream_t st);
abilu_status export_dispatch(abilu_factors f, double *X, double *Dinv, cudaStream_t st);
abilu_status scan_i32(const int32_t *in, int32_t *out, int n, long long *scratch, unsigned *err,
                      cudaStream_t st);
abilu_status form_scaled_upper(abilu_factors f, cudaStream_t st);
__global__ void k_block_norm2(const double *__restrict__ A, long long nnzb, double *__restrict__ w);

constexpr int PLU_THREADS = 128;
constexpr int PLU_MAX_ROW = 192;   // blocks per row of the pattern of L U

// Row i of the pattern of L U: the columns j >= k of row k for k = i and for
// every column k < i of row i, sorted and distinct.  FILL = false: count only
// (cnt[i]); FILL: write them at out_col + out_ptr[i].  A row longer than
// PLU_MAX_ROW sets *err and is cut (the host then fails the call).
template <bool FILL>
__global__ void __launch_bounds__(PLU_THREADS)
k_lu_pattern(int n, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colind,
             const int32_t *__restrict__ diagpos, int32_t *__restrict__ cnt,
             const int32_t *__restrict__ out_ptr, int32_t *__restrict__ out_col, unsigned *err) {
    const int i = blockIdx.x * PLU_THREADS + threadIdx.x;
    if (i >= n) return;
    int buf[PLU_MAX_ROW];
    int m = 0;
    const int p0 = rowptr[i], pd = diagpos[i];
    for (int p = p0; p <= pd; p++) {   // k < i (L blocks), then k = i
        const int k = colind[p];
        for (int q = diagpos[k]; q < rowptr[k + 1]; q++) {
            const int j = colind[q];
            int a = 0, b = m;   // lower bound of j in buf[0..m)
            while (a < b) {
                const int h = (a + b) >> 1;
                if (buf[h] < j) a = h + 1; else b = h;
            }
            if (a < m && buf[a] == j) continue;
            if (m == PLU_MAX_ROW) {
                atomicOr(err, 1u);
                continue;
            }
            for (int t = m; t > a; t--) buf[t] = buf[t - 1];
            buf[a] = j;
            m++;
        }
    }
    if constexpr (FILL) {
        int32_t *o = out_col + out_ptr[i];
        for (int t = 0; t < m; t++) o[t] = buf[t];
    } else {
        cnt[i] = m;
    }
}

// Values of row i on the new pattern: a quad per row merges the sorted old
// and new columns; thread q copies row q of each matched block (zero where the
// old pattern has none).  Two sources (X on the old pattern, A on its own).
__global__ void __launch_bounds__(PLU_THREADS)
k_map_blocks(int n, const int32_t *__restrict__ rp_new, const int32_t *__restrict__ ci_new,
             const int32_t *__restrict__ rp_x, const int32_t *__restrict__ ci_x,
             const double *__restrict__ X, const int32_t *__restrict__ rp_a,
             const int32_t *__restrict__ ci_a, const double *__restrict__ A,
             double *__restrict__ X_new, double *__restrict__ A_new) {
    const int i = blockIdx.x * (PLU_THREADS / 4) + (threadIdx.x >> 2), q = threadIdx.x & 3;
    if (i >= n) return;
    int px = rp_x[i], pa = rp_a[i];
    const int px1 = rp_x[i + 1], pa1 = rp_a[i + 1];
    for (int p = rp_new[i]; p < rp_new[i + 1]; p++) {
        const int j = ci_new[p];
        while (px < px1 && ci_x[px] < j) px++;
        while (pa < pa1 && ci_a[pa] < j) pa++;
        double v[4] = {0.0, 0.0, 0.0, 0.0}, w[4] = {0.0, 0.0, 0.0, 0.0};
        if (px < px1 && ci_x[px] == j) ld_row(X + (size_t)px * BB + q * BS, v);
        if (pa < pa1 && ci_a[pa] == j) ld_row(A + (size_t)pa * BB + q * BS, w);
        st_row(X_new + (size_t)p * BB + q * BS, v);
        st_row(A_new + (size_t)p * BB + q * BS, w);
    }
}

// Factors from X in the pattern layout (L_ij at column < row, U_ij at column
// > row, U_ii on the diagonal) and Dinv: the compact arrays of iterate `cur`,
// rounded to the storage type T
template <typename T>
__global__ void __launch_bounds__(PLU_THREADS)
k_import(PatternView P, const double *__restrict__ X, const double *__restrict__ Dinv,
         T *__restrict__ L, T *__restrict__ U, T *__restrict__ D, T *__restrict__ Udiag) {
    const int i = blockIdx.x * (PLU_THREADS / 4) + (threadIdx.x >> 2), q = threadIdx.x & 3;
    if (i >= P.n) return;
    const int p0 = P.rowptr[i], p1 = P.rowptr[i + 1], dp = P.diagpos[i];
    for (int p = p0; p < p1; p++) {
        double v[4];
        ld_row(X + (size_t)p * BB + q * BS, v);
        if (p < dp) st_row(L + (size_t)(P.lrow[i] + p - p0) * BB + q * BS, v);
        else if (p > dp) st_row(U + (size_t)(P.urow[i] + p - dp - 1) * BB + q * BS, v);
        else st_row(Udiag + (size_t)i * BB + q * BS, v);
    }
    double d[4];
    ld_row(Dinv + (size_t)i * BB + q * BS, d);
    st_row(D + (size_t)i * BB + q * BS, d);
}

// cnt[0] += strictly lower blocks with key bits >= tl, cnt[1] += strictly
// upper ones with key bits >= tu (keys: squared norms, non-negative, so the
// bit patterns order like the values)
__global__ void __launch_bounds__(256)
k_count_at_least(int n, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colind,
                 const unsigned long long *__restrict__ key, unsigned long long tl,
                 unsigned long long tu, unsigned long long *cnt) {
    const int i = blockIdx.x * 256 + threadIdx.x;
    unsigned long long cl = 0, cu = 0;
    if (i < n) {
        for (int p = rowptr[i]; p < rowptr[i + 1]; p++) {
            const int j = colind[p];
            if (j < i) cl += key[p] >= tl;
            else if (j > i) cu += key[p] >= tu;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        cl += __shfl_down_sync(0xffffffffu, cl, o);
        cu += __shfl_down_sync(0xffffffffu, cu, o);
    }
    if ((threadIdx.x & 31) == 0 && (cl | cu)) {
        atomicAdd(cnt, cl);
        atomicAdd(cnt + 1, cu);
    }
}

// kept blocks of row i: diagonal, lower with key bits > tl, upper with > tu
// (KEEP_ALL_L / _U in the flags: every lower / upper block)
template <bool FILL>
__global__ void __launch_bounds__(PLU_THREADS)
k_compact(int n, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colind,
          const unsigned long long *__restrict__ key, unsigned long long tl, unsigned long long tu,
          int keep_all_l, int keep_all_u, int32_t *__restrict__ cnt,
          const int32_t *__restrict__ out_ptr, int32_t *__restrict__ out_col,
          const double *__restrict__ X, const double *__restrict__ A, double *__restrict__ X_out,
          double *__restrict__ A_out) {
    const int i = blockIdx.x * (PLU_THREADS / 4) + (threadIdx.x >> 2), q = threadIdx.x & 3;
    if (i >= n) return;
    int o = FILL ? out_ptr[i] : 0;
    for (int p = rowptr[i]; p < rowptr[i + 1]; p++) {
        const int j = colind[p];
        const bool keep = j == i || (j < i ? (keep_all_l || key[p] > tl) : (keep_all_u || key[p] > tu));
        if (!keep) continue;
        if constexpr (FILL) {
            if (q == 0) out_col[o] = j;
            double v[4];
            ld_row(X + (size_t)p * BB + q * BS, v);
            st_row(X_out + (size_t)o * BB + q * BS, v);
            ld_row(A + (size_t)p * BB + q * BS, v);
            st_row(A_out + (size_t)o * BB + q * BS, v);
        }
        o++;
    }
    if (!FILL && q == 0) cnt[i] = o;
}

}  // namespace abilu

// ------------------------------------------------------------------- host

namespace abilu {

namespace {

// device allocations released at scope exit
struct DevBufs {
    std::vector<void *> p;
    ~DevBufs() {
        for (void *q : p) cudaFree(q);
    }
    template <typename T> abilu_status get(T **out, size_t count) {
        void *q = nullptr;
        cudaError_t e = cudaMalloc(&q, sizeof(T) * (count > 0 ? count : 1));
        if (e != cudaSuccess) return cuda_fail(e, "abilu_parilut: cudaMalloc");
        p.push_back(q);
        *out = static_cast<T *>(q);
        return ABILU_OK;
    }
};

struct PatternGuard {
    abilu_pattern p = nullptr;
    ~PatternGuard() {
        if (p) abilu_pattern_destroy(p);
    }
};
struct FactorsGuard {
    abilu_factors f = nullptr;
    ~FactorsGuard() {
        if (f) abilu_factors_destroy(f);
    }
};

}  // namespace

static int grid_rows(int n, int per_cta) { return (n + per_cta - 1) / per_cta; }

// factors on p from X (pattern layout) and Dinv, then `sweeps` synchronous
// sweeps with the values Ap (p's layout); *out receives the handle
static abilu_status factors_from(abilu_pattern p, const double *X, const double *Dinv,
                                 const double *Ap, int sweeps, cudaStream_t st, abilu_factors *out) {
    abilu_factors f = nullptr;
    abilu_status s = abilu_factors_create(p, ABILU_F64, &f);
    if (s != ABILU_OK) return s;
    const int c = f->cur;
    k_import<double><<<counted(grid_rows(p->v.n, PLU_THREADS / 4)), PLU_THREADS, 0, st>>>(
        p->v, X, Dinv, static_cast<double *>(f->L[c]), static_cast<double *>(f->U[c]),
        static_cast<double *>(f->D[c]), static_cast<double *>(f->Udiag));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        abilu_factors_destroy(f);
        return cuda_fail(e, "k_import");
    }
    s = build_dispatch(f, Ap, sweeps, ABILU_SYNC, ABILU_INIT_FROM_PREVIOUS, st);
    if (s != ABILU_OK) {
        abilu_factors_destroy(f);
        return s;
    }
    *out = f;
    return ABILU_OK;
}

// largest t with #{keys of the side >= t} >= budget + 1, both sides at once,
// by bisection on the 64-bit patterns (64 counting passes)
static abilu_status select_thresholds(int n, const int32_t *rowptr, const int32_t *colind,
                                      const unsigned long long *key, long long bl, long long bu,
                                      bool need_l, bool need_u, unsigned long long *cnt,
                                      cudaStream_t st, unsigned long long *tl,
                                      unsigned long long *tu) {
    unsigned long long lo[2] = {0ull, 0ull}, hi[2] = {~0ull, ~0ull};
    const long long need[2] = {bl + 1, bu + 1};
    const bool act[2] = {need_l, need_u};
    for (int step = 0; step < 64; step++) {
        unsigned long long mid[2];
        for (int k = 0; k < 2; k++) mid[k] = lo[k] + (hi[k] - lo[k]) / 2 + ((hi[k] - lo[k]) & 1);
        ABILU_CUDA(cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), st));
        k_count_at_least<<<counted(grid_rows(n, 256)), 256, 0, st>>>(n, rowptr, colind, key, mid[0],
                                                                     mid[1], cnt);
        ABILU_LAUNCH_CHECK("k_count_at_least");
        unsigned long long h[2];
        ABILU_CUDA(cudaMemcpyAsync(h, cnt, sizeof h, cudaMemcpyDeviceToHost, st));
        ABILU_CUDA(cudaStreamSynchronize(st));
        for (int k = 0; k < 2; k++) {
            if (!act[k] || lo[k] == hi[k]) continue;
            if ((long long)h[k] >= need[k]) lo[k] = mid[k];
            else hi[k] = mid[k] - 1;
        }
    }
    *tl = lo[0];
    *tu = lo[1];
    return ABILU_OK;
}

// the final FP64 factors stored in `dtype` (FP32: with Dinv U for the upper
// sweeps): a new handle on the same pattern
template <typename T>
static abilu_status store_as(abilu_factors f64, abilu_dtype dtype, double *X, double *D,
                             cudaStream_t st, abilu_factors *out) {
    abilu_pattern p = f64->p;
    abilu_status s = export_dispatch(f64, X, D, st);
    if (s != ABILU_OK) return s;
    abilu_factors f = nullptr;
    if ((s = abilu_factors_create(p, dtype, &f)) != ABILU_OK) return s;
    const int c = f->cur;
    k_import<T><<<counted(grid_rows(p->v.n, PLU_THREADS / 4)), PLU_THREADS, 0, st>>>(
        p->v, X, D, static_cast<T *>(f->L[c]), static_cast<T *>(f->U[c]), static_cast<T *>(f->D[c]),
        static_cast<T *>(f->Udiag));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        abilu_factors_destroy(f);
        return cuda_fail(e, "k_import");
    }
    if ((s = form_scaled_upper(f, st)) != ABILU_OK) {
        abilu_factors_destroy(f);
        return s;
    }
    *out = f;
    return ABILU_OK;
}

static abilu_status read_total(const int32_t *ptr_n, const unsigned *err, cudaStream_t st,
                               int32_t *total) {
    unsigned e = 0;
    ABILU_CUDA(cudaMemcpyAsync(total, ptr_n, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    ABILU_CUDA(cudaMemcpyAsync(&e, err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    ABILU_CUDA(cudaStreamSynchronize(st));
    if (e & 1u) return fail(ABILU_EINVAL, "abilu_parilut: a row of L U exceeds %d blocks", PLU_MAX_ROW);
    if (e & (1u << 8)) return fail(ABILU_EINVAL, "abilu_parilut: more than 2^31 - 1 blocks");
    return ABILU_OK;
}

}  // namespace abilu

using namespace abilu;

extern "C" void abilu_parilut_default_opts(abilu_parilut_opts *o) {
    if (!o) return;
    o->fill = 2.0;
    o->iters = 3;
    o->sweeps = 2;
    o->factor_dtype = ABILU_F64;
}

extern "C" abilu_status abilu_parilut(abilu_pattern pA, const double *A,
                                      const abilu_parilut_opts *o, abilu_stream stream,
                                      abilu_pattern *pattern_out, abilu_factors *factors_out) {
    if (!pA || !A || !o || !pattern_out || !factors_out)
        return fail(ABILU_EINVAL, "abilu_parilut: NULL argument");
    *pattern_out = nullptr;
    *factors_out = nullptr;
    if ((reinterpret_cast<uintptr_t>(A) & 15u) != 0)
        return fail(ABILU_EINVAL, "abilu_parilut: A_vals must be 16-byte aligned");
    if (!(o->fill >= 0.0 && o->fill <= 1e9) || o->iters < 0 || o->sweeps < 0 ||
        (o->factor_dtype != ABILU_F64 && o->factor_dtype != ABILU_F32 && o->factor_dtype != ABILU_BF16))
        return fail(ABILU_EINVAL, "abilu_parilut: bad options");
    cudaStream_t st = S(stream);
    const PatternView &VA = pA->v;
    const int n = VA.n;
    const long long bl = (long long)(o->fill * (double)VA.nl), bu = (long long)(o->fill * (double)VA.nu);
    DevBufs bufs;
    unsigned *err = nullptr;
    unsigned long long *cnt = nullptr;
    long long *scratch = nullptr;
    int32_t *rowcnt = nullptr;
    double *D = nullptr;
    abilu_status s;
    if ((s = bufs.get(&err, 1)) != ABILU_OK || (s = bufs.get(&cnt, 2)) != ABILU_OK ||
        (s = bufs.get(&scratch, (size_t)n / 4096 + 2)) != ABILU_OK ||
        (s = bufs.get(&rowcnt, (size_t)n)) != ABILU_OK || (s = bufs.get(&D, (size_t)n * BB)) != ABILU_OK)
        return s;
    ABILU_CUDA(cudaMemsetAsync(err, 0, sizeof(unsigned), st));

    // start: X = A, `sweeps` synchronous sweeps on A's pattern
    PatternGuard pcur;   // the current pattern when owned (NULL: A's)
    double *X = nullptr;
    {
        FactorsGuard f0;
        if ((s = abilu_factors_create(pA, ABILU_F64, &f0.f)) != ABILU_OK) return s;
        if ((s = build_dispatch(f0.f, A, o->sweeps, ABILU_SYNC, ABILU_INIT_FROM_A, st)) != ABILU_OK) return s;
        if (o->iters == 0) {
            PatternGuard pc;
            if ((s = abilu_pattern_create(n, VA.nnzb, VA.rowptr, VA.colind, stream, &pc.p)) != ABILU_OK) return s;
            FactorsGuard fo;
            if ((s = abilu_factors_create(pc.p, ABILU_F64, &fo.f)) != ABILU_OK) return s;
            if ((s = build_dispatch(fo.f, A, o->sweeps, ABILU_SYNC, ABILU_INIT_FROM_A, st)) != ABILU_OK) return s;
            if (o->factor_dtype != ABILU_F64) {
                double *Xs = nullptr;
                if ((s = bufs.get(&Xs, (size_t)VA.nnzb * BB)) != ABILU_OK) return s;
                FactorsGuard fn;
                s = o->factor_dtype == ABILU_F32
                        ? store_as<float>(fo.f, ABILU_F32, Xs, D, st, &fn.f)
                        : store_as<__nv_bfloat16>(fo.f, ABILU_BF16, Xs, D, st, &fn.f);
                if (s != ABILU_OK) return s;
                std::swap(fo.f, fn.f);
            }
            ABILU_CUDA(cudaStreamSynchronize(st));
            *pattern_out = pc.p;
            *factors_out = fo.f;
            pc.p = nullptr;
            fo.f = nullptr;
            return ABILU_OK;
        }
        if ((s = bufs.get(&X, (size_t)VA.nnzb * BB)) != ABILU_OK) return s;
        if ((s = export_dispatch(f0.f, X, D, st)) != ABILU_OK) return s;
        ABILU_CUDA(cudaStreamSynchronize(st));
    }
    for (int it = 0; it < o->iters; it++) {
        const PatternView &VC = pcur.p ? pcur.p->v : VA;
        // fill: the pattern of L U
        int32_t *rp2 = nullptr, *ci2 = nullptr;
        if ((s = bufs.get(&rp2, (size_t)n + 1)) != ABILU_OK) return s;
        k_lu_pattern<false><<<counted(grid_rows(n, PLU_THREADS)), PLU_THREADS, 0, st>>>(
            n, VC.rowptr, VC.colind, VC.diagpos, rowcnt, nullptr, nullptr, err);
        ABILU_LAUNCH_CHECK("k_lu_pattern");
        if ((s = scan_i32(rowcnt, rp2, n, scratch, err, st)) != ABILU_OK) return s;
        int32_t nnz2 = 0;
        if ((s = read_total(rp2 + n, err, st, &nnz2)) != ABILU_OK) return s;
        if ((s = bufs.get(&ci2, (size_t)nnz2)) != ABILU_OK) return s;
        k_lu_pattern<true><<<counted(grid_rows(n, PLU_THREADS)), PLU_THREADS, 0, st>>>(
            n, VC.rowptr, VC.colind, VC.diagpos, nullptr, rp2, ci2, err);
        ABILU_LAUNCH_CHECK("k_lu_pattern");
        double *X2 = nullptr, *A2 = nullptr;
        if ((s = bufs.get(&X2, (size_t)nnz2 * BB)) != ABILU_OK) return s;
        if ((s = bufs.get(&A2, (size_t)nnz2 * BB)) != ABILU_OK) return s;
        k_map_blocks<<<counted(grid_rows(n, PLU_THREADS / 4)), PLU_THREADS, 0, st>>>(
            n, rp2, ci2, VC.rowptr, VC.colind, X, VA.rowptr, VA.colind, A, X2, A2);
        ABILU_LAUNCH_CHECK("k_map_blocks");
        PatternGuard p2;
        if ((s = abilu_pattern_create(n, nnz2, rp2, ci2, stream, &p2.p)) != ABILU_OK) return s;
        {
            FactorsGuard f2;
            if ((s = factors_from(p2.p, X2, D, A2, o->sweeps, st, &f2.f)) != ABILU_OK) return s;
            if ((s = export_dispatch(f2.f, X2, D, st)) != ABILU_OK) return s;
            ABILU_CUDA(cudaStreamSynchronize(st));
        }
        // drop: the largest strictly lower and strictly upper blocks
        const PatternView &V2 = p2.p->v;
        unsigned long long *key = nullptr;
        if ((s = bufs.get(&key, (size_t)nnz2)) != ABILU_OK) return s;
        k_block_norm2<<<counted(grid_rows(nnz2, 256)), 256, 0, st>>>(X2, nnz2, reinterpret_cast<double *>(key));
        ABILU_LAUNCH_CHECK("k_block_norm2");
        const bool all_l = (long long)V2.nl <= bl, all_u = (long long)V2.nu <= bu;
        unsigned long long tl = 0, tu = 0;
        if (!all_l || !all_u) {
            s = select_thresholds(n, V2.rowptr, V2.colind, key, bl, bu, !all_l, !all_u, cnt, st, &tl, &tu);
            if (s != ABILU_OK) return s;
        }
        int32_t *rp3 = nullptr, *ci3 = nullptr;
        if ((s = bufs.get(&rp3, (size_t)n + 1)) != ABILU_OK) return s;
        k_compact<false><<<counted(grid_rows(n, PLU_THREADS / 4)), PLU_THREADS, 0, st>>>(
            n, V2.rowptr, V2.colind, key, tl, tu, all_l, all_u, rowcnt, nullptr, nullptr, nullptr,
            nullptr, nullptr, nullptr);
        ABILU_LAUNCH_CHECK("k_compact");
        if ((s = scan_i32(rowcnt, rp3, n, scratch, err, st)) != ABILU_OK) return s;
        int32_t nnz3 = 0;
        if ((s = read_total(rp3 + n, err, st, &nnz3)) != ABILU_OK) return s;
        double *X3 = nullptr, *A3 = nullptr;
        if ((s = bufs.get(&ci3, (size_t)nnz3)) != ABILU_OK) return s;
        if ((s = bufs.get(&X3, (size_t)nnz3 * BB)) != ABILU_OK) return s;
        if ((s = bufs.get(&A3, (size_t)nnz3 * BB)) != ABILU_OK) return s;
        k_compact<true><<<counted(grid_rows(n, PLU_THREADS / 4)), PLU_THREADS, 0, st>>>(
            n, V2.rowptr, V2.colind, key, tl, tu, all_l, all_u, nullptr, rp3, ci3, X2, A2, X3, A3);
        ABILU_LAUNCH_CHECK("k_compact");
        PatternGuard p3;
        if ((s = abilu_pattern_create(n, nnz3, rp3, ci3, stream, &p3.p)) != ABILU_OK) return s;
        FactorsGuard f3;
        if ((s = factors_from(p3.p, X3, D, A3, o->sweeps, st, &f3.f)) != ABILU_OK) return s;
        if (it == o->iters - 1) {
            if (o->factor_dtype != ABILU_F64) {
                FactorsGuard fn;
                s = o->factor_dtype == ABILU_F32
                        ? store_as<float>(f3.f, ABILU_F32, X3, D, st, &fn.f)
                        : store_as<__nv_bfloat16>(f3.f, ABILU_BF16, X3, D, st, &fn.f);
                if (s != ABILU_OK) return s;
                std::swap(f3.f, fn.f);   // the FP64 factors are released with fn
            }
            ABILU_CUDA(cudaStreamSynchronize(st));
            *pattern_out = p3.p;
            *factors_out = f3.f;
            p3.p = nullptr;
            f3.f = nullptr;
            return ABILU_OK;
        }
        if ((s = export_dispatch(f3.f, X3, D, st)) != ABILU_OK) return s;
        ABILU_CUDA(cudaStreamSynchronize(st));
        X = X3;
        std::swap(pcur.p, p3.p);   // the old current pattern is released with p3
    }
    return fail(ABILU_EINVAL, "abilu_parilut: unreachable");
}
