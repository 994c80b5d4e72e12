// Aggregation multigrid with block ILU smoothing.
//
// The paper's closing section names asynchronous block ILU iterations as
// fine-grain parallel multigrid smoothers (and the study of their smoothing
// property) as future work, without fixing a cycle.  This file provides one: a
// V-cycle on a hierarchy of Galerkin coarse operators, whose smoother on every
// level is x += M^{-1}(b - A x), M = L U the block ILU(0) of that level's
// matrix, computed by the build sweeps and applied by the triangular sweeps of
// build.cu / apply.cu (synchronous or asynchronous, any factor precision).
//
// Hierarchy (abilu_mg_create, host code, once per pattern):
//   strength  ||A_ij||_F^2 of every block, formed on the device in storage
//             order without contraction, compared on the host;
//   aggregation, greedy: in row i, j != i is strong when ||A_ij||^2 > 0 and
//             ||A_ij||^2 >= theta^2 max_{k != i} ||A_ik||^2.  Pass 1 (cells
//             ascending): an unplaced cell with a strong coupling and no placed
//             strong neighbour roots an aggregate of itself and its strong
//             neighbours.  Pass 2: a leftover cell joins the pass-1 aggregate of
//             its strongest placed neighbour (lowest column on ties), else
//             becomes an aggregate of its own.  Numbered in creation order;
//   transfer  piecewise constant: P_{i,agg(i)} = I_4, restriction P^T;
//   coarse    A_c = P^T A P: coarse block (I,J) = sum of the fine blocks (i,j)
//             with agg(i) = I, agg(j) = J, added in ascending fine position.
// Coarsening stops at max_levels, at or below min_coarse cells, or when an
// aggregation no longer reduces the cell count.
//
// Numeric set-up (abilu_mg_setup): the coarse values on the device (a quad per
// coarse block, fixed order), then every level's block ILU build.
//
// Cycle (abilu_mg_apply, fgmres_solve_mg): on level l from x = 0,
//   pre_smooth smoothing steps, b_c = P^T (b - A x), the cycle on level l+1,
//   x += P x_c, post_smooth steps; the coarsest level takes coarse_smooth
//   steps.  The first step from x = 0 is x = M^{-1} b (no residual pass).
//   Kernels: the residual (the SpMV's FMA chain, spmv.cuh; a quad per row,
//   coalesced), the restriction (a quad per aggregate summing its cells'
//   residuals in ascending order), the prolongation, x += z.
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "spmv.cuh"

namespace abilu {

abilu_status build_dispatch(abilu_factors f, const double *A, int nsweeps, abilu_mode mode,
                            abilu_init init, cudaStream_t st);
abilu_status apply_dispatch(abilu_factors f, const double *r, const float *r32, double *z,
                            int nl, int nu, abilu_mode mode, cudaStream_t st, Skip skip);
abilu_status fgmres_run(const PatternView &P, const double *A, abilu_factors ws, const Precond &pc,
                        const double *b, double *x, const fgmres_opts *opts, fgmres_result *res,
                        cudaStream_t st, abilu_factors const *cnt, int ncnt);
abilu_status fgmres_check_opts(const fgmres_opts *opts, const char *who);
abilu_status export_dispatch(abilu_factors f, double *X, double *Dinv, cudaStream_t st);

constexpr int MG_THREADS = 256;
constexpr int MG_ROWS = MG_THREADS / 4;   // quads per CTA

// w[p] = ||A_p||_F^2: the 16 entries in storage order, products and sums
// rounded separately (the host compares these values against each other)
__global__ void __launch_bounds__(MG_THREADS)
k_block_norm2(const double *__restrict__ A, long long nnzb, double *__restrict__ w) {
    const long long p = (long long)blockIdx.x * MG_THREADS + threadIdx.x;
    if (p >= nnzb) return;
    const double2 *a = reinterpret_cast<const double2 *>(A + (size_t)p * BB);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < BB / 2; k++) {
        const double2 v = a[k];
        s = __dadd_rn(s, __dmul_rn(v.x, v.x));
        s = __dadd_rn(s, __dmul_rn(v.y, v.y));
    }
    w[p] = s;
}

// Ac[c] = sum of A[gidx[t]], t = gptr[c] .. gptr[c+1]-1 (ascending fine
// positions); a quad per coarse block, thread q sums row q.  Up to four fine
// blocks are loaded before they are added (in list order), so the gathers of
// a coarse block overlap instead of forming a chain.
__global__ void __launch_bounds__(MG_THREADS)
k_galerkin(long long nnzb_c, const int *__restrict__ gptr, const int *__restrict__ gidx,
           const double *__restrict__ A, double *__restrict__ Ac) {
    pdl_wait();
    pdl_trigger();
    const long long c = ((long long)blockIdx.x * MG_THREADS + threadIdx.x) >> 2;
    const int q = threadIdx.x & 3;
    if (c >= nnzb_c) return;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    const int t1 = gptr[c + 1];
    for (int t = gptr[c]; t < t1; t += 4) {
        double v[4][4];
#pragma unroll
        for (int u = 0; u < 4; u++)
            if (t + u < t1) ld_row(A + (size_t)__ldg(gidx + t + u) * BB + q * BS, v[u]);
#pragma unroll
        for (int u = 0; u < 4; u++)
            if (t + u < t1) {
#pragma unroll
                for (int k = 0; k < 4; k++) s[k] = __dadd_rn(s[k], v[u][k]);
            }
    }
    st_row(Ac + (size_t)c * BB + q * BS, s);
}

// r = b - A x, a quad per block row
__global__ void __launch_bounds__(MG_THREADS)
k_mg_residual(PatternView P, const double *__restrict__ A, const double *__restrict__ b,
              const double *__restrict__ x, double *__restrict__ r, Skip skip) {
    pdl_wait();
    pdl_trigger();
    if (skip_all(skip)) return;
    const int i = blockIdx.x * MG_ROWS + (threadIdx.x >> 2), q = threadIdx.x & 3;
    if (i >= P.n) return;
    const size_t o = (size_t)i * BS + q;
    r[o] = b[o] - row_dot_blocks(P, A, x, i, q);
}

// Restriction bc = P^T r: bc[I] = sum over the cells i of aggregate I, in
// ascending order, of r_i.  A quad per aggregate, thread q sums component q;
// up to four members' entries are loaded before they are added in order.
__global__ void __launch_bounds__(MG_THREADS)
k_mg_restrict(const double *__restrict__ r, const int *__restrict__ mptr,
              const int *__restrict__ mem, int nc, double *__restrict__ bc, Skip skip) {
    pdl_wait();
    pdl_trigger();
    if (skip_all(skip)) return;
    const int I = blockIdx.x * MG_ROWS + (threadIdx.x >> 2), q = threadIdx.x & 3;
    if (I >= nc) return;
    double s = 0.0;
    const int t1 = mptr[I + 1];
    for (int t = mptr[I]; t < t1; t += 4) {
        double v[4];
#pragma unroll
        for (int u = 0; u < 4; u++)
            if (t + u < t1) v[u] = __ldg(r + (size_t)__ldg(mem + t + u) * BS + q);
#pragma unroll
        for (int u = 0; u < 4; u++)
            if (t + u < t1) s += v[u];
    }
    bc[(size_t)I * BS + q] = s;
}

// x_i += x_c[agg(i)] (ASSIGN: x_i = x_c[agg(i)], x was zero)
template <bool ASSIGN>
__global__ void __launch_bounds__(MG_THREADS)
k_mg_prolong(const int *__restrict__ agg, const double *__restrict__ xc, double *__restrict__ x,
             long long n4, Skip skip) {
    pdl_wait();
    pdl_trigger();
    if (skip_all(skip)) return;
    for (long long e = (long long)blockIdx.x * MG_THREADS + threadIdx.x; e < n4;
         e += (long long)gridDim.x * MG_THREADS) {
        const double v = xc[(size_t)agg[e >> 2] * BS + (e & 3)];
        if constexpr (ASSIGN) x[e] = v;
        else x[e] += v;
    }
}

// x += z
__global__ void __launch_bounds__(MG_THREADS)
k_mg_axpy(double *__restrict__ x, const double *__restrict__ z, long long n2, Skip skip) {
    pdl_wait();
    pdl_trigger();
    if (skip_all(skip)) return;
    double2 *x2 = reinterpret_cast<double2 *>(x);
    const double2 *z2 = reinterpret_cast<const double2 *>(z);
    for (long long e = (long long)blockIdx.x * MG_THREADS + threadIdx.x; e < n2;
         e += (long long)gridDim.x * MG_THREADS) {
        const double2 a = x2[e], d = z2[e];
        x2[e] = make_double2(a.x + d.x, a.y + d.y);
    }
}

// ------------------------------------------------------------------ handle

struct MgLevel {
    abilu_pattern p = nullptr;   // level 0: the caller's pattern (not owned)
    abilu_factors f = nullptr;   // this level's block ILU factors (owned)
    const double *A = nullptr;   // level 0: the values of the last set-up; else owned (Ac)
    double *Ac = nullptr;        // owned coarse values
    int n = 0;
    long long nnzb = 0;
    // transfer to the next level (all NULL on the coarsest)
    int *agg = nullptr;          // [n] aggregate of each cell
    int *mptr = nullptr, *mem = nullptr;   // [nc+1], [n]: cells of each aggregate, ascending
    int *gptr = nullptr, *gidx = nullptr;  // [nnzb_c+1], [nnzb]: fine blocks of each coarse block
    // vectors, double[n][4]: right-hand side and solution (coarse levels; level
    // 0 uses the caller's), residual and smoother correction
    double *b = nullptr, *x = nullptr, *r = nullptr, *z = nullptr;
};

}  // namespace abilu

struct abilu_mg_s {
    abilu_mg_opts o;
    int device;
    int nlevels;
    abilu::MgLevel L[ABILU_MG_MAX_LEVELS];
    std::vector<void *> dev;     // device allocations
};

namespace abilu {

static void mg_free(abilu_mg mg) {
    if (!mg) return;
    for (int l = 0; l < mg->nlevels; l++) {
        if (mg->L[l].f) abilu_factors_destroy(mg->L[l].f);
        if (l > 0 && mg->L[l].p) abilu_pattern_destroy(mg->L[l].p);
    }
    for (void *p : mg->dev) cudaFree(p);
    delete mg;
}

template <typename T> static abilu_status mg_alloc(abilu_mg mg, T **out, size_t count) {
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, sizeof(T) * (count > 0 ? count : 1));
    if (e != cudaSuccess) return cuda_fail(e, "abilu_mg_create: cudaMalloc");
    mg->dev.push_back(p);
    *out = static_cast<T *>(p);
    return ABILU_OK;
}

// The aggregation rule of the file header, on host arrays; returns the
// number of aggregates.  w[p] = ||A_p||_F^2.
static int aggregate_host(int n, const std::vector<int> &rowptr, const std::vector<int> &colind,
                          const std::vector<double> &w, double theta, std::vector<int> &agg) {
    const double t2 = theta * theta;
    std::vector<double> rmax(n, 0.0);
    for (int i = 0; i < n; i++)
        for (int p = rowptr[i]; p < rowptr[i + 1]; p++)
            if (colind[p] != i && w[p] > rmax[i]) rmax[i] = w[p];
    auto strong = [&](int i, int p) { return colind[p] != i && w[p] > 0.0 && w[p] >= t2 * rmax[i]; };
    agg.assign(n, -1);
    int nc = 0;
    for (int i = 0; i < n; i++) {   // pass 1: roots
        if (agg[i] >= 0) continue;
        bool any = false, free_nbrs = true;
        for (int p = rowptr[i]; p < rowptr[i + 1]; p++)
            if (strong(i, p)) {
                any = true;
                if (agg[colind[p]] >= 0) free_nbrs = false;
            }
        if (!any || !free_nbrs) continue;
        agg[i] = nc;
        for (int p = rowptr[i]; p < rowptr[i + 1]; p++)
            if (strong(i, p)) agg[colind[p]] = nc;
        nc++;
    }
    const std::vector<int> first(agg);
    for (int i = 0; i < n; i++) {   // pass 2: leftovers
        if (first[i] >= 0) continue;
        int best = -1;
        for (int p = rowptr[i]; p < rowptr[i + 1]; p++) {
            const int j = colind[p];
            if (j == i || first[j] < 0) continue;
            if (best < 0 || w[p] > w[best]) best = p;
        }
        agg[i] = best >= 0 ? first[colind[best]] : nc++;
    }
    return nc;
}

// Coarse pattern of P^T A P and the transfer lists, on the host.
struct Coarse {
    std::vector<int> rowptr, colind;   // coarse pattern
    std::vector<int> mptr, mem;        // cells of each aggregate
    std::vector<int> gptr, gidx;       // fine blocks summed into each coarse block
};

static void coarse_host(int n, const std::vector<int> &rowptr, const std::vector<int> &colind,
                        const std::vector<int> &agg, int nc, Coarse &c) {
    c.mptr.assign(nc + 1, 0);
    for (int i = 0; i < n; i++) c.mptr[agg[i] + 1]++;
    for (int I = 0; I < nc; I++) c.mptr[I + 1] += c.mptr[I];
    c.mem.resize(n);
    {
        std::vector<int> pos(c.mptr.begin(), c.mptr.end() - 1);
        for (int i = 0; i < n; i++) c.mem[pos[agg[i]]++] = i;
    }
    // coarse columns of each aggregate: the aggregates of its cells' neighbours
    c.rowptr.assign(nc + 1, 0);
    c.colind.clear();
    std::vector<int> mark(nc, -1);
    for (int I = 0; I < nc; I++) {
        const size_t start = c.colind.size();
        for (int t = c.mptr[I]; t < c.mptr[I + 1]; t++) {
            const int i = c.mem[t];
            for (int p = rowptr[i]; p < rowptr[i + 1]; p++) {
                const int J = agg[colind[p]];
                if (mark[J] != I) {
                    mark[J] = I;
                    c.colind.push_back(J);
                }
            }
        }
        std::sort(c.colind.begin() + start, c.colind.end());
        c.rowptr[I + 1] = (int)c.colind.size();
    }
    // each fine block's coarse position, then a stable counting sort
    const long long nnzb = rowptr[n];
    std::vector<int> cpos(nnzb);
    for (int i = 0; i < n; i++) {
        const int I = agg[i];
        const int *b0 = c.colind.data() + c.rowptr[I], *b1 = c.colind.data() + c.rowptr[I + 1];
        for (int p = rowptr[i]; p < rowptr[i + 1]; p++)
            cpos[p] = (int)(std::lower_bound(b0, b1, agg[colind[p]]) - c.colind.data());
    }
    const int nnzc = (int)c.colind.size();
    c.gptr.assign(nnzc + 1, 0);
    for (long long p = 0; p < nnzb; p++) c.gptr[cpos[p] + 1]++;
    for (int k = 0; k < nnzc; k++) c.gptr[k + 1] += c.gptr[k];
    c.gidx.resize(nnzb);
    std::vector<int> fill(c.gptr.begin(), c.gptr.end() - 1);
    for (long long p = 0; p < nnzb; p++) c.gidx[fill[cpos[p]]++] = (int)p;
}

template <typename T>
static abilu_status upload(abilu_mg mg, T **dst, const std::vector<T> &src, cudaStream_t st) {
    abilu_status s = mg_alloc(mg, dst, src.size());
    if (s != ABILU_OK) return s;
    if (!src.empty())
        ABILU_CUDA(cudaMemcpyAsync(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice, st));
    return ABILU_OK;
}

static int grid_of(long long threads) { return (int)((threads + MG_THREADS - 1) / MG_THREADS); }

// coarse values of level l + 1 from level l's
static abilu_status galerkin_values(abilu_mg mg, int l, cudaStream_t st) {
    MgLevel &F = mg->L[l], &Cl = mg->L[l + 1];
    if (Cl.nnzb == 0) return ABILU_OK;
    launch_pdl(k_galerkin, grid_of(4 * Cl.nnzb), MG_THREADS, 0, st, Cl.nnzb, F.gptr, F.gidx, F.A, Cl.Ac);
    ABILU_LAUNCH_CHECK("k_galerkin");
    return ABILU_OK;
}

}  // namespace abilu

// ------------------------------------------------------------------- cycle

namespace abilu {

// `steps` smoothing steps x += M^{-1}(b - A x) on level l; *xzero says x is
// (still) zero and not yet written: the first step is then x = M^{-1} b
static abilu_status smooth(abilu_mg mg, int l, int steps, const double *b, double *x, bool *xzero,
                           cudaStream_t st, Skip skip) {
    MgLevel &L = mg->L[l];
    const abilu_mg_opts &o = mg->o;
    const abilu_mode mode = (abilu_mode)o.mode;
    for (int k = 0; k < steps; k++) {
        abilu_status s;
        if (*xzero) {
            s = apply_dispatch(L.f, b, nullptr, x, o.apply_sweeps_lower, o.apply_sweeps_upper, mode,
                               st, skip);
            if (s != ABILU_OK) return s;
            *xzero = false;
            continue;
        }
        launch_pdl(k_mg_residual, grid_of(4LL * L.n), MG_THREADS, 0, st, L.p->v, L.A, b, x, L.r, skip);
        ABILU_LAUNCH_CHECK("k_mg_residual");
        s = apply_dispatch(L.f, L.r, nullptr, L.z, o.apply_sweeps_lower, o.apply_sweeps_upper, mode,
                           st, skip);
        if (s != ABILU_OK) return s;
        const long long n2 = 2LL * L.n;
        launch_pdl(k_mg_axpy, grid_of(n2), MG_THREADS, 0, st, x, L.z, n2, skip);
        ABILU_LAUNCH_CHECK("k_mg_axpy");
    }
    return ABILU_OK;
}

// x = the V-cycle from level l applied to b
static abilu_status vcycle(abilu_mg mg, int l, const double *b, double *x, cudaStream_t st,
                           Skip skip) {
    MgLevel &L = mg->L[l];
    const abilu_mg_opts &o = mg->o;
    bool xzero = true;
    abilu_status s;
    if (l == mg->nlevels - 1) {
        s = smooth(mg, l, o.coarse_smooth, b, x, &xzero, st, skip);
        if (s == ABILU_OK && xzero)
            ABILU_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * 4 * (size_t)L.n, st));
        return s;
    }
    MgLevel &Cl = mg->L[l + 1];
    if ((s = smooth(mg, l, o.pre_smooth, b, x, &xzero, st, skip)) != ABILU_OK) return s;
    const double *rf = b;   // the fine residual: b itself while x = 0
    if (!xzero) {
        launch_pdl(k_mg_residual, grid_of(4LL * L.n), MG_THREADS, 0, st, L.p->v, L.A, b, x, L.r, skip);
        ABILU_LAUNCH_CHECK("k_mg_residual");
        rf = L.r;
    }
    launch_pdl(k_mg_restrict, grid_of(4LL * Cl.n), MG_THREADS, 0, st, rf, L.mptr, L.mem, Cl.n, Cl.b,
        skip);
    ABILU_LAUNCH_CHECK("k_mg_restrict");
    if ((s = vcycle(mg, l + 1, Cl.b, Cl.x, st, skip)) != ABILU_OK) return s;
    const long long n4 = 4LL * L.n;
    if (xzero)
        launch_pdl(k_mg_prolong<true>, grid_of(n4), MG_THREADS, 0, st, L.agg, Cl.x, x, n4, skip);
    else
        launch_pdl(k_mg_prolong<false>, grid_of(n4), MG_THREADS, 0, st, L.agg, Cl.x, x, n4, skip);
    ABILU_LAUNCH_CHECK("k_mg_prolong");
    xzero = false;
    return smooth(mg, l, o.post_smooth, b, x, &xzero, st, skip);
}

static abilu_status mg_pc(void *ctx, const double *v, const float *, double *z, cudaStream_t st,
                          Skip skip) {
    abilu_mg mg = static_cast<abilu_mg>(ctx);
    return vcycle(mg, 0, v, z, st, skip);
}

static abilu_status mg_setup(abilu_mg mg, const double *A, cudaStream_t st) {
    mg->L[0].A = A;
    for (int l = 0; l + 1 < mg->nlevels; l++) {
        abilu_status s = galerkin_values(mg, l, st);
        if (s != ABILU_OK) return s;
    }
    for (int l = 0; l < mg->nlevels; l++) {
        abilu_status s = build_dispatch(mg->L[l].f, mg->L[l].A, mg->o.build_sweeps,
                                        (abilu_mode)mg->o.mode, (abilu_init)mg->o.init, st);
        if (s != ABILU_OK) return s;
    }
    return ABILU_OK;
}

static inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Builds the hierarchy (host aggregation level by level; every coarse level's
// strengths come from its Galerkin values) and allocates every level.
static abilu_status mg_build_hierarchy(abilu_mg mg, abilu_pattern p, const double *A, cudaStream_t st) {
    const abilu_mg_opts &o = mg->o;
    MgLevel &L0 = mg->L[0];
    L0.p = p;
    L0.A = A;
    L0.n = p->v.n;
    L0.nnzb = p->v.nnzb;
    mg->nlevels = 1;
    std::vector<int> rp(L0.n + 1), ci(L0.nnzb);
    ABILU_CUDA(cudaMemcpyAsync(rp.data(), p->v.rowptr, sizeof(int) * rp.size(), cudaMemcpyDeviceToHost, st));
    ABILU_CUDA(cudaMemcpyAsync(ci.data(), p->v.colind, sizeof(int) * ci.size(), cudaMemcpyDeviceToHost, st));
    double *wdev = nullptr;
    abilu_status s;
    while (mg->nlevels < o.max_levels && mg->L[mg->nlevels - 1].n > o.min_coarse) {
        MgLevel &F = mg->L[mg->nlevels - 1];
        if (!wdev && (s = mg_alloc(mg, &wdev, (size_t)L0.nnzb)) != ABILU_OK) return s;
        k_block_norm2<<<counted(grid_of(F.nnzb)), MG_THREADS, 0, st>>>(F.A, F.nnzb, wdev);
        ABILU_LAUNCH_CHECK("k_block_norm2");
        std::vector<double> w(F.nnzb);
        ABILU_CUDA(cudaMemcpyAsync(w.data(), wdev, sizeof(double) * w.size(), cudaMemcpyDeviceToHost, st));
        ABILU_CUDA(cudaStreamSynchronize(st));
        std::vector<int> agg;
        const int nc = aggregate_host(F.n, rp, ci, w, o.theta, agg);
        if (nc >= F.n) break;
        Coarse c;
        coarse_host(F.n, rp, ci, agg, nc, c);
        if ((s = upload(mg, &F.agg, agg, st)) != ABILU_OK) return s;
        if ((s = upload(mg, &F.mptr, c.mptr, st)) != ABILU_OK) return s;
        if ((s = upload(mg, &F.mem, c.mem, st)) != ABILU_OK) return s;
        if ((s = upload(mg, &F.gptr, c.gptr, st)) != ABILU_OK) return s;
        if ((s = upload(mg, &F.gidx, c.gidx, st)) != ABILU_OK) return s;
        int *rpd = nullptr, *cid = nullptr;
        if ((s = upload(mg, &rpd, c.rowptr, st)) != ABILU_OK) return s;
        if ((s = upload(mg, &cid, c.colind, st)) != ABILU_OK) return s;
        MgLevel &Cl = mg->L[mg->nlevels];
        s = abilu_pattern_create(nc, (int32_t)c.colind.size(), rpd, cid, st, &Cl.p);
        if (s != ABILU_OK) return s;
        mg->nlevels++;   // from here on mg_free releases Cl.p
        Cl.n = nc;
        Cl.nnzb = (long long)c.colind.size();
        if ((s = mg_alloc(mg, &Cl.Ac, (size_t)Cl.nnzb * BB)) != ABILU_OK) return s;
        Cl.A = Cl.Ac;
        if ((s = galerkin_values(mg, mg->nlevels - 2, st)) != ABILU_OK) return s;
        rp.swap(c.rowptr);
        ci.swap(c.colind);
    }
    for (int l = 0; l < mg->nlevels; l++) {
        MgLevel &L = mg->L[l];
        if ((s = abilu_factors_create(L.p, (abilu_dtype)o.factor_dtype, &L.f)) != ABILU_OK) return s;
        const size_t nv = 4 * (size_t)L.n;
        if ((s = mg_alloc(mg, &L.r, nv)) != ABILU_OK) return s;
        if ((s = mg_alloc(mg, &L.z, nv)) != ABILU_OK) return s;
        if (l > 0) {
            if ((s = mg_alloc(mg, &L.b, nv)) != ABILU_OK) return s;
            if ((s = mg_alloc(mg, &L.x, nv)) != ABILU_OK) return s;
        }
    }
    ABILU_CUDA(cudaStreamSynchronize(st));
    return ABILU_OK;
}

}  // namespace abilu

using namespace abilu;

extern "C" void abilu_mg_default_opts(abilu_mg_opts *o) {
    if (!o) return;
    o->max_levels = 10;
    o->min_coarse = 512;
    o->theta = 0.25;
    o->factor_dtype = ABILU_F32;
    o->build_sweeps = 4;
    o->apply_sweeps_lower = 2;
    o->apply_sweeps_upper = 2;
    o->pre_smooth = 1;
    o->post_smooth = 1;
    o->coarse_smooth = 2;
    o->mode = ABILU_SYNC;
    o->init = ABILU_INIT_FROM_A;
}

extern "C" abilu_status abilu_mg_create(abilu_pattern p, const double *A, const abilu_mg_opts *o,
                                        abilu_stream stream, abilu_mg *out) {
    if (!p || !A || !o || !out) return fail(ABILU_EINVAL, "abilu_mg_create: NULL argument");
    *out = nullptr;
    if (!aligned16(A)) return fail(ABILU_EINVAL, "abilu_mg_create: A_vals must be 16-byte aligned");
    if (o->max_levels < 1 || o->max_levels > ABILU_MG_MAX_LEVELS || o->min_coarse < 1 ||
        !(o->theta >= 0.0 && o->theta <= 1.0) ||
        (o->factor_dtype != ABILU_F64 && o->factor_dtype != ABILU_F32 && o->factor_dtype != ABILU_BF16) ||
        o->build_sweeps < 0 || o->apply_sweeps_lower < 0 || o->apply_sweeps_upper < 0 ||
        o->pre_smooth < 0 || o->post_smooth < 0 || o->coarse_smooth < 0 ||
        (o->mode != ABILU_SYNC && o->mode != ABILU_ASYNC) ||
        (o->init != ABILU_INIT_FROM_A && o->init != ABILU_INIT_FROM_PREVIOUS))
        return fail(ABILU_EINVAL, "abilu_mg_create: bad options");
    abilu_mg mg = new abilu_mg_s();
    mg->o = *o;
    cudaGetDevice(&mg->device);
    abilu_status s = mg_build_hierarchy(mg, p, A, S(stream));
    if (s != ABILU_OK) {
        mg_free(mg);
        return s;
    }
    *out = mg;
    return ABILU_OK;
}

extern "C" void abilu_mg_destroy(abilu_mg mg) { mg_free(mg); }

extern "C" abilu_status abilu_mg_setup(abilu_mg mg, const double *A, abilu_stream stream) {
    if (!mg || !A) return fail(ABILU_EINVAL, "abilu_mg_setup: NULL argument");
    if (!aligned16(A)) return fail(ABILU_EINVAL, "abilu_mg_setup: A_vals must be 16-byte aligned");
    return mg_setup(mg, A, S(stream));
}

extern "C" abilu_status abilu_mg_apply(abilu_mg mg, const double *r, double *z, abilu_stream stream) {
    if (!mg || !r || !z) return fail(ABILU_EINVAL, "abilu_mg_apply: NULL argument");
    if (r == z) return fail(ABILU_EINVAL, "abilu_mg_apply: r and z must be distinct");
    if (!aligned16(r) || !aligned16(z))
        return fail(ABILU_EINVAL, "abilu_mg_apply: vectors must be 16-byte aligned");
    return vcycle(mg, 0, r, z, S(stream), Skip{});
}

extern "C" abilu_status abilu_mg_levels(abilu_mg mg, int64_t *out) {
    if (!mg || !out) return fail(ABILU_EINVAL, "abilu_mg_levels: NULL argument");
    memset(out, 0, sizeof(int64_t) * (2 * ABILU_MG_MAX_LEVELS + 1));
    out[0] = mg->nlevels;
    for (int l = 0; l < mg->nlevels; l++) {
        out[1 + 2 * l] = mg->L[l].n;
        out[2 + 2 * l] = mg->L[l].nnzb;
    }
    return ABILU_OK;
}

extern "C" abilu_status abilu_mg_level_data(abilu_mg mg, int32_t level, int32_t *agg,
                                            int32_t *rowptr, int32_t *colind, double *vals,
                                            double *X, double *Dinv, abilu_stream stream) {
    if (!mg || level < 0 || level >= mg->nlevels)
        return fail(ABILU_EINVAL, "abilu_mg_level_data: bad handle or level");
    const MgLevel &L = mg->L[level];
    cudaStream_t st = S(stream);
    if (agg) {
        if (!L.agg) return fail(ABILU_EINVAL, "abilu_mg_level_data: the coarsest level has no aggregates");
        ABILU_CUDA(cudaMemcpyAsync(agg, L.agg, sizeof(int) * L.n, cudaMemcpyDeviceToDevice, st));
    }
    if (rowptr)
        ABILU_CUDA(cudaMemcpyAsync(rowptr, L.p->v.rowptr, sizeof(int) * (L.n + 1), cudaMemcpyDeviceToDevice, st));
    if (colind)
        ABILU_CUDA(cudaMemcpyAsync(colind, L.p->v.colind, sizeof(int) * L.nnzb, cudaMemcpyDeviceToDevice, st));
    if (vals)
        ABILU_CUDA(cudaMemcpyAsync(vals, L.A, sizeof(double) * BB * L.nnzb, cudaMemcpyDeviceToDevice, st));
    if (X || Dinv) {
        if ((X && !aligned16(X)) || (Dinv && !aligned16(Dinv)))
            return fail(ABILU_EINVAL, "abilu_mg_level_data: X and Dinv must be 16-byte aligned");
        return export_dispatch(L.f, X, Dinv, st);
    }
    return ABILU_OK;
}

extern "C" abilu_status fgmres_solve_mg(abilu_mg mg, const double *A, const double *b, double *x,
                                        const fgmres_opts *opts, fgmres_result *res,
                                        abilu_stream stream) {
    if (!mg || !A || !b || !x || !opts || !res) return fail(ABILU_EINVAL, "fgmres_solve_mg: NULL argument");
    memset(res, 0, sizeof *res);
    abilu_status s = fgmres_check_opts(opts, "fgmres_solve_mg");
    if (s != ABILU_OK) return s;
    cudaStream_t st = S(stream);
    abilu_factors cnt[ABILU_MG_MAX_LEVELS];
    unsigned long long keep[ABILU_MG_MAX_LEVELS];
    for (int l = 0; l < mg->nlevels; l++) {   // the solve's spin limit on every level
        cnt[l] = mg->L[l].f;
        keep[l] = cnt[l]->spin_limit;
        cnt[l]->spin_limit = (unsigned long long)opts->spin_limit;
    }
    if (!opts->build || (s = mg_setup(mg, A, st)) == ABILU_OK) {
        const Precond pc{mg_pc, mg, nullptr};
        s = fgmres_run(mg->L[0].p->v, A, mg->L[0].f, pc, b, x, opts, res, st, cnt, mg->nlevels);
    }
    for (int l = 0; l < mg->nlevels; l++) cnt[l]->spin_limit = keep[l];
    return s;
}
