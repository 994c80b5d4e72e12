// Right-preconditioned flexible GMRES(m) (Saad's FGMRES, which the paper uses
// through PETSc with restart 30, Sec. 2 and Sec. 6 setup), FP64 on the device.
//
// Per Arnoldi step j:  z_j = M^{-1} v_j (block ILU sweeps, any precision),
// w = A z_j (FP64 SpMV), classical Gram-Schmidt h = V^T w, w -= V h (one pass,
// or two with reorth), h_{j+1,j} = ||w|| (for rtol >= 1e-7 formed with the dot
// products in one reduction, see k_spmv_dots and gs_form_for), Givens rotation
// of the new column, residual estimate |g_{j+1}|, v_{j+1} = w / h_{j+1,j}.  At
// the end of a cycle y = R^{-1} g, x += Z y, and the true residual b - A x is
// formed in FP64; an estimate that passed but is not confirmed by it restarts
// the cycle.
//
// Every reduction runs on a fixed grid with a fixed order (per-thread partial
// sums, a block sum staged in shared memory, per-CTA partials, and the last
// CTA to finish adding the partials in CTA order), so a synchronous-mode solve
// is bit-reproducible run to run.  The small Hessenberg/Givens state lives on
// the device; the last CTA of each reduction updates it, so the host only
// enqueues kernels.  The host learns that a cycle ended from a pinned
// host-mapped status word, read one step late (after step j+1 is already
// enqueued), so the GPU never idles on the host; kernels of steps past the
// end of a cycle see the device flag and return at once.
#include <math.h>
#include <string.h>

#include "common.cuh"
#include "reduce.cuh"
#include "spmv.cuh"

namespace abilu {

abilu_status build_dispatch(abilu_factors f, const double *A, int nsweeps, abilu_mode mode,
                            abilu_init init, cudaStream_t st);
abilu_status apply_dispatch(abilu_factors f, const double *r, const float *r32, double *z,
                            int nl, int nu, abilu_mode mode, cudaStream_t st, Skip skip);
abilu_status apply_dispatch_ready(abilu_factors f, const double *r, const float *r32, double *z,
                                  int nl, int nu, abilu_mode mode, cudaStream_t st, Skip skip);
bool apply_y_ready(abilu_factors f, int nl, int nu, abilu_mode mode);
abilu_status ensure_krylov(abilu_factors f, int m);
int red_ctas();

constexpr int MAXM = 64;
constexpr int TILE = 6;   // Krylov vectors per pass of the dot kernel (64 registers)

struct HostStatus {       // pinned, host-mapped mirror
    int done, iters, converged, kdim, restarts, breakdown;
    double est, beta, bnorm;
    unsigned long long nsing, ntimeout;   // factor handles' counters at the end of a solve
};

struct SolveState {       // device
    double H[MAXM * MAXM]; // R after rotations, H[i*MAXM + j], i <= j
    double cs[MAXM], sn[MAXM], g[MAXM + 1];
    double h[MAXM + 1];    // current column (first Gram-Schmidt pass)
    double h2[MAXM + 1];   // second pass (reorthogonalisation)
    double bnorm, beta, hn_inv, est, rtol;
    int done, iters, max_iters, converged, kdim, restarts, m, breakdown;
    unsigned counter;      // last-CTA detection for the reductions
    HostStatus *hs;        // host-mapped mirror
};

__device__ __forceinline__ void publish(SolveState *S) {
    HostStatus *h = S->hs;
    volatile HostStatus *vh = h;
    vh->done = S->done;
    vh->iters = S->iters;
    vh->converged = S->converged;
    vh->kdim = S->kdim;
    vh->restarts = S->restarts;
    vh->breakdown = S->breakdown;
    vh->est = S->est;
    vh->beta = S->beta;
    vh->bnorm = S->bnorm;
    __threadfence_system();
}

// In the first CTA of the kernel after a Gram-Schmidt step or a residual: that
// kernel's status to the host-mapped mirror (see givens_column)
__device__ __forceinline__ void publish_early(SolveState *S) {
    if (blockIdx.x == 0 && threadIdx.x == 0) publish(S);
}

// last-CTA election after this CTA stored its partials
__device__ __forceinline__ bool last_cta(SolveState *S) {
    __shared__ bool am_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) am_last = atomicAdd(&S->counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (am_last) __threadfence();
    return am_last;
}

// In the last CTA: out[k] = sum over CTAs c of partials[c*stride + k0 + k],
// k < kn <= TILE.  Thread t adds the partials of CTAs t, t+256, ... in that
// order (the loads of R of them issued before their adds), then a fixed-order
// block reduction: deterministic for a fixed grid.  Every thread of the CTA
// calls it.
// R: CTAs whose partials are loaded before any add
template <int K, int R = (K <= 2 ? 4 : 1)>
__device__ __forceinline__ void reduce_partials(const double *partials, int stride, int k0,
                                                int kn, double *sh_w, double *out) {
    double v[K];
#pragma unroll
    for (int k = 0; k < K; k++) v[k] = 0.0;
    for (int c0 = threadIdx.x; c0 < (int)gridDim.x; c0 += R * blockDim.x) {
        double t[R][K];
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int c = c0 + r * blockDim.x;
            const double *p = partials + (size_t)c * stride + k0;
#pragma unroll
            for (int k = 0; k < K; k++) t[r][k] = (c < (int)gridDim.x && k < kn) ? __ldcg(p + k) : 0.0;
        }
#pragma unroll
        for (int r = 0; r < R; r++)
#pragma unroll
            for (int k = 0; k < K; k++) v[k] += t[r][k];
    }
    block_sum<K>(v, sh_w, out, kn);
}

// ---------------------------------------------------------------- residual
// r = b - A x into r_out (= V_0 unnormalised), ||r||^2 and (init) ||b||^2.
// The last CTA sets beta, the convergence flag and starts the next cycle.
// Launched with 3 CTAs per SM (its registers allow 3 resident: one wave).
// Every FP64 operation counts on this GPU (two FP64 lanes per SM): with x = 0
// (ZERO) r = b and ||r||^2 = ||b||^2 is accumulated once, and r_out is not
// written (the caller scales b itself); after a cycle (init = 0) ||b||^2 is
// not formed.
template <bool ZERO>
__global__ void __launch_bounds__(RED_THREADS, 3)
k_residual(PatternView P, const double *__restrict__ A, const double *__restrict__ b,
           const double *__restrict__ x, double *__restrict__ r_out, SolveState *S,
           double *partials, int init) {
    pdl_wait();
    pdl_trigger();
    // a restart after a cycle in which no step ran (the initial guess had
    // already converged) would recompute the same residual: keep the state
    if (!init && S->kdim == 0) return;
    __shared__ double sh_w[RED_THREADS * 2], sh_o[2];
    const int q = threadIdx.x & 3;
    double v[2] = {0.0, 0.0};
    const int rows_per_grid = gridDim.x * (RED_THREADS / 4);
    int i = blockIdx.x * (RED_THREADS / 4) + (threadIdx.x >> 2);
    if constexpr (ZERO) {
        // r = b, not stored (the scale kernel that forms v_0 = r / beta reads
        // b itself); ||b||^2 with four rows' loads in flight per thread (one
        // per iteration left each thread waiting on a load 18 times in a
        // row: 24 us for the 512x512 grid); the same rows in the same order
        constexpr int U = 4;
        for (; i < P.n; i += U * rows_per_grid) {
            double bu[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int iu = i + u * rows_per_grid;
                bu[u] = iu < P.n ? b[(size_t)iu * BS + q] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int iu = i + u * rows_per_grid;
                if (iu >= P.n) break;
                v[0] += bu[u] * bu[u];
            }
        }
        v[1] = v[0];
    } else {
        for (; i < P.n; i += rows_per_grid) {
            const size_t o = (size_t)i * BS + q;
            // b issued with the row's matrix loads (after the product: 81.7
            // against 78.6 us per launch at 512x512, ncu)
            const double bi = __ldg(b + o);
            // the SpMV kernel's arithmetic
            const double s = row_dot_blocks(P, A, x, i, q);
            const double ri = bi - s;
            r_out[o] = ri;
            v[0] += ri * ri;
            if (init) v[1] += bi * bi;
        }
    }
    block_sum<2>(v, sh_w, sh_o, 2);
    if (threadIdx.x == 0) {
        partials[blockIdx.x * 2 + 0] = sh_o[0];
        partials[blockIdx.x * 2 + 1] = sh_o[1];
    }
    if (!last_cta(S)) return;
    // the last CTA: g_1.. zeroed by the whole CTA, the scalars staged while
    // the partials are reduced; thread 0's chain then reads no global memory,
    // and the status is published by the next kernel's first CTA (k_scale)
    for (int k = 1 + threadIdx.x; k <= MAXM; k += blockDim.x) S->g[k] = 0.0;
    __shared__ double sh_b[2];   // bnorm (restart), rtol
    __shared__ int sh_i[2];      // iters, max_iters
    switch (threadIdx.x) {
    case 0: sh_b[0] = S->bnorm; break;
    case 1: sh_b[1] = S->rtol; break;
    case 2: sh_i[0] = S->iters; break;
    case 3: sh_i[1] = S->max_iters; break;
    default: break;
    }
    reduce_partials<2>(partials, 2, 0, 2, sh_w, sh_o);
    if (threadIdx.x == 0) {
        const double rr = sh_o[0];
        const double bnorm = init ? sqrt(sh_o[1]) : sh_b[0];
        if (init) S->bnorm = bnorm;
        else S->restarts += 1;
        const double beta = sqrt(rr);
        S->beta = beta;
        S->hn_inv = beta > 0.0 ? 1.0 / beta : 0.0;
        const int converged = (beta <= sh_b[1] * bnorm || bnorm == 0.0) ? 1 : 0;
        S->converged = converged;
        S->done = (converged || sh_i[0] >= sh_i[1]) ? 1 : 0;
        S->kdim = 0;
        S->breakdown = 0;
        S->g[0] = beta;
        if (init) S->est = bnorm > 0.0 ? beta / bnorm : 0.0;
        S->counter = 0;
    }
}

// the preconditioner's ticket counters zeroed for its next application
// (Precond::tickets; the kernels that write its right-hand side)
__device__ __forceinline__ void zero_tickets(unsigned long long *tk) {
    if (tk && blockIdx.x == 0 && threadIdx.x < 2) tk[threadIdx.x] = 0ull;
}

// v_out = v_in * S->hn_inv; with FP32/BF16 factors also v32 = (float) v_out,
// the right-hand side the next preconditioner application reads (and the
// same into y0, the application's in-place iterate, when given)
__global__ void __launch_bounds__(RED_THREADS)
k_scale(const double *vin, double *vout, float *v32, long long nv2, SolveState *S, float *y0,
        unsigned long long *tk) {
    pdl_wait();
    pdl_trigger();
    publish_early(S);      // the previous kernel's status (k_residual: a new cycle's)
    if (S->done) return;   // set by an earlier kernel: a plain load
    zero_tickets(tk);
    const double s = S->hn_inv;
    const double2 *a = reinterpret_cast<const double2 *>(vin);
    double2 *o = reinterpret_cast<double2 *>(vout);
    float2 *o32 = reinterpret_cast<float2 *>(v32);
    // four grid strides per iteration: four loads in flight per thread before
    // any store (a streaming kernel with a few elements per thread is bound by
    // the loads it keeps in flight)
    constexpr int U = 4;
    const long long st = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nv2; e += U * st) {
        double2 t[U];
#pragma unroll
        for (int u = 0; u < U; u++)
            if (e + u * st < nv2) t[u] = a[e + u * st];
#pragma unroll
        for (int u = 0; u < U; u++) {
            if (e + u * st >= nv2) break;
            const double2 r = make_double2(t[u].x * s, t[u].y * s);
            o[e + u * st] = r;
            if (v32) {
                const float2 f = make_float2(to_f32_int(r.x), to_f32_int(r.y));
                o32[e + u * st] = f;
                if (y0) reinterpret_cast<float2 *>(y0)[e + u * st] = f;
            }
        }
    }
}

// Partial dot products of K consecutive basis vectors with w for this CTA.
// K is a compile-time width so no predicated-off FP64 FMA is issued.
template <int K, bool PIPE>
__device__ __forceinline__ void dots_tile(const double2 *__restrict__ V2, long long nv2,
                                          int k0, const double2 *__restrict__ w2,
                                          double *sh_w, double *sh_o, double *partials) {
    double acc[K];
#pragma unroll
    for (int k = 0; k < K; k++) acc[k] = 0.0;
    const long long st = (long long)gridDim.x * blockDim.x;
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    // PIPE (the kernels of one to four basis vectors): software-pipelined, the
    // next element's loads issued before this element's FMAs, so the FP64 work
    // overlaps the memory latency instead of following it (both take
    // microseconds here); the accumulation order (e, e + st, e + 2 st, ...) is
    // the plain loop's, so each thread's sums are the same bit for bit
    if constexpr (PIPE) {
        if (e < nv2) {
            double2 wn = w2[e], vn[K];
#pragma unroll
            for (int k = 0; k < K; k++) vn[k] = V2[(size_t)(k0 + k) * nv2 + e];
            for (;;) {
                const double2 wc = wn;
                double2 vc[K];
#pragma unroll
                for (int k = 0; k < K; k++) vc[k] = vn[k];
                const long long en = e + st;
                if (en < nv2) {
                    wn = w2[en];
#pragma unroll
                    for (int k = 0; k < K; k++) vn[k] = V2[(size_t)(k0 + k) * nv2 + en];
                }
#pragma unroll
                for (int k = 0; k < K; k++) acc[k] = fma(vc[k].y, wc.y, fma(vc[k].x, wc.x, acc[k]));
                e = en;
                if (e >= nv2) break;
            }
        }
    } else if constexpr (K <= 4) {
        // two grid strides per iteration, twice the loads in flight, same
        // accumulation order (the general kernel has no registers left to
        // pipeline)
        for (; e + st < nv2; e += 2 * st) {
            const double2 wa = w2[e], wb = w2[e + st];
            double2 va[K], vb[K];
#pragma unroll
            for (int k = 0; k < K; k++) {
                va[k] = V2[(size_t)(k0 + k) * nv2 + e];
                vb[k] = V2[(size_t)(k0 + k) * nv2 + e + st];
            }
#pragma unroll
            for (int k = 0; k < K; k++) {
                acc[k] = fma(va[k].y, wa.y, fma(va[k].x, wa.x, acc[k]));
                acc[k] = fma(vb[k].y, wb.y, fma(vb[k].x, wb.x, acc[k]));
            }
        }
    }
    for (; e < nv2; e += st) {   // wide tiles (K + 1 loads in flight already) and tails
        const double2 wv = w2[e];
#pragma unroll
        for (int k = 0; k < K; k++) {
            const double2 v = V2[(size_t)(k0 + k) * nv2 + e];
            acc[k] = fma(v.y, wv.y, fma(v.x, wv.x, acc[k]));
        }
    }
    block_sum<K>(acc, sh_w, sh_o, K);
    if (threadIdx.x < K) partials[(size_t)blockIdx.x * (MAXM + 2) + k0 + threadIdx.x] = sh_o[threadIdx.x];
}

// The Givens update of column j of the Hessenberg matrix (from the
// Gram-Schmidt coefficients h, plus h2 after a second pass) with
// h_{j+1,j} = hn, the residual estimate and the end-of-cycle test.  One
// thread of the last CTA.  With `pub` the status goes to the host-mapped
// mirror here; otherwise the next kernel's first CTA publishes it at its start
// (publish_early), off this kernel's serial tail: the system-scope fence of
// the host-mapped stores then overlaps that kernel's work.
__device__ __forceinline__ void givens_column(SolveState *S, int j, int two_pass, double hn,
                                              bool pub = true) {
    // the previous rotations, i = 0 .. j-1, each mixing entries i and i+1 of
    // the new column: entry i+1 is still the Gram-Schmidt coefficient when
    // rotation i reaches it, so one carried value replaces a column array
    // (which lived in local memory)
    double a = S->h[0] + (two_pass ? S->h2[0] : 0.0);
    for (int i = 0; i < j; i++) {
        const double c = S->h[i + 1] + (two_pass ? S->h2[i + 1] : 0.0);
        S->H[i * MAXM + j] = S->cs[i] * a + S->sn[i] * c;
        a = -S->sn[i] * a + S->cs[i] * c;
    }
    const double c = hn;
    const double d = sqrt(a * a + c * c);
    double cs = 1.0, sn = 0.0;
    if (d != 0.0) { cs = a / d; sn = c / d; }
    S->cs[j] = cs;
    S->sn[j] = sn;
    S->H[j * MAXM + j] = cs * a + sn * c;
    const double gj = S->g[j];
    S->g[j + 1] = -sn * gj;
    S->g[j] = cs * gj;
    S->iters += 1;
    S->kdim = j + 1;
    S->est = fabs(S->g[j + 1]) / S->bnorm;
    S->breakdown = hn == 0.0 ? 1 : 0;
    S->done = (fabs(S->g[j + 1]) <= S->rtol * S->bnorm || hn == 0.0 ||
               S->iters >= S->max_iters || j + 1 >= S->m) ? 1 : 0;
    S->hn_inv = hn != 0.0 ? 1.0 / hn : 0.0;
    S->counter = 0;
    if (pub) publish(S);
}

// What givens_column reads of the solve state besides the new column, staged
// in shared memory by the last CTA of a reduction while it reduces the
// partials, so that the serial FP64 chain of one thread reads no global
// memory (an FP64 operation takes 64 cycles on this GPU and an L2 load
// several hundred; with the loads in the chain the update took 4-9 us)
struct GivensIn {
    double cs[MAXM], sn[MAXM], gj, bnorm, rtol;
    int iters, max_iters, m;
};
__device__ __forceinline__ void givens_stage(const SolveState *S, int j, GivensIn *G) {
    for (int i = threadIdx.x; i < j; i += blockDim.x) {
        G->cs[i] = S->cs[i];
        G->sn[i] = S->sn[i];
    }
    switch (threadIdx.x) {
    case 0: G->gj = S->g[j]; break;
    case 1: G->bnorm = S->bnorm; break;
    case 2: G->rtol = S->rtol; break;
    case 3: G->iters = S->iters; break;
    case 4: G->max_iters = S->max_iters; break;
    case 5: G->m = S->m; break;
    default: break;
    }
}

// givens_column (one pass, the status published by the next kernel) from the
// staged inputs and the coefficients h[0..j] in shared memory: the same
// operations in the same order, so the same results bit for bit
__device__ __forceinline__ void givens_column_staged(SolveState *S, int j, const double *h,
                                                     const GivensIn *G, double hn) {
    // independent of the rotations: overlaps their chain
    S->hn_inv = hn != 0.0 ? 1.0 / hn : 0.0;
    double a = h[0];
    for (int i = 0; i < j; i++) {
        const double c = h[i + 1];
        S->H[i * MAXM + j] = G->cs[i] * a + G->sn[i] * c;
        a = -G->sn[i] * a + G->cs[i] * c;
    }
    const double c = hn;
    const double d = sqrt(a * a + c * c);
    double cs = 1.0, sn = 0.0;
    if (d != 0.0) { cs = a / d; sn = c / d; }
    S->cs[j] = cs;
    S->sn[j] = sn;
    S->H[j * MAXM + j] = cs * a + sn * c;
    const double gj = G->gj;
    const double g1 = -sn * gj;
    S->g[j + 1] = g1;
    S->g[j] = cs * gj;
    const int iters = G->iters + 1;
    S->iters = iters;
    S->kdim = j + 1;
    S->est = fabs(g1) / G->bnorm;
    S->breakdown = hn == 0.0 ? 1 : 0;
    S->done = (fabs(g1) <= G->rtol * G->bnorm || hn == 0.0 || iters >= G->max_iters ||
               j + 1 >= G->m) ? 1 : 0;
    S->counter = 0;
}


// The last CTA of a dot-product pass: h[k] = sum over CTAs of the partials of
// slot k, k < jp1, in tiles of T (pass 0 -> S->h, pass 1 -> S->h2).  sh_w
// holds RED_THREADS * T doubles.
template <int T>
__device__ __forceinline__ void dots_last(SolveState *S, const double *partials, int jp1, int pass,
                                          double *sh_w, double *sh_o) {
    double *h = pass == 0 ? S->h : S->h2;
    for (int k0 = 0; k0 < jp1; k0 += T) {
        const int kn = jp1 - k0 < T ? jp1 - k0 : T;
        reduce_partials<T>(partials, MAXM + 2, k0, kn, sh_w, sh_o);
        if (threadIdx.x < kn) h[k0 + threadIdx.x] = sh_o[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0) S->counter = 0;
}

// The last CTA of a single-reduction step (one classical Gram-Schmidt pass and
// one reduction, the solve's default for rtol >= 1e-7, gs_form_for): the dots
// of slots k < jp1 and ||w||^2 (slot jp1) reduced in tiles of T, the last tile
// with the norm; the Givens inputs staged while the partials are reduced;
// every thread's partials loaded before any add (R CTAs per thread in one
// round); then h_{j+1,j} = sqrt(||w||^2 - sum_k h_k^2) (Pythagoras: w - V h is
// orthogonal to V_0..V_j when they are orthonormal, so the norm needs neither
// a pass over the updated w nor a second reduction) and the Givens update of
// column j by one thread.  sh_w holds RED_THREADS * (T + 1) doubles.  A
// difference below 1e-12 ||w||^2 (more than twelve digits cancelled, or
// negative) is taken as a breakdown: the cycle ends at this column and the
// explicit FP64 residual at its end decides whether it restarts.
template <int T>
__device__ __forceinline__ void dots_norm_last(SolveState *S, const double *partials, int jp1,
                                               double *sh_w, double *sh_o) {
    __shared__ GivensIn G;
    __shared__ double sh_h[MAXM + 1], sh_ww;
    givens_stage(S, jp1 - 1, &G);
    for (int k0 = 0; k0 < jp1; k0 += T) {
        const int kn = jp1 - k0 < T ? jp1 - k0 : T;
        const bool lastt = k0 + T >= jp1;
        reduce_partials<T + 1, (T + 1 <= 5 ? 3 : 2)>(partials, MAXM + 2, k0,
                                                     lastt ? kn + 1 : kn, sh_w, sh_o);
        if (threadIdx.x < kn) {
            S->h[k0 + threadIdx.x] = sh_o[threadIdx.x];
            sh_h[k0 + threadIdx.x] = sh_o[threadIdx.x];
        }
        if (lastt && threadIdx.x == 0) sh_ww = sh_o[kn];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const double ww = sh_ww;
    double hh = 0.0;
    for (int k = 0; k < jp1; k++) hh = fma(sh_h[k], sh_h[k], hh);
    const double d = ww - hh;
    givens_column_staged(S, jp1 - 1, sh_h, &G, d > 1e-12 * ww ? sqrt(d) : 0.0);   // the next kernel publishes
}

// h[k] = <V_k, w>, k < jp1 (pass 0 -> S->h, pass 1 -> S->h2).  The grid is
// 4 CTAs per SM and all of them must be resident at once (one wave), so the
// kernel is held to 64 registers.  NW = 0: any jp1, in tiles of up to TILE
// vectors; NW = 1 .. 4: jp1 == NW, one software-pipelined tile (its own
// kernel, so the general one keeps its register allocation; five vectors
// would spill).
template <int NW>
__global__ void __launch_bounds__(RED_THREADS, 4)
k_dots(const double *__restrict__ V, long long nv2, int jp1, const double *__restrict__ w,
       SolveState *S, double *partials, int pass) {
    pdl_wait();
    pdl_trigger();
    if (S->done) return;   // set by an earlier kernel: a plain load
    constexpr int T = NW > 0 ? NW : TILE;
    __shared__ double sh_w[RED_THREADS * T], sh_o[T];
    const double2 *w2 = reinterpret_cast<const double2 *>(w);
    const double2 *V2 = reinterpret_cast<const double2 *>(V);
    if constexpr (NW > 0) {
        dots_tile<NW, true>(V2, nv2, 0, w2, sh_w, sh_o, partials);
    } else {
        for (int k0 = 0; k0 < jp1; k0 += TILE) {
            switch (jp1 - k0 < TILE ? jp1 - k0 : TILE) {
            case 1: dots_tile<1, false>(V2, nv2, k0, w2, sh_w, sh_o, partials); break;
            case 2: dots_tile<2, false>(V2, nv2, k0, w2, sh_w, sh_o, partials); break;
            case 3: dots_tile<3, false>(V2, nv2, k0, w2, sh_w, sh_o, partials); break;
            case 4: dots_tile<4, false>(V2, nv2, k0, w2, sh_w, sh_o, partials); break;
            case 5: dots_tile<5, false>(V2, nv2, k0, w2, sh_w, sh_o, partials); break;
            default: dots_tile<6, false>(V2, nv2, k0, w2, sh_w, sh_o, partials); break;
            }
        }
    }
    if (!last_cta(S)) return;
    dots_last<T>(S, partials, jp1, pass, sh_w, sh_o);
}

// k_dots for jp1 basis vectors (the pipelined kernels for one to four)
static void launch_dots(int nred, cudaStream_t st, const double *V, long long nv2, int jp1,
                        const double *w, SolveState *S, double *partials, int pass) {
    if (jp1 == 1)
        launch_pdl(k_dots<1>, nred, RED_THREADS, 0, st, V, nv2, jp1, w, S, partials, pass);
    else if (jp1 == 2)
        launch_pdl(k_dots<2>, nred, RED_THREADS, 0, st, V, nv2, jp1, w, S, partials, pass);
    else if (jp1 == 3)
        launch_pdl(k_dots<3>, nred, RED_THREADS, 0, st, V, nv2, jp1, w, S, partials, pass);
    else if (jp1 == 4)
        launch_pdl(k_dots<4>, nred, RED_THREADS, 0, st, V, nv2, jp1, w, S, partials, pass);
    else
        launch_pdl(k_dots<0>, nred, RED_THREADS, 0, st, V, nv2, jp1, w, S, partials, pass);
}

// Partial dots <V_k0+k, w>, k < K, over this thread's rows of the fused
// kernel's grid stride (the same value-to-thread map as its product pass), for
// the tiles past the first: w was written earlier in the same kernel by this
// thread, so it is read back through L2 (never the read-only path).
template <int K>
__device__ __forceinline__ void rows_dots_tile(int n, const double *__restrict__ V, long long nv,
                                               int k0, const double *w, double *sh_w, double *sh_o,
                                               double *partials) {
    double acc[K];
#pragma unroll
    for (int k = 0; k < K; k++) acc[k] = 0.0;
    const int q = threadIdx.x & 3;
    const int rows_per_grid = gridDim.x * (RED_THREADS / 4);
    for (int i = blockIdx.x * (RED_THREADS / 4) + (threadIdx.x >> 2); i < n; i += rows_per_grid) {
        const size_t o = (size_t)i * BS + q;
        const double wv = __ldcg(w + o);
#pragma unroll
        for (int k = 0; k < K; k++) acc[k] = fma(__ldg(V + (size_t)(k0 + k) * nv + o), wv, acc[k]);
    }
    block_sum<K>(acc, sh_w, sh_o, K);
    if (threadIdx.x < K) partials[(size_t)blockIdx.x * (MAXM + 2) + k0 + threadIdx.x] = sh_o[threadIdx.x];
}

// w = A z_j and, in the same pass over the rows, the first Gram-Schmidt pass's
// dots h[k] = <V_k, w> for the first KF basis vectors, plus ||w||^2 with NORM
// (the single-reduction step): each product is consumed where it is formed, so
// w is written once and not read back by a second kernel, and one launch ramp
// and tail go per step.  Both halves are bound by the FP64 pipe (two lanes
// per SM), which they now share.  A quad of threads per block row as in the
// SpMV kernel (row q of each 4x4 block, the same FMA chain, spmv.cuh), rows
// in a grid stride.  KF = j + 1 <= SPMV_DOTS_MAX; WIDE (KF = SPMV_DOTS_MAX,
// any wider step): the tiles of V_KF..V_j follow in the same kernel, each a
// pass over the thread's own rows that re-reads its entries of w through L2.
// Per thread the sums run over its rows in order, then the block sum; the
// last CTA reduces the partials (slots 0..j, the norm in slot j + 1) and with
// NORM forms h_{j+1,j} and the Givens update, so the result is deterministic
// for a fixed grid.  Launched like the residual kernel, 3 CTAs per SM in one
// wave: 80 registers hold a row's four blocks, its x gathers and the basis
// entries in flight (at 64 registers and 4 CTAs per SM every width spilled,
// and the solve was 0.5% slower).  SPMV_DOTS_MAX = 3: with four and five
// basis vectors in the product's pass the accumulators spilled and the FP64
// pipe's busy share fell from 89-92% to 84%; three there and the rest in a
// tile that re-reads w measured 1.661 against 1.666 ms per solve.
constexpr int SPMV_DOTS_MAX = 3;
template <int KF, bool NORM, bool WIDE>
__global__ void __launch_bounds__(RED_THREADS, 3)
k_spmv_dots(PatternView P, const double *__restrict__ A, const double *__restrict__ z,
            double *w, const double *__restrict__ V, long long nv, int jp1, SolveState *S,
            double *partials) {
    pdl_wait();
    pdl_trigger();
    if (S->done) return;   // set by an earlier kernel: a plain load
    constexpr int KA = KF + (NORM ? 1 : 0);
    constexpr int T = WIDE ? TILE : KF;   // the tail's reduction tiles
    static_assert(KA <= TILE + 1, "the product pass's values fit the tail's staging");
    __shared__ double sh_w[RED_THREADS * (T + 1)], sh_o[T + 1];
    const int q = threadIdx.x & 3;
    double acc[KA];
#pragma unroll
    for (int k = 0; k < KA; k++) acc[k] = 0.0;
    const int rows_per_grid = gridDim.x * (RED_THREADS / 4);
    for (int i = blockIdx.x * (RED_THREADS / 4) + (threadIdx.x >> 2); i < P.n; i += rows_per_grid) {
        const size_t o = (size_t)i * BS + q;
        double v[KF];   // issued with the row's matrix loads
#pragma unroll
        for (int k = 0; k < KF; k++) v[k] = __ldg(V + (size_t)k * nv + o);
        const double s = row_dot_blocks(P, A, z, i, q);
        w[o] = s;
#pragma unroll
        for (int k = 0; k < KF; k++) acc[k] = fma(v[k], s, acc[k]);
        if constexpr (NORM) acc[KF] = fma(s, s, acc[KF]);
    }
    block_sum<KA>(acc, sh_w, sh_o, KA);
    double *pc = partials + (size_t)blockIdx.x * (MAXM + 2);
    if (threadIdx.x < KF) pc[threadIdx.x] = sh_o[threadIdx.x];
    if (NORM && threadIdx.x == 0) pc[WIDE ? jp1 : KF] = sh_o[KF];   // the norm's slot: j + 1
    if constexpr (WIDE) {
        for (int k0 = KF; k0 < jp1; k0 += TILE) {
            switch (jp1 - k0 < TILE ? jp1 - k0 : TILE) {
            case 1: rows_dots_tile<1>(P.n, V, nv, k0, w, sh_w, sh_o, partials); break;
            case 2: rows_dots_tile<2>(P.n, V, nv, k0, w, sh_w, sh_o, partials); break;
            case 3: rows_dots_tile<3>(P.n, V, nv, k0, w, sh_w, sh_o, partials); break;
            case 4: rows_dots_tile<4>(P.n, V, nv, k0, w, sh_w, sh_o, partials); break;
            case 5: rows_dots_tile<5>(P.n, V, nv, k0, w, sh_w, sh_o, partials); break;
            default: rows_dots_tile<6>(P.n, V, nv, k0, w, sh_w, sh_o, partials); break;
            }
        }
    }
    if (!last_cta(S)) return;
    if constexpr (NORM) dots_norm_last<T>(S, partials, jp1, sh_w, sh_o);   // k_update_scale publishes
    else dots_last<T>(S, partials, jp1, 0, sh_w, sh_o);
}

// k_spmv_dots for step j (jp1 = j + 1 basis vectors)
template <bool NORM>
static void launch_spmv_dots_n(int grid, cudaStream_t st, const PatternView &P, const double *A,
                               const double *z, double *w, const double *V, long long nv, int jp1,
                               SolveState *S, double *partials) {
    switch (jp1) {
    case 1: launch_pdl(k_spmv_dots<1, NORM, false>, grid, RED_THREADS, 0, st, P, A, z, w, V, nv, jp1, S, partials); break;
    case 2: launch_pdl(k_spmv_dots<2, NORM, false>, grid, RED_THREADS, 0, st, P, A, z, w, V, nv, jp1, S, partials); break;
    case 3: launch_pdl(k_spmv_dots<3, NORM, false>, grid, RED_THREADS, 0, st, P, A, z, w, V, nv, jp1, S, partials); break;
    default: launch_pdl(k_spmv_dots<3, NORM, true>, grid, RED_THREADS, 0, st, P, A, z, w, V, nv, jp1, S, partials); break;
    }
}
static_assert(SPMV_DOTS_MAX == 3, "one instance per width up to SPMV_DOTS_MAX");

// v_{j+1} = (w - sum_k h[k] V_k) * hn_inv and its FP32 copy (the next
// preconditioner's input) in one pass; w itself is not written back.  J =
// 1 .. 3: j + 1 == J, software-pipelined like update_pipelined; 0: any j.
template <int J>
__global__ void __launch_bounds__(RED_THREADS, 4)
k_update_scale(const double *__restrict__ V, long long nv2, int j, const double *__restrict__ w,
               double *__restrict__ vnext, float *__restrict__ v32, SolveState *S,
               float *__restrict__ y0, unsigned long long *tk) {
    pdl_wait();
    pdl_trigger();
    publish_early(S);      // the previous kernel's step status
    if (S->done) return;   // the cycle ended at this column: no next vector
    zero_tickets(tk);
    __shared__ double sh_h[MAXM + 1];
    const int jp1 = j + 1;
    for (int k = threadIdx.x; k < jp1; k += blockDim.x) sh_h[k] = S->h[k];
    __syncthreads();
    const double sc = S->hn_inv;
    const double2 *w2 = reinterpret_cast<const double2 *>(w);
    const double2 *V2 = reinterpret_cast<const double2 *>(V);
    double2 *o2 = reinterpret_cast<double2 *>(vnext);
    float2 *o32 = reinterpret_cast<float2 *>(v32);
    float2 *y2 = reinterpret_cast<float2 *>(y0);
    const long long st = (long long)gridDim.x * blockDim.x;
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    auto out = [&](long long i, double2 t) {
        const double2 r = make_double2(t.x * sc, t.y * sc);
        o2[i] = r;
        if (v32) {
            const float2 f = make_float2(to_f32_int(r.x), to_f32_int(r.y));
            o32[i] = f;
            if (y2) y2[i] = f;
        }
    };
    if constexpr (J > 0) {
        if (e >= nv2) return;
        double h[J];
#pragma unroll
        for (int k = 0; k < J; k++) h[k] = sh_h[k];
        double2 wn = w2[e], vn[J];
#pragma unroll
        for (int k = 0; k < J; k++) vn[k] = V2[(size_t)k * nv2 + e];
        for (;;) {
            double2 t = wn, vc[J];
#pragma unroll
            for (int k = 0; k < J; k++) vc[k] = vn[k];
            const long long en = e + st;
            if (en < nv2) {
                wn = w2[en];
#pragma unroll
                for (int k = 0; k < J; k++) vn[k] = V2[(size_t)k * nv2 + en];
            }
#pragma unroll
            for (int k = 0; k < J; k++) {
                t.x -= h[k] * vc[k].x;
                t.y -= h[k] * vc[k].y;
            }
            out(e, t);
            e = en;
            if (e >= nv2) break;
        }
        return;
    }
    for (; e + st < nv2; e += 2 * st) {  // two grid strides per iteration
        double2 ta = w2[e], tb = w2[e + st];
        for (int k = 0; k < jp1; k++) {
            const double2 va = V2[(size_t)k * nv2 + e], vb = V2[(size_t)k * nv2 + e + st];
            ta.x -= sh_h[k] * va.x;
            ta.y -= sh_h[k] * va.y;
            tb.x -= sh_h[k] * vb.x;
            tb.y -= sh_h[k] * vb.y;
        }
        out(e, ta);
        out(e + st, tb);
    }
    if (e < nv2) {
        double2 t = w2[e];
        for (int k = 0; k < jp1; k++) {
            const double2 v = V2[(size_t)k * nv2 + e];
            t.x -= sh_h[k] * v.x;
            t.y -= sh_h[k] * v.y;
        }
        out(e, t);
    }
}

static void launch_update_scale(int nred, cudaStream_t st, const double *V, long long nv2, int j,
                                const double *w, double *vnext, float *v32, SolveState *S,
                                float *y0, unsigned long long *tk) {
    switch (j + 1) {
    case 1: launch_pdl(k_update_scale<1>, nred, RED_THREADS, 0, st, V, nv2, j, w, vnext, v32, S, y0, tk); break;
    case 2: launch_pdl(k_update_scale<2>, nred, RED_THREADS, 0, st, V, nv2, j, w, vnext, v32, S, y0, tk); break;
    case 3: launch_pdl(k_update_scale<3>, nred, RED_THREADS, 0, st, V, nv2, j, w, vnext, v32, S, y0, tk); break;
    default: launch_pdl(k_update_scale<0>, nred, RED_THREADS, 0, st, V, nv2, j, w, vnext, v32, S, y0, tk); break;
    }
}

// w_e -= sum_k h[k] V_k,e for this thread's elements e (grid stride), J = j + 1
// basis vectors, software-pipelined: the next element's loads are issued
// before this element's FMAs, so the FP64 work overlaps the memory latency.
// Same operations in the same order as the plain loop (bit for bit).
template <int J>
__device__ __forceinline__ void update_pipelined(const double2 *__restrict__ V2, long long nv2,
                                                 double2 *__restrict__ w2, const double *sh_h,
                                                 double &nrm) {
    const long long st = (long long)gridDim.x * blockDim.x;
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nv2) return;
    double h[J];
#pragma unroll
    for (int k = 0; k < J; k++) h[k] = sh_h[k];
    double2 wn = w2[e], vn[J];
#pragma unroll
    for (int k = 0; k < J; k++) vn[k] = V2[(size_t)k * nv2 + e];
    for (;;) {
        double2 t = wn, vc[J];
#pragma unroll
        for (int k = 0; k < J; k++) vc[k] = vn[k];
        const long long en = e + st;
        if (en < nv2) {
            wn = w2[en];
#pragma unroll
            for (int k = 0; k < J; k++) vn[k] = V2[(size_t)k * nv2 + en];
        }
#pragma unroll
        for (int k = 0; k < J; k++) {
            t.x -= h[k] * vc[k].x;
            t.y -= h[k] * vc[k].y;
        }
        w2[e] = t;
        nrm = fma(t.y, t.y, fma(t.x, t.x, nrm));
        e = en;
        if (e >= nv2) break;
    }
}

// w -= sum_k h[k] V_k; on the final pass also ||w||^2, and the last CTA
// performs the Givens update of column j and the convergence test.  J = 0:
// any j; J = 1 .. 3: j + 1 == J, the pipelined loop (its own kernel; four
// vectors would spill).  Held to 64 registers so that all 4 CTAs per SM
// stay resident.
template <int J>
__global__ void __launch_bounds__(RED_THREADS, 4)
k_update(const double *__restrict__ V, long long nv2, int j, double *__restrict__ w,
         SolveState *S, double *partials, int pass, int final_pass) {
    pdl_wait();
    pdl_trigger();
    if (S->done) return;   // set by an earlier kernel: a plain load
    __shared__ double sh_h[MAXM + 1];
    __shared__ double sh_w[RED_THREADS], sh_o[1];
    const int jp1 = j + 1;
    const double *hsrc = pass == 0 ? S->h : S->h2;
    for (int k = threadIdx.x; k < jp1; k += blockDim.x) sh_h[k] = hsrc[k];
    __syncthreads();
    double2 *w2 = reinterpret_cast<double2 *>(w);
    const double2 *V2 = reinterpret_cast<const double2 *>(V);
    double nrm[1] = {0.0};
    const long long st = (long long)gridDim.x * blockDim.x;
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if constexpr (J > 0) {
        update_pipelined<J>(V2, nv2, w2, sh_h, nrm[0]);
        e = nv2;   // every element done
    }
    for (; e + st < nv2; e += 2 * st) {  // two grid strides per iteration
        double2 ta = w2[e], tb = w2[e + st];
        for (int k = 0; k < jp1; k++) {
            const double2 va = V2[(size_t)k * nv2 + e], vb = V2[(size_t)k * nv2 + e + st];
            ta.x -= sh_h[k] * va.x;
            ta.y -= sh_h[k] * va.y;
            tb.x -= sh_h[k] * vb.x;
            tb.y -= sh_h[k] * vb.y;
        }
        w2[e] = ta;
        w2[e + st] = tb;
        nrm[0] = fma(ta.y, ta.y, fma(ta.x, ta.x, nrm[0]));
        nrm[0] = fma(tb.y, tb.y, fma(tb.x, tb.x, nrm[0]));
    }
    if (e < nv2) {
        double2 t = w2[e];
        for (int k = 0; k < jp1; k++) {
            const double2 v = V2[(size_t)k * nv2 + e];
            t.x -= sh_h[k] * v.x;
            t.y -= sh_h[k] * v.y;
        }
        w2[e] = t;
        nrm[0] = fma(t.y, t.y, fma(t.x, t.x, nrm[0]));
    }
    if (!final_pass) return;
    block_sum<1>(nrm, sh_w, sh_o, 1);
    if (threadIdx.x == 0) partials[(size_t)blockIdx.x * (MAXM + 2) + MAXM + 1] = sh_o[0];
    if (!last_cta(S)) return;
    reduce_partials<1>(partials, MAXM + 2, MAXM + 1, 1, sh_w, sh_o);
    if (threadIdx.x != 0) return;
    givens_column(S, j, pass == 1, sqrt(sh_o[0]));
}

// k_update for step j (the pipelined kernels for one to three basis vectors)
template <int J>
static void launch_update_j(int nred, cudaStream_t st, const double *V, long long nv2, int j,
                            double *w, SolveState *S, double *partials, int pass, int fin) {
    launch_pdl(k_update<J>, nred, RED_THREADS, 0, st, V, nv2, j, w, S, partials, pass, fin);
}
static void launch_update(int nred, cudaStream_t st, const double *V, long long nv2, int j,
                          double *w, SolveState *S, double *partials, int pass, int fin) {
    switch (j + 1) {
    case 1: launch_update_j<1>(nred, st, V, nv2, j, w, S, partials, pass, fin); break;
    case 2: launch_update_j<2>(nred, st, V, nv2, j, w, S, partials, pass, fin); break;
    case 3: launch_update_j<3>(nred, st, V, nv2, j, w, S, partials, pass, fin); break;
    default: launch_update_j<0>(nred, st, V, nv2, j, w, S, partials, pass, fin); break;
    }
}

// y = R^{-1} g (every CTA, redundantly, in shared memory), then x += Z y
__global__ void __launch_bounds__(RED_THREADS)
k_xupdate(const double *__restrict__ Z, long long nv2, double *__restrict__ x, SolveState *S) {
    pdl_wait();
    pdl_trigger();
    __shared__ double y[MAXM];
    __shared__ double sR[MAXM * MAXM / 2 + MAXM], sg[MAXM], sinv[MAXM];   // R's upper triangle, g
    const int kd = S->kdim;
    if (kd == 0) return;
    // R and g into shared memory by the whole CTA (one round of loads), the
    // reciprocals of R's diagonal by kd threads at once, then the back
    // substitution by one thread from there: its chain of dependent FP64
    // operations waits on no global load and on no division (an FP64 division
    // is a chain of dependent FP64 operations of 64 cycles each on this GPU)
    for (int t = threadIdx.x; t < kd * kd; t += blockDim.x) {
        const int i = t / kd, k = t % kd;
        if (k >= i) sR[i * kd - i * (i - 1) / 2 + (k - i)] = S->H[i * MAXM + k];
    }
    for (int t = threadIdx.x; t < kd; t += blockDim.x) {
        sg[t] = S->g[t];
        sinv[t] = 1.0 / S->H[t * MAXM + t];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = kd - 1; i >= 0; i--) {
            const double *Ri = sR + i * kd - i * (i - 1) / 2 - i;   // Ri[k] = R[i][k], k >= i
            double s = sg[i];
            for (int k = i + 1; k < kd; k++) s -= Ri[k] * y[k];
            y[i] = s * sinv[i];
        }
    }
    __syncthreads();
    const double2 *Z2 = reinterpret_cast<const double2 *>(Z);
    double2 *x2 = reinterpret_cast<double2 *>(x);
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nv2;
         e += (long long)gridDim.x * blockDim.x) {
        double2 t = x2[e];
        for (int k = 0; k < kd; k++) {
            const double2 z = Z2[(size_t)k * nv2 + e];
            t.x += y[k] * z.x;
            t.y += y[k] * z.y;
        }
        x2[e] = t;
    }
}

// the singular-block and timed-out-wait counters of one factors handle into
// the host-mapped status (first: assign, else add), so the host reads them
// with the status after its final stream synchronisation
__global__ void k_counters(const unsigned long long *ctr, HostStatus *hs, int first) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    volatile HostStatus *vh = hs;
    vh->nsing = (first ? 0ull : vh->nsing) + ctr[0];
    vh->ntimeout = (first ? 0ull : vh->ntimeout) + ctr[4];
    __threadfence_system();
}

__global__ void k_solve_init(SolveState *S, HostStatus *hs, double rtol, int max_iters, int m) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    S->rtol = rtol;
    S->max_iters = max_iters;
    S->m = m;
    S->hs = hs;
}

}  // namespace abilu

using namespace abilu;

extern "C" void fgmres_default_opts(fgmres_opts *o) {
    if (!o) return;
    o->restart = 30;
    o->max_iters = 2500;
    o->rtol = 1e-6;
    o->build_sweeps = 1;
    o->apply_sweeps_lower = 3;
    o->apply_sweeps_upper = 3;
    o->mode = ABILU_ASYNC;
    o->build = 1;
    o->init = ABILU_INIT_FROM_A;
    o->reorth = 0;
    o->zero_guess = 0;
    o->spin_limit = 0;
}

namespace abilu {
static HostStatus read_status(const HostStatus *p) {
    const volatile HostStatus *v = p;
    HostStatus h;
    h.done = v->done; h.iters = v->iters; h.converged = v->converged; h.kdim = v->kdim;
    h.restarts = v->restarts; h.breakdown = v->breakdown;
    h.est = v->est; h.beta = v->beta; h.bnorm = v->bnorm;
    h.nsing = v->nsing; h.ntimeout = v->ntimeout;
    return h;
}
size_t solve_state_bytes() { return sizeof(SolveState); }
size_t host_status_bytes() { return sizeof(HostStatus); }
int max_restart() { return MAXM; }
}  // namespace abilu

namespace abilu {

// block ILU(0) preconditioner of fgmres_solve
struct IluPc {
    abilu_factors f;
    int nl, nu;
    abilu_mode mode;
    bool y_ready;   // the FGMRES kernels that write v32 also prepare y[0] and the tickets
};
static abilu_status ilu_pc(void *ctx, const double *v, const float *v32, double *z,
                           cudaStream_t st, Skip skip) {
    const IluPc *c = static_cast<const IluPc *>(ctx);
    if (c->y_ready) return apply_dispatch_ready(c->f, v, v32, z, c->nl, c->nu, c->mode, st, skip);
    return apply_dispatch(c->f, v, v32, z, c->nl, c->nu, c->mode, st, skip);
}

// FGMRES(m) on pattern P with the preconditioner `pc`; the Krylov basis, the
// device solve state and the reductions' partials live in `ws` (a factors
// handle of P).  Singular-block and timeout counters are collected from the
// handles `cnt[0..ncnt)`.
abilu_status fgmres_run(const PatternView &P, const double *A, abilu_factors ws, const Precond &pc,
                        const double *b, double *x, const fgmres_opts *opts, fgmres_result *res,
                        cudaStream_t st, abilu_factors const *cnt, int ncnt) {
    const int m = opts->restart;
    abilu_status s = ensure_krylov(ws, m);
    if (s != ABILU_OK) return s;
    const long long nv = (long long)P.n * BS, nv2 = nv / 2;
    double *V = ws->krylov;
    double *Z = V + (size_t)(m + 1) * nv;
    double *w = Z + (size_t)m * nv;
    SolveState *SS = reinterpret_cast<SolveState *>(ws->scal);
    HostStatus *hs = reinterpret_cast<HostStatus *>(ws->host_status);
    const int nred = red_ctas();
    const int nres = nred / 4 * 3;   // k_residual: 3 CTAs per SM
    const Skip skip{&SS->done, nullptr, nullptr};
    float *v32 = pc.v32;
    const int form = gs_form_for(opts->reorth, opts->rtol);

    ABILU_CUDA(cudaMemsetAsync(SS, 0, sizeof(SolveState), st));
    k_solve_init<<<counted(1), 1, 0, st>>>(SS, hs, opts->rtol, opts->max_iters, m);
    if (opts->zero_guess) ABILU_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * nv, st));
    if (opts->zero_guess)
        launch_pdl(k_residual<true>, nres, RED_THREADS, 0, st, P, A, b, x, V, SS, ws->partials, 1);
    else
        launch_pdl(k_residual<false>, nres, RED_THREADS, 0, st, P, A, b, x, V, SS, ws->partials, 1);
    // v_0 = r / beta; with x = 0, r = b is read from b itself
    launch_pdl(k_scale, nred, RED_THREADS, 0, st, opts->zero_guess ? b : V, V, v32, nv2, SS,
               pc.y0, pc.tickets);
    ABILU_LAUNCH_CHECK("fgmres init");
    // the look-ahead events live in the workspace handle (made on first use)
    for (int k = 0; k < 2; k++)
        if (!ws->ev[k]) ABILU_CUDA(cudaEventCreateWithFlags(reinterpret_cast<cudaEvent_t *>(&ws->ev[k]),
                                                            cudaEventDisableTiming));
    cudaEvent_t ev[2] = {static_cast<cudaEvent_t>(ws->ev[0]), static_cast<cudaEvent_t>(ws->ev[1])};
    // No wait for the initial residual: the first cycle is enqueued at once,
    // and its kernels return at once if the initial guess already converged
    // (the device flag is set).  The host reads the status one step behind.
    HostStatus h = {};
    abilu_status ret = ABILU_OK;
    for (bool first = true; first || (!h.converged && h.iters < opts->max_iters); first = false) {
        int j = 0;
        double e_prev = -1.0;   // the estimate after step j-2, as the host last read it
        for (; j < m; j++) {
            s = pc.fn(pc.ctx, V + (size_t)j * nv, v32, Z + (size_t)j * nv, st, skip);
            if (s != ABILU_OK) { ret = s; break; }
            // w = A z_j with the first pass's dots (and, in the single-reduction
            // form, ||w||^2, h_{j+1,j} and the Givens update) in one kernel
            if (form == GS_SINGLE)
                launch_spmv_dots_n<true>(nres, st, P, A, Z + (size_t)j * nv, w, V, nv, j + 1, SS,
                                         ws->partials);
            else
                launch_spmv_dots_n<false>(nres, st, P, A, Z + (size_t)j * nv, w, V, nv, j + 1, SS,
                                          ws->partials);
            if (form == GS_SINGLE) {            // one pass, one reduction (see k_spmv_dots)
                launch_update_scale(nred, st, V, nv2, j, w, V + (size_t)(j + 1) * nv, v32, SS,
                                    pc.y0, pc.tickets);
            } else if (form == GS_CLASSICAL) {  // one pass, the norm of the updated w
                launch_update(nred, st, V, nv2, j, w, SS, ws->partials, 0, 1);
                launch_pdl(k_scale, nred, RED_THREADS, 0, st, w, V + (size_t)(j + 1) * nv, v32, nv2, SS,
                           pc.y0, pc.tickets);
            } else {               // CGS2: two passes, the norm of the updated w
                launch_update(nred, st, V, nv2, j, w, SS, ws->partials, 0, 0);
                launch_dots(nred, st, V, nv2, j + 1, w, SS, ws->partials, 1);
                launch_update(nred, st, V, nv2, j, w, SS, ws->partials, 1, 1);
                launch_pdl(k_scale, nred, RED_THREADS, 0, st, w, V + (size_t)(j + 1) * nv, v32, nv2, SS,
                           pc.y0, pc.tickets);
            }
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) { ret = cuda_fail(e, "fgmres step"); break; }
            e = cudaEventRecord(ev[j & 1], st);
            if (e != cudaSuccess) { ret = cuda_fail(e, "fgmres event record"); break; }
            if (j >= 1) {  // look at step j-1 while step j runs
                // an asynchronous error shows here: stop enqueuing (the mapped
                // status would be stale)
                e = cudaEventSynchronize(ev[(j - 1) & 1]);
                if (e != cudaSuccess) { ret = cuda_fail(e, "fgmres step wait"); break; }
                const volatile HostStatus *vh = reinterpret_cast<volatile HostStatus *>(hs);
                if (vh->done) { j++; break; }
                // when the estimates after steps j-2 and j-1, extrapolated
                // geometrically, put step j at the tolerance, wait for step j
                // before enqueuing step j+1: a step past the end of the cycle
                // would be launched only to return at once
                const double e1 = vh->est;
                if (e_prev > 0.0 && e1 < e_prev && e1 * (e1 / e_prev) <= opts->rtol) {
                    e = cudaEventSynchronize(ev[j & 1]);
                    if (e != cudaSuccess) { ret = cuda_fail(e, "fgmres step wait"); break; }
                    if (vh->done) { j++; break; }
                }
                e_prev = e1;
            }
        }
        if (ret != ABILU_OK) break;
        launch_pdl(k_xupdate, nred, RED_THREADS, 0, st, Z, nv2, x, SS);
        launch_pdl(k_residual<false>, nres, RED_THREADS, 0, st, P, A, b, x, V, SS, ws->partials, 0);
        launch_pdl(k_scale, nred, RED_THREADS, 0, st, V, V, v32, nv2, SS, pc.y0, pc.tickets);
        // the handles' counters into the status with every cycle's result, so
        // the synchronisation that ends the last cycle also ends the solve
        for (int k = 0; k < ncnt; k++)
            k_counters<<<counted(1), 32, 0, st>>>(cnt[k]->ctr, hs, k == 0);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) { ret = cuda_fail(e, "fgmres restart"); break; }
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { ret = cuda_fail(e, "fgmres sync"); break; }
        h = read_status(hs);
    }
    const bool zero_b = ret == ABILU_OK && h.bnorm == 0.0;
    if (zero_b)  // b = 0: the solution is x = 0
        ABILU_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * nv, st));
    if (ret != ABILU_OK || zero_b) {   // a cycle that did not finish, or the memset
        for (int k = 0; k < ncnt; k++)
            k_counters<<<counted(1), 32, 0, st>>>(cnt[k]->ctr, hs, k == 0);
        cudaStreamSynchronize(st);
        h = read_status(hs);
    }
    res->iters = h.iters;
    res->restarts = h.restarts;
    res->rel_resid_est = h.est;
    res->rel_resid_true = h.bnorm > 0.0 ? h.beta / h.bnorm : 0.0;
    const unsigned long long ns = h.nsing, nto = h.ntimeout;
    if (nto)   // reset the timed-out-wait words (never expected)
        for (int k = 0; k < ncnt; k++) cudaMemset(cnt[k]->ctr + 4, 0, sizeof(unsigned long long));
    res->singular_blocks = (int64_t)ns;
    if (nto && ret == ABILU_OK)  // a staged sweep's bounded wait ran out: results invalid
        ret = fail(ABILU_ETIMEOUT, "fgmres_solve: %llu pipeline waits timed out", nto);
    if (ret == ABILU_OK) {
        if (!h.converged) ret = fail(ABILU_ENOCONV, "fgmres_solve: %d iterations, relative residual %.3e > rtol %.3e", h.iters, res->rel_resid_true, opts->rtol);
        else if (ns > 0) ret = fail(ABILU_WARN_SINGULAR, "fgmres_solve: %llu singular diagonal blocks replaced", ns);
    }
    res->status = ret;
    return ret;
}

// options shared by every FGMRES entry point
abilu_status fgmres_check_opts(const fgmres_opts *opts, const char *who) {
    if (opts->restart < 1 || opts->restart > MAXM)
        return fail(ABILU_EINVAL, "%s: restart must be in 1..%d", who, MAXM);
    if (opts->max_iters < 0 || !(opts->rtol >= 0.0))
        return fail(ABILU_EINVAL, "%s: bad options", who);
    if (opts->spin_limit < 0) return fail(ABILU_EINVAL, "%s: spin_limit must be >= 0", who);
    return ABILU_OK;
}

}  // namespace abilu

extern "C" abilu_status fgmres_solve(abilu_pattern p, const double *A, abilu_factors f,
                                     const double *b, double *x, const fgmres_opts *opts,
                                     fgmres_result *res, abilu_stream stream) {
    if (!p || !A || !f || !b || !x || !opts || !res)
        return fail(ABILU_EINVAL, "fgmres_solve: NULL argument");
    memset(res, 0, sizeof *res);
    if (f->p != p && (f->p->v.n != p->v.n || opts->build))
        return fail(ABILU_EINVAL, "fgmres_solve: factors of another pattern need the same n and opts->build = 0");
    abilu_status s = fgmres_check_opts(opts, "fgmres_solve");
    if (s != ABILU_OK) return s;
    if (opts->apply_sweeps_lower < 0 || opts->apply_sweeps_upper < 0 || opts->build_sweeps < 0 ||
        (opts->mode != ABILU_SYNC && opts->mode != ABILU_ASYNC))
        return fail(ABILU_EINVAL, "fgmres_solve: bad options");
    cudaStream_t st = S(stream);
    const abilu_mode mode = (abilu_mode)opts->mode;
    // the solve's spin limit on the handle for the solve's build and
    // applications, the handle's own afterwards
    const unsigned long long keep_limit = f->spin_limit;
    f->spin_limit = (unsigned long long)opts->spin_limit;
    if (opts->build) {
        s = build_dispatch(f, A, opts->build_sweeps, mode, (abilu_init)opts->init, st);
        if (s != ABILU_OK) { f->spin_limit = keep_limit; return s; }
    }
    const bool ready = apply_y_ready(f, opts->apply_sweeps_lower, opts->apply_sweeps_upper, mode);
    IluPc ctx{f, opts->apply_sweeps_lower, opts->apply_sweeps_upper, mode, ready};
    // v32: NULL for FP64 factors; y0 and the tickets: the asynchronous
    // application's in-place lower iterate and its ticket counters
    const Precond pc{ilu_pc, &ctx, reinterpret_cast<float *>(f->r32),
                     ready ? reinterpret_cast<float *>(f->y[0]) : nullptr, ready ? f->ctr + 2 : nullptr};
    s = fgmres_run(p->v, A, f, pc, b, x, opts, res, st, &f, 1);
    f->spin_limit = keep_limit;
    return s;
}
