// Batched solve of many independent systems of uneven size in the same
// launches.
//
// The systems are concatenated into one block-diagonal pattern (no block
// couples two systems), each system's rows padded to a multiple of 64 with
// identity rows.  Because the fixed-point map of Eq. (bilu), the triangular
// sweeps and the SpMV never read across a block row's pattern, one build
// sweep, one triangular sweep or one SpMV over the concatenation is exactly
// that step for every system at once: the single-system kernels run
// unchanged, one launch for the whole batch (the large systems load-balance
// the small ones across the GPU).  The padding makes every 64-row chunk belong
// to one system, so the Krylov kernels below keep a separate FGMRES state per
// system: per-system dot products and norms (each CTA of a reducing kernel
// sums a run of up to 16 of one system's chunks, and the partials of a
// system's runs are summed in order by the last of them to finish),
// per-system Hessenberg, Givens rotations and convergence.  The systems iterate
// in lockstep; a system that has converged (or left its cycle) skips its
// chunks in the Krylov kernels.  Padding rows have b = 0 and stay x = 0, so they
// change no norm.
#include <stdlib.h>
#include <string.h>

#include <vector>

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
void apply_warm(abilu_dtype dt);
size_t solve_state_bytes();
int red_ctas();

constexpr int BMAXM = 64;
constexpr int CHUNK_ROWS = 64;           // rows per CTA = padding unit
constexpr int CHUNK_VALS = CHUNK_ROWS * BS;
constexpr int BTILE = 8;
constexpr int PSTRIDE = BMAXM + 2;       // partials per chunk

struct BState {
    double H[BMAXM * BMAXM];   // R after rotations, H[i*BMAXM + j]
    double cs[BMAXM], sn[BMAXM], g[BMAXM + 1], h[BMAXM + 1], h2[BMAXM + 1], y[BMAXM];
    double bnorm, beta, hn_inv, est;
    int done;        // out of the current cycle (converged estimate, breakdown, cycle end, max)
    int finished;    // converged (true residual) or max_iters reached
    int converged, iters, kdim, restarts, breakdown;
    unsigned counter;
};

struct BConf {
    double rtol;
    int max_iters, m;
};

// The reducing kernels (residual, Gram-Schmidt dots, norms) give each CTA a
// super-chunk: up to SUPER_CHUNKS consecutive 64-row chunks of one system, so
// one block reduction covers up to 4,096 values (one per 256 values made the
// reductions' latency, not memory, bound those kernels).  A system's
// super-chunks split its chunks from its first one, whatever its place in
// the batch, so its reductions are the same alone and in any batch.
constexpr int SUPER_CHUNKS = 16;
struct BTab {
    const int *sc_first;   // [nsc + 1] first chunk of each super-chunk
    const int *sc_sys;     // [nsc] its system
    const int *sys_sc0;    // [nsys + 1] first super-chunk of each system
};

__device__ __forceinline__ bool last_cta_of(BState *St, int nck) {
    __shared__ bool am_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) am_last = atomicAdd(&St->counter, 1u) == (unsigned)(nck - 1);
    __syncthreads();
    if (am_last) __threadfence();
    return am_last;
}

// sum over the system's chunks c0..c1-1 (in this order per thread, then a
// fixed-order block reduction) of partials[c*PS + k0 + k], k < kn <= K
template <int K, int PS>
__device__ __forceinline__ void reduce_sys(const double *partials, int c0, int c1, int k0, int kn,
                                           double *sh_w, double *out) {
    double v[K];
#pragma unroll
    for (int k = 0; k < K; k++) v[k] = 0.0;
    for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
        const double *p = partials + (size_t)c * PS + k0;
#pragma unroll
        for (int k = 0; k < K; k++)
            if (k < kn) v[k] += __ldcg(p + k);
    }
    block_sum<K>(v, sh_w, out, kn);
}

// r = b - A x for the chunk's rows (into r_out), ||r||^2 and ||b||^2 per system;
// the system's last chunk sets beta, the convergence state and a new cycle
__global__ void __launch_bounds__(RED_THREADS)
k_b_residual(PatternView P, const double *__restrict__ A, const double *__restrict__ b,
             const double *__restrict__ x, double *__restrict__ r_out, BState *S, BTab T,
             double *partials, BConf cf, int init, int *hs_done, int *hs_fin, int *sys_done,
             int *bflag) {
    pdl_wait();
    pdl_trigger();
    __shared__ double sh_w[RED_THREADS * 2], sh_o[2];
    const int sc = blockIdx.x, s = T.sc_sys[sc];
    BState *St = S + s;
    if (!init && St->finished) return;  // whole system skips
    const int q = threadIdx.x & 3;
    double v[2] = {0.0, 0.0};
    for (int chunk = T.sc_first[sc]; chunk < T.sc_first[sc + 1]; chunk++) {
        const int i = chunk * CHUNK_ROWS + (threadIdx.x >> 2);
        // a solve starts from x = 0, where r = b needs no product
        const double acc = init ? 0.0 : row_dot_blocks(P, A, x, i, q);
        const size_t o = (size_t)i * BS + q;
        const double bi = b[o], ri = bi - acc;
        r_out[o] = ri;
        v[0] = fma(ri, ri, v[0]);
        v[1] = fma(bi, bi, v[1]);
    }
    block_sum<2>(v, sh_w, sh_o, 2);
    if (threadIdx.x == 0) {
        partials[(size_t)sc * 2 + 0] = sh_o[0];
        partials[(size_t)sc * 2 + 1] = sh_o[1];
    }
    const int c0 = T.sys_sc0[s], c1 = T.sys_sc0[s + 1];
    if (!last_cta_of(St, c1 - c0)) return;
    reduce_sys<2, 2>(partials, c0, c1, 0, 2, sh_w, sh_o);
    if (threadIdx.x == 0) {
        if (init) St->bnorm = sqrt(sh_o[1]);
        else St->restarts += 1;
        St->beta = sqrt(sh_o[0]);
        St->converged = (St->beta <= cf.rtol * St->bnorm || St->bnorm == 0.0) ? 1 : 0;
        St->finished = (St->converged || St->iters >= cf.max_iters) ? 1 : 0;
        St->done = St->finished;
        St->hn_inv = St->beta > 0.0 ? 1.0 / St->beta : 0.0;
        St->kdim = 0;
        St->breakdown = 0;
        St->g[0] = St->beta;
        for (int k = 1; k <= BMAXM; k++) St->g[k] = 0.0;
        if (init) St->est = St->bnorm > 0.0 ? St->beta / St->bnorm : 0.0;
        St->counter = 0;
        sys_done[s] = St->done;
        if (!St->done) {  // active in the coming cycle (bflag was reset to {1, 0})
            bflag[0] = 0;
            atomicAdd(bflag + 1, 1);
        }
        reinterpret_cast<volatile int *>(hs_done)[s] = St->done;
        reinterpret_cast<volatile int *>(hs_fin)[s] = St->finished;
        __threadfence_system();
    }
}

// bflag = {all systems done with the cycle, systems still active}; reset
// before the residual kernel that starts a cycle
__global__ void k_b_flags_reset(int *bflag) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        bflag[0] = 1;
        bflag[1] = 0;
    }
}

// The apply's two ticket counters zeroed for its next application (first
// CTA, whatever its system's state), when the kernels that write its FP32
// right-hand side also prepare its start (see apply_dispatch_ready)
__device__ __forceinline__ void b_zero_tickets(unsigned long long *tk) {
    if (tk && blockIdx.x == 0 && threadIdx.x < 2) tk[threadIdx.x] = 0ull;
}

// v_out = v_in * hn_inv of the chunk's system (and the FP32 copy for the
// apply, also into y0, the asynchronous apply's in-place iterate, when given)
__global__ void __launch_bounds__(RED_THREADS)
k_b_scale(const double *vin, double *vout, float *v32, const BState *S,
          const int *__restrict__ chunk_sys, float *y0, unsigned long long *tk) {
    pdl_wait();
    pdl_trigger();
    b_zero_tickets(tk);
    const int chunk = blockIdx.x;
    const BState *St = S + chunk_sys[chunk];
    if (St->done) return;
    const size_t e = (size_t)chunk * CHUNK_VALS + threadIdx.x;
    const double t = vin[e] * St->hn_inv;
    vout[e] = t;
    if (v32) {
        const float f = to_f32_int(t);
        v32[e] = f;
        if (y0) y0[e] = f;
    }
}

// partial dots <V_k0+k, w> over the super-chunk's chunks c0..c1-1 (one value
// per thread per chunk), one block reduction, partials of super-chunk sc.
// CG: w was written earlier in the same kernel (by this thread): read through
// L2, never the read-only path
template <int K, bool CG = false>
__device__ __forceinline__ void b_dots_tile(const double *__restrict__ V, size_t nv, int k0,
                                            const double *w, int c0, int c1,
                                            double *sh_w, double *sh_o, double *partials, int sc) {
    double acc[K];
#pragma unroll
    for (int k = 0; k < K; k++) acc[k] = 0.0;
    for (int c = c0; c < c1; c++) {
        const size_t e = (size_t)c * CHUNK_VALS + threadIdx.x;
        const double wv = CG ? __ldcg(w + e) : w[e];
#pragma unroll
        for (int k = 0; k < K; k++) acc[k] = fma(V[(size_t)(k0 + k) * nv + e], wv, acc[k]);
    }
    block_sum<K>(acc, sh_w, sh_o, K);
    if (threadIdx.x < K) partials[(size_t)sc * PSTRIDE + k0 + threadIdx.x] = sh_o[threadIdx.x];
}

// the dots tiles of basis vectors kbeg..jp1-1 over a super-chunk
template <bool CG = false>
__device__ __forceinline__ void b_dots_tiles(const double *__restrict__ V, size_t nv, int jp1,
                                             const double *w, int c0, int c1,
                                             double *sh_w, double *sh_o, double *partials, int sc,
                                             int kbeg = 0) {
    for (int k0 = kbeg; k0 < jp1; k0 += BTILE) {
        switch (jp1 - k0 < BTILE ? jp1 - k0 : BTILE) {
        case 1: b_dots_tile<1, CG>(V, nv, k0, w, c0, c1, sh_w, sh_o, partials, sc); break;
        case 2: b_dots_tile<2, CG>(V, nv, k0, w, c0, c1, sh_w, sh_o, partials, sc); break;
        case 3: b_dots_tile<3, CG>(V, nv, k0, w, c0, c1, sh_w, sh_o, partials, sc); break;
        case 4: b_dots_tile<4, CG>(V, nv, k0, w, c0, c1, sh_w, sh_o, partials, sc); break;
        case 5: b_dots_tile<5, CG>(V, nv, k0, w, c0, c1, sh_w, sh_o, partials, sc); break;
        case 6: b_dots_tile<6, CG>(V, nv, k0, w, c0, c1, sh_w, sh_o, partials, sc); break;
        case 7: b_dots_tile<7, CG>(V, nv, k0, w, c0, c1, sh_w, sh_o, partials, sc); break;
        default: b_dots_tile<8, CG>(V, nv, k0, w, c0, c1, sh_w, sh_o, partials, sc); break;
        }
    }
}

// The system's last CTA of a dots pass: h[k] (pass 0) or h2[k] (pass 1), k < jp1,
// from the partials of super-chunks c0..c1-1
__device__ __forceinline__ void b_dots_last(BState *St, int jp1, int pass, const double *partials,
                                            int c0, int c1, double *sh_w, double *sh_o) {
    double *h = pass == 0 ? St->h : St->h2;
    for (int k0 = 0; k0 < jp1; k0 += BTILE) {
        const int kn = jp1 - k0 < BTILE ? jp1 - k0 : BTILE;
        reduce_sys<BTILE, PSTRIDE>(partials, c0, c1, k0, kn, sh_w, sh_o);
        if (threadIdx.x < kn) h[k0 + threadIdx.x] = sh_o[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0) St->counter = 0;
}

// h[k] = <V_k, w>_s for k <= j, per system (pass 0 -> h, 1 -> h2)
__global__ void __launch_bounds__(RED_THREADS)
k_b_dots(const double *__restrict__ V, size_t nv, int j, const double *__restrict__ w, BState *S,
         BTab T, double *partials, int pass) {
    pdl_wait();
    pdl_trigger();
    __shared__ double sh_w[RED_THREADS * BTILE], sh_o[BTILE];
    const int sc = blockIdx.x, s = T.sc_sys[sc];
    BState *St = S + s;
    if (St->done) return;
    const int jp1 = j + 1;
    b_dots_tiles(V, nv, jp1, w, T.sc_first[sc], T.sc_first[sc + 1], sh_w, sh_o, partials, sc);
    const int c0 = T.sys_sc0[s], c1 = T.sys_sc0[s + 1];
    if (!last_cta_of(St, c1 - c0)) return;
    b_dots_last(St, jp1, pass, partials, c0, c1, sh_w, sh_o);
}

__device__ __forceinline__ void b_givens(BState *St, int s, int j, int two_pass, double hn,
                                         const BConf &cf, int *hs_done, int *sys_done,
                                         int *bflag);

// w -= sum_k h[k] V_k per system; on the final pass ||w||, and the system's last
// chunk applies the Givens update of column j and the convergence test
__global__ void __launch_bounds__(RED_THREADS)
k_b_update(const double *__restrict__ V, size_t nv, int j, double *__restrict__ w, BState *S,
           BTab T, double *partials, BConf cf, int pass, int final_pass, int *hs_done,
           int *sys_done, int *bflag) {
    pdl_wait();
    pdl_trigger();
    __shared__ double sh_h[BMAXM + 1];
    __shared__ double sh_w[RED_THREADS], sh_o[1];
    const int sc = blockIdx.x, s = T.sc_sys[sc];
    BState *St = S + s;
    if (St->done) return;
    const int jp1 = j + 1;
    const double *hsrc = pass == 0 ? St->h : St->h2;
    for (int k = threadIdx.x; k < jp1; k += blockDim.x) sh_h[k] = hsrc[k];
    __syncthreads();
    double nrm[1] = {0.0};
    for (int chunk = T.sc_first[sc]; chunk < T.sc_first[sc + 1]; chunk++) {
        const size_t e = (size_t)chunk * CHUNK_VALS + threadIdx.x;
        double t = w[e];
        for (int k = 0; k < jp1; k++) t = fma(-sh_h[k], V[(size_t)k * nv + e], t);
        w[e] = t;
        nrm[0] = fma(t, t, nrm[0]);
    }
    if (!final_pass) return;
    block_sum<1>(nrm, sh_w, sh_o, 1);
    if (threadIdx.x == 0) partials[(size_t)sc * PSTRIDE + BMAXM + 1] = sh_o[0];
    const int c0 = T.sys_sc0[s], c1 = T.sys_sc0[s + 1];
    if (!last_cta_of(St, c1 - c0)) return;
    reduce_sys<1, PSTRIDE>(partials, c0, c1, BMAXM + 1, 1, sh_w, sh_o);
    if (threadIdx.x != 0) return;
    b_givens(St, s, j, pass == 1, sqrt(sh_o[0]), cf, hs_done, sys_done, bflag);
}

// The Givens update of system s's column j with h_{j+1,j} = hn, its estimate
// and cycle-end test (one thread of the system's last CTA)
__device__ __forceinline__ void b_givens(BState *St, int s, int j, int two_pass, double hn,
                                         const BConf &cf, int *hs_done, int *sys_done,
                                         int *bflag) {
    // the previous rotations, i = 0 .. j-1, each mixing entries i and i+1 of
    // the new column: entry i+1 is still the Gram-Schmidt coefficient when
    // rotation i reaches it, so one carried value replaces a column array
    // (which lived in local memory)
    double a = St->h[0] + (two_pass ? St->h2[0] : 0.0);
    for (int i = 0; i < j; i++) {
        const double c = St->h[i + 1] + (two_pass ? St->h2[i + 1] : 0.0);
        St->H[i * BMAXM + j] = St->cs[i] * a + St->sn[i] * c;
        a = -St->sn[i] * a + St->cs[i] * c;
    }
    const double c = hn;
    const double d = sqrt(a * a + c * c);
    double cs = 1.0, sn = 0.0;
    if (d != 0.0) { cs = a / d; sn = c / d; }
    St->cs[j] = cs;
    St->sn[j] = sn;
    St->H[j * BMAXM + j] = cs * a + sn * c;
    const double gj = St->g[j];
    St->g[j + 1] = -sn * gj;
    St->g[j] = cs * gj;
    St->iters += 1;
    St->kdim = j + 1;
    St->est = St->bnorm > 0.0 ? fabs(St->g[j + 1]) / St->bnorm : 0.0;
    St->breakdown = hn == 0.0 ? 1 : 0;
    St->done = (fabs(St->g[j + 1]) <= cf.rtol * St->bnorm || hn == 0.0 ||
                St->iters >= cf.max_iters || j + 1 >= cf.m) ? 1 : 0;
    St->hn_inv = hn != 0.0 ? 1.0 / hn : 0.0;
    St->counter = 0;
    if (St->done) {
        sys_done[s] = 1;
        if (atomicSub(bflag + 1, 1) == 1) bflag[0] = 1;  // the last active system left
        reinterpret_cast<volatile int *>(hs_done)[s] = 1;
        __threadfence_system();
    }
}

// The system's last CTA of a single-reduction step: h[k], k <= j, and ||w||^2
// (slot BMAXM + 1) from the partials of super-chunks c0..c1-1, then
// h_{j+1,j} = sqrt(||w||^2 - sum h_k^2) (a difference below 1e-12 ||w||^2 is a
// breakdown) and the Givens update
__device__ __forceinline__ void b_dots_norm_last(BState *St, int s, int j, const double *partials,
                                                 int c0, int c1, double *sh_w, double *sh_o,
                                                 const BConf &cf, int *hs_done, int *sys_done,
                                                 int *bflag) {
    const int jp1 = j + 1;
    for (int k0 = 0; k0 < jp1; k0 += BTILE) {
        const int kn = jp1 - k0 < BTILE ? jp1 - k0 : BTILE;
        reduce_sys<BTILE, PSTRIDE>(partials, c0, c1, k0, kn, sh_w, sh_o);
        if (threadIdx.x < kn) St->h[k0 + threadIdx.x] = sh_o[threadIdx.x];
        __syncthreads();
    }
    reduce_sys<1, PSTRIDE>(partials, c0, c1, BMAXM + 1, 1, sh_w, sh_o);
    if (threadIdx.x != 0) return;
    const double ww = sh_o[0];
    double hh = 0.0;
    for (int k = 0; k < jp1; k++) hh = fma(St->h[k], St->h[k], hh);
    const double d = ww - hh;
    b_givens(St, s, j, 0, d > 1e-12 * ww ? sqrt(d) : 0.0, cf, hs_done, sys_done, bflag);
}

// w = A z for the super-chunk's rows (a quad of threads per block row, one
// 64-row chunk per pass, the SpMV kernel's FMA chain, spmv.cuh) and, from the
// same registers, the dots with V_0..V_{KF-1} and, with NORM, ||w||^2; w is
// stored once.  The same value-to-thread map as the dot tiles (value e =
// chunk * 256 + thread), so a later tile of the same kernel re-reads only
// this thread's own entries of w.
template <int KF, bool NORM>
__device__ __forceinline__ void b_spmv_tile(const PatternView &P, const double *__restrict__ A,
                                            const double *__restrict__ z, double *w,
                                            const double *__restrict__ V, size_t nv, int c0, int c1,
                                            double *sh_w, double *sh_o, double *partials, int sc) {
    constexpr int KA = KF + (NORM ? 1 : 0);
    double acc[KA];
#pragma unroll
    for (int k = 0; k < KA; k++) acc[k] = 0.0;
    const int q = threadIdx.x & 3;
    for (int c = c0; c < c1; c++) {
        const int i = c * CHUNK_ROWS + (threadIdx.x >> 2);
        const size_t e = (size_t)c * CHUNK_VALS + threadIdx.x;   // = i * BS + q
        double v[KF];   // issued with the row's matrix loads
#pragma unroll
        for (int k = 0; k < KF; k++) v[k] = __ldg(V + (size_t)k * nv + e);
        const double r = row_dot_blocks(P, A, z, i, q);
        w[e] = r;
#pragma unroll
        for (int k = 0; k < KF; k++) acc[k] = fma(v[k], r, acc[k]);
        if constexpr (NORM) acc[KF] = fma(r, r, acc[KF]);
    }
    block_sum<KA>(acc, sh_w, sh_o, KA);
    if (threadIdx.x < KF) partials[(size_t)sc * PSTRIDE + threadIdx.x] = sh_o[threadIdx.x];
    if (NORM && threadIdx.x == 0) partials[(size_t)sc * PSTRIDE + BMAXM + 1] = sh_o[KF];
}

// The Arnoldi product of the batch fused with the first Gram-Schmidt pass (the
// single-system solve's k_spmv_dots): w = A z_j per super-chunk with the dots
// of the first min(j + 1, B_FUSED) basis vectors (and ||w||^2 with NORM) in
// the same pass; the tiles past B_FUSED re-read the CTA's own entries of w
// through L2.  The system's last CTA then reduces the partials: with NORM,
// h and h_{j+1,j} = sqrt(||w||^2 - sum h_k^2) and the Givens update (the
// single-reduction step, b_dots_norm_last), else h of the first pass
// (b_dots_last).  One launch and one pass over w fewer per step than the
// product followed by the dots.  3 CTAs per SM: 80 registers hold a row's
// four blocks, its x gathers and the basis entries in flight.  B_FUSED = 3:
// with four in the product's pass the kernel spilled 100-156 bytes, and the
// 64-system batch took 7.59-7.62 against 7.57 ms per solve (asynchronous).
constexpr int B_FUSED = 3;
template <bool NORM>
__global__ void __launch_bounds__(RED_THREADS, 3)
k_b_spmv_dots(PatternView P, const double *__restrict__ A, const double *__restrict__ z,
              double *w, const double *__restrict__ V, size_t nv, int j, BState *S, BTab T,
              double *partials, BConf cf, int *hs_done, int *sys_done, int *bflag) {
    pdl_wait();
    pdl_trigger();
    __shared__ double sh_w[RED_THREADS * BTILE], sh_o[BTILE];
    const int sc = blockIdx.x, s = T.sc_sys[sc];
    BState *St = S + s;
    if (St->done) return;
    const int jp1 = j + 1;
    const int f0 = T.sc_first[sc], f1 = T.sc_first[sc + 1];
    switch (jp1 < B_FUSED ? jp1 : B_FUSED) {
    case 1: b_spmv_tile<1, NORM>(P, A, z, w, V, nv, f0, f1, sh_w, sh_o, partials, sc); break;
    case 2: b_spmv_tile<2, NORM>(P, A, z, w, V, nv, f0, f1, sh_w, sh_o, partials, sc); break;
    default: b_spmv_tile<3, NORM>(P, A, z, w, V, nv, f0, f1, sh_w, sh_o, partials, sc); break;
    }
    if (jp1 > B_FUSED) b_dots_tiles<true>(V, nv, jp1, w, f0, f1, sh_w, sh_o, partials, sc, B_FUSED);
    const int c0 = T.sys_sc0[s], c1 = T.sys_sc0[s + 1];
    if (!last_cta_of(St, c1 - c0)) return;
    if constexpr (NORM) b_dots_norm_last(St, s, j, partials, c0, c1, sh_w, sh_o, cf, hs_done, sys_done, bflag);
    else b_dots_last(St, jp1, 0, partials, c0, c1, sh_w, sh_o);
}

// v_{j+1} = (w - sum_k h[k] V_k) * hn_inv per system and its FP32 copy (w is
// not written back)
__global__ void __launch_bounds__(RED_THREADS)
k_b_update_scale(const double *__restrict__ V, size_t nv, int j, const double *__restrict__ w,
                 double *__restrict__ vnext, float *__restrict__ v32, const BState *S,
                 const int *__restrict__ chunk_sys, float *__restrict__ y0, unsigned long long *tk) {
    pdl_wait();
    pdl_trigger();
    b_zero_tickets(tk);
    __shared__ double sh_h[BMAXM + 1];
    const int chunk = blockIdx.x;
    const BState *St = S + chunk_sys[chunk];
    if (St->done) return;
    const int jp1 = j + 1;
    for (int k = threadIdx.x; k < jp1; k += blockDim.x) sh_h[k] = St->h[k];
    __syncthreads();
    const size_t e = (size_t)chunk * CHUNK_VALS + threadIdx.x;
    double t = w[e];
    for (int k = 0; k < jp1; k++) t = fma(-sh_h[k], V[(size_t)k * nv + e], t);
    const double r = t * St->hn_inv;
    vnext[e] = r;
    if (v32) {
        const float f = to_f32_int(r);
        v32[e] = f;
        if (y0) y0[e] = f;
    }
}

// y = R^{-1} g per system (one thread per system)
__global__ void k_b_ysolve(BState *S, int nsys) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys) return;
    BState *St = S + s;
    const int kd = St->kdim;
    for (int i = kd - 1; i >= 0; i--) {
        double v = St->g[i];
        for (int k = i + 1; k < kd; k++) v -= St->H[i * BMAXM + k] * St->y[k];
        St->y[i] = v / St->H[i * BMAXM + i];
    }
}

// x += Z y for the chunk's system
__global__ void __launch_bounds__(RED_THREADS)
k_b_xupdate(const double *__restrict__ Z, size_t nv, double *__restrict__ x, const BState *S,
            const int *__restrict__ chunk_sys) {
    pdl_wait();
    pdl_trigger();
    const int chunk = blockIdx.x;
    const BState *St = S + chunk_sys[chunk];
    const int kd = St->kdim;
    if (kd == 0) return;
    const size_t e = (size_t)chunk * CHUNK_VALS + threadIdx.x;
    double t = x[e];
    for (int k = 0; k < kd; k++) t = fma(St->y[k], Z[(size_t)k * nv + e], t);
    x[e] = t;
}

__global__ void k_b_init(BState *S, int nsys) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys) return;
    S[s].iters = 0;
    S[s].restarts = 0;
    S[s].counter = 0;
    S[s].finished = 0;
    S[s].done = 0;
}

// ---- concatenation
// rows of system s (padded): rowptr of the concatenation; the padding rows'
// single (diagonal) block and their identity values
__global__ void k_cat_rows(int row_off, int nnz_off, int n, int nnzb, int nrows_padded,
                           const int32_t *__restrict__ rowptr, int32_t *__restrict__ rowptr_cat,
                           int32_t *__restrict__ colind_cat, double *__restrict__ A_cat) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows_padded) return;
    if (r < n) {
        rowptr_cat[row_off + r] = nnz_off + rowptr[r];
    } else {
        const int p = nnz_off + nnzb + (r - n);
        rowptr_cat[row_off + r] = p;
        colind_cat[p] = row_off + r;
        double *a = A_cat + (size_t)p * BB;
        for (int k = 0; k < BB; k++) a[k] = (k % 5 == 0) ? 1.0 : 0.0;
    }
}

__global__ void k_cat_cols(int row_off, int nnz_off, int nnzb, const int32_t *__restrict__ colind,
                           int32_t *__restrict__ colind_cat) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < nnzb) colind_cat[nnz_off + p] = row_off + colind[p];
}

__global__ void k_fill_int(int *a, int n, int v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

}  // namespace abilu

using namespace abilu;

struct abilu_batch_s {
    int nsys;
    std::vector<int> n, nnzb, row_off, nnz_off, chunk0;
    int rows, blocks, nchunks;
    int32_t *rowptr, *colind;   // concatenation (device)
    double *A, *b, *x;          // concatenation (device)
    int *chunk_sys, *sys_chunk0;
    int *sc_tab;                // super-chunks: sc_first [nsc + 1], sc_sys [nsc], sys_sc0 [nsys + 1]
    int nsc;
    BState *S;
    double *partials;
    double *krylov;
    int krylov_m;
    int *hs_done, *hs_fin;      // pinned, host-mapped
    int *sys_done, *bflag;      // device: per-system cycle exit; {all done, active count}
    cudaGraphExec_t graph;      // one restart cycle, captured on first use
    int gkey[12];
    long long g_fixed, g_step;  // kernels per replay outside the steps; per step run
    cudaStream_t cap_stream;    // capture happens here: the caller's stream may be the
                                // legacy default stream, which cannot be captured
    cudaStream_t body_stream;   // capture of the conditional step bodies
    int no_graph;               // 1: host-driven cycles (ABILU_NO_GRAPH set or capture failed)
    abilu_pattern pat;
    abilu_factors fac;
    std::vector<void *> allocs;
    int arena;                  // 1: a server's arena (capacity allocation, re-laid out)
};

// The super-chunk tables of the current systems (their chunk ranges in
// b->chunk0) into `h` (host, 2 * nchunks + nsys + 2 ints at least), then to
// the device on `st` (h must stay valid until the copy is done).
static abilu_status batch_super_chunks(abilu_batch b, int *h, cudaStream_t st) {
    const int nsys = b->nsys;
    std::vector<int> first, sys, s0(nsys + 1);
    for (int q = 0; q < nsys; q++) {
        s0[q] = (int)first.size();
        for (int c = b->chunk0[q]; c < b->chunk0[q + 1]; c += SUPER_CHUNKS) {
            first.push_back(c);
            sys.push_back(q);
        }
    }
    const int nsc = (int)first.size();
    s0[nsys] = nsc;
    first.push_back(b->chunk0[nsys]);
    memcpy(h, first.data(), sizeof(int) * (nsc + 1));
    memcpy(h + nsc + 1, sys.data(), sizeof(int) * nsc);
    memcpy(h + 2 * nsc + 1, s0.data(), sizeof(int) * (nsys + 1));
    ABILU_CUDA(cudaMemcpyAsync(b->sc_tab, h, sizeof(int) * (2 * nsc + nsys + 2),
                               cudaMemcpyHostToDevice, st));
    b->nsc = nsc;
    return ABILU_OK;
}

static BTab batch_tab(abilu_batch b) {
    return BTab{b->sc_tab, b->sc_tab + b->nsc + 1, b->sc_tab + 2 * b->nsc + 1};
}

static void batch_free(abilu_batch b) {
    if (!b) return;
    if (b->fac) abilu_factors_destroy(b->fac);
    if (b->pat) abilu_pattern_destroy(b->pat);
    for (void *p : b->allocs) cudaFree(p);
    if (b->krylov) cudaFree(b->krylov);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->body_stream) cudaStreamDestroy(b->body_stream);
    if (b->hs_done) cudaFreeHost(b->hs_done);
    if (b->hs_fin) cudaFreeHost(b->hs_fin);
    delete b;
}

extern "C" void abilu_batch_destroy(abilu_batch b) { batch_free(b); }

extern "C" abilu_status abilu_batch_create(int32_t nsys, const int32_t *n, const int32_t *nnzb,
                                           const int32_t *const *rowptr,
                                           const int32_t *const *colind, abilu_dtype dtype,
                                           abilu_stream stream, abilu_batch *out) {
    if (!out) return fail(ABILU_EINVAL, "batch_create: out is NULL");
    *out = nullptr;
    if (nsys < 1 || !n || !nnzb || !rowptr || !colind)
        return fail(ABILU_EINVAL, "batch_create: need nsys >= 1 and the host arrays");
    cudaStream_t st = S(stream);
    abilu_batch b = new abilu_batch_s();
    b->nsys = nsys;
    b->pat = nullptr;
    b->fac = nullptr;
    b->krylov = nullptr;
    b->krylov_m = 0;
    b->hs_done = b->hs_fin = nullptr;
    b->graph = nullptr;
    b->cap_stream = nullptr;
    b->body_stream = nullptr;
    b->no_graph = getenv("ABILU_NO_GRAPH") != nullptr;
    long long rows = 0, blocks = 0;
    for (int s = 0; s < nsys; s++) {
        if (n[s] < 1 || nnzb[s] < n[s] || !rowptr[s] || !colind[s]) {
            batch_free(b);
            return fail(ABILU_EINVAL, "batch_create: system %d has n=%d nnzb=%d or NULL arrays", s, n[s], nnzb[s]);
        }
        const int padded = (n[s] + CHUNK_ROWS - 1) / CHUNK_ROWS * CHUNK_ROWS;
        b->n.push_back(n[s]);
        b->nnzb.push_back(nnzb[s]);
        b->row_off.push_back((int)rows);
        b->nnz_off.push_back((int)blocks);
        b->chunk0.push_back((int)(rows / CHUNK_ROWS));
        rows += padded;
        blocks += (long long)nnzb[s] + (padded - n[s]);
    }
    if (rows > 0x7fffffffLL / BB || blocks > 0x7fffffffLL / BB) {
        batch_free(b);
        return fail(ABILU_EINVAL, "batch_create: batch too large for 32-bit block indices");
    }
    b->chunk0.push_back((int)(rows / CHUNK_ROWS));
    b->rows = (int)rows;
    b->blocks = (int)blocks;
    b->nchunks = (int)(rows / CHUNK_ROWS);
    auto alloc = [&](void **p, size_t bytes) -> abilu_status {
        cudaError_t e = cudaMalloc(p, bytes < 16 ? 16 : bytes);
        if (e != cudaSuccess) return cuda_fail(e, "batch_create: cudaMalloc");
        b->allocs.push_back(*p);
        return ABILU_OK;
    };
#define TRY(x)                                                  \
    do {                                                        \
        abilu_status s_ = (x);                                  \
        if (s_ != ABILU_OK) { batch_free(b); return s_; }       \
    } while (0)
    TRY(alloc((void **)&b->rowptr, sizeof(int32_t) * (rows + 1)));
    TRY(alloc((void **)&b->colind, sizeof(int32_t) * blocks));
    TRY(alloc((void **)&b->A, sizeof(double) * BB * blocks));
    TRY(alloc((void **)&b->b, sizeof(double) * BS * rows));
    TRY(alloc((void **)&b->x, sizeof(double) * BS * rows));
    TRY(alloc((void **)&b->chunk_sys, sizeof(int) * b->nchunks));
    TRY(alloc((void **)&b->sys_chunk0, sizeof(int) * (nsys + 1)));
    TRY(alloc((void **)&b->sc_tab, sizeof(int) * (2 * (size_t)b->nchunks + nsys + 2)));
    TRY(alloc((void **)&b->S, sizeof(BState) * nsys));
    TRY(alloc((void **)&b->partials, sizeof(double) * PSTRIDE * b->nchunks));
    TRY(alloc((void **)&b->sys_done, sizeof(int) * nsys));
    TRY(alloc((void **)&b->bflag, sizeof(int) * 4));
    auto cu = [&](cudaError_t e, const char *w) -> abilu_status {
        return e == cudaSuccess ? ABILU_OK : cuda_fail(e, w);
    };
    TRY(cu(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking), "stream"));
    TRY(cu(cudaStreamCreateWithFlags(&b->body_stream, cudaStreamNonBlocking), "stream"));
    TRY(cu(cudaHostAlloc((void **)&b->hs_done, sizeof(int) * nsys, cudaHostAllocMapped), "hostalloc"));
    TRY(cu(cudaHostAlloc((void **)&b->hs_fin, sizeof(int) * nsys, cudaHostAllocMapped), "hostalloc"));
    TRY(cu(cudaMemsetAsync(b->A, 0, sizeof(double) * BB * blocks, st), "memset A"));
    TRY(cu(cudaMemsetAsync(b->b, 0, sizeof(double) * BS * rows, st), "memset b"));
    TRY(cu(cudaMemsetAsync(b->x, 0, sizeof(double) * BS * rows, st), "memset x"));
    for (int s = 0; s < nsys; s++) {
        const int padded = b->chunk0[s + 1] * CHUNK_ROWS - b->row_off[s];
        k_cat_rows<<<counted((padded + 255) / 256), 256, 0, st>>>(
            b->row_off[s], b->nnz_off[s], b->n[s], b->nnzb[s], padded, rowptr[s], b->rowptr,
            b->colind, b->A);
        k_cat_cols<<<counted((b->nnzb[s] + 255) / 256), 256, 0, st>>>(b->row_off[s], b->nnz_off[s],
                                                                      b->nnzb[s], colind[s], b->colind);
        const int nck = b->chunk0[s + 1] - b->chunk0[s];
        k_fill_int<<<counted((nck + 255) / 256), 256, 0, st>>>(b->chunk_sys + b->chunk0[s], nck, s);
        TRY(cu(cudaGetLastError(), "batch concatenation"));
    }
    const int32_t last = (int32_t)blocks;
    TRY(cu(cudaMemcpyAsync(b->rowptr + rows, &last, sizeof last, cudaMemcpyHostToDevice, st), "rowptr end"));
    TRY(cu(cudaMemcpyAsync(b->sys_chunk0, b->chunk0.data(), sizeof(int) * (nsys + 1),
                           cudaMemcpyHostToDevice, st), "chunk table"));
    std::vector<int> h_sc(2 * (size_t)b->nchunks + nsys + 2);
    TRY(batch_super_chunks(b, h_sc.data(), st));
    TRY(cu(cudaStreamSynchronize(st), "sync"));
    TRY(abilu_pattern_create(b->rows, b->blocks, b->rowptr, b->colind, stream, &b->pat));
    TRY(abilu_factors_create(b->pat, dtype, &b->fac));
#undef TRY
    *out = b;
    return ABILU_OK;
}

extern "C" abilu_status abilu_batch_counts(abilu_batch b, int64_t *out) {
    if (!b || !out) return fail(ABILU_EINVAL, "batch_counts: NULL argument");
    out[0] = b->nsys;
    out[1] = b->rows;
    out[2] = b->blocks;
    out[3] = b->nchunks;
    return ABILU_OK;
}

extern "C" abilu_status abilu_batch_set_system(abilu_batch b, int32_t s, const double *A_vals,
                                               const double *rhs, abilu_stream stream) {
    if (!b || s < 0 || s >= b->nsys) return fail(ABILU_EINVAL, "batch_set_system: bad batch or index");
    cudaStream_t st = S(stream);
    if (A_vals)
        ABILU_CUDA(cudaMemcpyAsync(b->A + (size_t)b->nnz_off[s] * BB, A_vals,
                                   sizeof(double) * BB * b->nnzb[s], cudaMemcpyDeviceToDevice, st));
    if (rhs)
        ABILU_CUDA(cudaMemcpyAsync(b->b + (size_t)b->row_off[s] * BS, rhs,
                                   sizeof(double) * BS * b->n[s], cudaMemcpyDeviceToDevice, st));
    return ABILU_OK;
}

extern "C" abilu_status abilu_batch_set_build_chunk(abilu_batch b, int32_t blocks) {
    if (!b) return fail(ABILU_EINVAL, "batch_set_build_chunk: NULL batch");
    return abilu_factors_set_build_chunk(b->fac, blocks);
}

extern "C" abilu_status abilu_batch_get_solution(abilu_batch b, int32_t s, double *x,
                                                 abilu_stream stream) {
    if (!b || s < 0 || s >= b->nsys || !x) return fail(ABILU_EINVAL, "batch_get_solution: bad argument");
    ABILU_CUDA(cudaMemcpyAsync(x, b->x + (size_t)b->row_off[s] * BS, sizeof(double) * BS * b->n[s],
                               cudaMemcpyDeviceToDevice, S(stream)));
    return ABILU_OK;
}

static bool all_set(const int *flags, int n) {
    const volatile int *v = flags;
    for (int s = 0; s < n; s++)
        if (!v[s]) return false;
    return true;
}

// The asynchronous application's in-place iterate and ticket counters when
// the kernels that write its FP32 right-hand side also prepare its start
// (apply_dispatch_ready), else nulls (the application's own start kernel)
struct BStart {
    float *y0;
    unsigned long long *tk;
};
static BStart batch_start(abilu_batch b, const fgmres_opts *opts) {
    if (!apply_y_ready(b->fac, opts->apply_sweeps_lower, opts->apply_sweeps_upper,
                       (abilu_mode)opts->mode))
        return BStart{nullptr, nullptr};
    return BStart{reinterpret_cast<float *>(b->fac->y[0]), b->fac->ctr + 2};
}

// The Gram-Schmidt form of a solve's Arnoldi steps (see gs_form_for)
static int gs_form(const fgmres_opts *opts) { return gs_form_for(opts->reorth, opts->rtol); }

// One Arnoldi step j of every active system.  Every kernel skips the chunks of
// systems that have left the cycle (and returns at once when all have).
static abilu_status enqueue_step(abilu_batch b, const fgmres_opts *opts, const BConf &cf, int j,
                                 cudaStream_t st) {
    const PatternView &P = b->pat->v;
    const int m = cf.m, nck = b->nchunks;
    const size_t nv = (size_t)b->rows * BS;
    double *V = b->krylov, *Z = V + (size_t)(m + 1) * nv, *w = Z + (size_t)m * nv;
    float *v32 = reinterpret_cast<float *>(b->fac->r32);
    const Skip skip{b->bflag, b->chunk_sys, b->sys_done};
    const BStart y = batch_start(b, opts);
    abilu_status s = (y.y0 ? apply_dispatch_ready : apply_dispatch)(
        b->fac, V + (size_t)j * nv, v32, Z + (size_t)j * nv, opts->apply_sweeps_lower,
        opts->apply_sweeps_upper, (abilu_mode)opts->mode, st, skip);
    if (s != ABILU_OK) return s;
    const BTab T = batch_tab(b);
    const int nsc = b->nsc;
    const int form = gs_form(opts);
    // w = A z_j with the first Gram-Schmidt pass's dots (and ||w||^2 in the
    // single-reduction form) in one kernel
    const double *zj = Z + (size_t)j * nv;
    if (form == GS_SINGLE)
        launch_pdl(k_b_spmv_dots<true>, nsc, RED_THREADS, 0, st, P, b->A, zj, w, V, nv, j, b->S, T,
            b->partials, cf, b->hs_done, b->sys_done, b->bflag);
    else
        launch_pdl(k_b_spmv_dots<false>, nsc, RED_THREADS, 0, st, P, b->A, zj, w, V, nv, j, b->S, T,
            b->partials, cf, b->hs_done, b->sys_done, b->bflag);
    if (form == GS_SINGLE) {   // one pass, one reduction per system
        launch_pdl(k_b_update_scale, nck, RED_THREADS, 0, st, V, nv, j, w,
            V + (size_t)(j + 1) * nv, v32, b->S, b->chunk_sys, y.y0, y.tk);
    } else if (form == GS_CLASSICAL) {   // one pass, the norm of the updated w
        launch_pdl(k_b_update, nsc, RED_THREADS, 0, st, V, nv, j, w, b->S, T, b->partials, cf, 0, 1,
            b->hs_done, b->sys_done, b->bflag);
        launch_pdl(k_b_scale, nck, RED_THREADS, 0, st, w, V + (size_t)(j + 1) * nv, v32, b->S,
            b->chunk_sys, y.y0, y.tk);
    } else {               // CGS2: two passes, the norm of the updated w
        launch_pdl(k_b_update, nsc, RED_THREADS, 0, st, V, nv, j, w, b->S, T, b->partials, cf, 0, 0,
            b->hs_done, b->sys_done, b->bflag);
        launch_pdl(k_b_dots, nsc, RED_THREADS, 0, st, V, nv, j, w, b->S, T, b->partials, 1);
        launch_pdl(k_b_update, nsc, RED_THREADS, 0, st, V, nv, j, w, b->S, T, b->partials, cf, 1, 1,
            b->hs_done, b->sys_done, b->bflag);
        launch_pdl(k_b_scale, nck, RED_THREADS, 0, st, w, V + (size_t)(j + 1) * nv, v32, b->S,
            b->chunk_sys, y.y0, y.tk);
    }
    ABILU_LAUNCH_CHECK("batch step");
    return ABILU_OK;
}

// End of a cycle: x += Z y per system, true residual, new v_0, new cycle flags.
static abilu_status enqueue_restart(abilu_batch b, const fgmres_opts *opts, const BConf &cf,
                                    cudaStream_t st) {
    const BStart ys = batch_start(b, opts);
    const PatternView &P = b->pat->v;
    const int m = cf.m, nck = b->nchunks, nsys = b->nsys;
    const size_t nv = (size_t)b->rows * BS;
    double *V = b->krylov, *Z = V + (size_t)(m + 1) * nv;
    float *v32 = reinterpret_cast<float *>(b->fac->r32);
    k_b_ysolve<<<counted((nsys + 127) / 128), 128, 0, st>>>(b->S, nsys);
    launch_pdl(k_b_xupdate, nck, RED_THREADS, 0, st, Z, nv, b->x, b->S, b->chunk_sys);
    k_b_flags_reset<<<counted(1), 32, 0, st>>>(b->bflag);
    launch_pdl(k_b_residual, b->nsc, RED_THREADS, 0, st, P, b->A, b->b, b->x, V, b->S, batch_tab(b),
        b->partials, cf, 0, b->hs_done, b->hs_fin, b->sys_done, b->bflag);
    launch_pdl(k_b_scale, nck, RED_THREADS, 0, st, V, V, v32, b->S, b->chunk_sys, ys.y0, ys.tk);
    ABILU_LAUNCH_CHECK("batch restart");
    return ABILU_OK;
}

// condition of the IF node around an Arnoldi step: run it unless every system
// has left the cycle; bflag[2] counts the steps that ran
__global__ void k_b_set_cond(cudaGraphConditionalHandle h, int *bflag) {
    const int run = *reinterpret_cast<const volatile int *>(bflag) == 0;
    cudaGraphSetConditional(h, run ? 1u : 0u);
    if (run) bflag[2]++;
}

// Capture one restart cycle as a graph: each of the m steps is the body of an
// IF node whose condition a one-thread kernel sets from the device flag, so
// the steps after every system has converged cost a condition check, not a
// launch of their kernels; then the restart.
static abilu_status capture_cycle(abilu_batch b, const fgmres_opts *opts, const BConf &cf,
                                  cudaGraph_t *out) {
    cudaStream_t cs = b->cap_stream, bs = b->body_stream;
    *out = nullptr;
    const unsigned long long l0 = launches();
    unsigned long long in_steps = 0;
    ABILU_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    abilu_status st = ABILU_OK;
    cudaError_t e = cudaSuccess;
    for (int j = 0; j < cf.m && st == ABILU_OK && e == cudaSuccess; j++) {
        cudaStreamCaptureStatus cstat;
        cudaGraph_t g = nullptr;
        e = cudaStreamGetCaptureInfo(cs, &cstat, nullptr, &g, nullptr, nullptr, nullptr);
        if (e != cudaSuccess) break;
        cudaGraphConditionalHandle h;
        e = cudaGraphConditionalHandleCreate(&h, g, 0, 0);
        if (e != cudaSuccess) break;
        k_b_set_cond<<<counted(1), 1, 0, cs>>>(h, b->bflag);
        const cudaGraphNode_t *deps = nullptr;
        size_t ndeps = 0;
        e = cudaStreamGetCaptureInfo(cs, &cstat, nullptr, &g, &deps, nullptr, &ndeps);
        if (e != cudaSuccess) break;
        cudaGraphNodeParams prm = {};
        prm.type = cudaGraphNodeTypeConditional;
        prm.conditional.handle = h;
        prm.conditional.type = cudaGraphCondTypeIf;
        prm.conditional.size = 1;
        cudaGraphNode_t node;
        e = cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &prm);
        if (e != cudaSuccess) break;
        e = cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
        if (e != cudaSuccess) break;
        e = cudaStreamBeginCaptureToGraph(bs, prm.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) break;
        const unsigned long long s0 = launches();
        st = enqueue_step(b, opts, cf, j, bs);
        in_steps += launches() - s0;
        cudaGraph_t body;
        cudaError_t e2 = cudaStreamEndCapture(bs, &body);
        if (e == cudaSuccess) e = e2;
    }
    if (st == ABILU_OK && e == cudaSuccess) st = enqueue_restart(b, opts, cf, cs);
    cudaGraph_t g = nullptr;
    cudaError_t e3 = cudaStreamEndCapture(cs, &g);
    const long long captured = (long long)(launches() - l0);
    note_launches(-captured);   // captured, not launched: replays are counted
    b->g_step = cf.m ? (long long)in_steps / cf.m : 0;
    b->g_fixed = captured - (long long)in_steps;
    if (st != ABILU_OK || e != cudaSuccess || e3 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        if (st != ABILU_OK) return st;
        return cuda_fail(e != cudaSuccess ? e : e3, "batch_solve: conditional graph capture");
    }
    *out = g;
    return ABILU_OK;
}

static abilu_status batch_solve_core(abilu_batch b, const fgmres_opts *opts, fgmres_result *res,
                                     cudaStream_t st);

extern "C" abilu_status abilu_batch_solve(abilu_batch b, const fgmres_opts *opts,
                                          fgmres_result *res, abilu_stream stream) {
    if (!b || !opts || !res) return fail(ABILU_EINVAL, "batch_solve: NULL argument");
    if (b->arena) return fail(ABILU_EINVAL, "batch_solve: a server's arena is solved by abilu_server_step");
    return batch_solve_core(b, opts, res, S(stream));
}

static abilu_status batch_solve_core(abilu_batch b, const fgmres_opts *opts, fgmres_result *res,
                                     cudaStream_t st) {
    const int m = opts->restart;
    if (m < 1 || m > BMAXM) return fail(ABILU_EINVAL, "batch_solve: restart must be in 1..%d", BMAXM);
    if (opts->max_iters < 0 || !(opts->rtol >= 0.0) || opts->apply_sweeps_lower < 0 ||
        opts->apply_sweeps_upper < 0 || opts->build_sweeps < 0 || opts->spin_limit < 0 ||
        (opts->mode != ABILU_SYNC && opts->mode != ABILU_ASYNC))
        return fail(ABILU_EINVAL, "batch_solve: bad options");
    // the solve's spin limit for its build and its sweeps (captured graphs
    // keep it: it is part of the graph key)
    b->fac->spin_limit = (unsigned long long)opts->spin_limit;
    const PatternView &P = b->pat->v;
    const size_t nv = (size_t)b->rows * BS;
    if (!b->krylov || b->krylov_m < m) {
        if (b->arena)   // the arena's Krylov workspace is sized once, at creation
            return fail(ABILU_EINVAL, "server step: restart %d exceeds the server's %d", m, b->krylov_m);
        if (b->krylov) cudaFree(b->krylov);
        b->krylov = nullptr;
        if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
        ABILU_CUDA(cudaMalloc(&b->krylov, sizeof(double) * nv * (2 * (size_t)m + 2)));
        b->krylov_m = m;
    }
    double *V = b->krylov;
    float *v32 = reinterpret_cast<float *>(b->fac->r32);
    const BConf cf = {opts->rtol, opts->max_iters, m};
    const int nck = b->nchunks, nsys = b->nsys;
    const BStart ys = batch_start(b, opts);
    abilu_status s;
    if (opts->build) {
        ABILU_CUDA(cudaMemsetAsync(b->fac->ctr, 0, sizeof(unsigned long long), st));
        s = build_dispatch(b->fac, b->A, opts->build_sweeps, (abilu_mode)opts->mode,
                           (abilu_init)opts->init, st);
        if (s != ABILU_OK) return s;
    }
    ABILU_CUDA(cudaMemsetAsync(b->x, 0, sizeof(double) * nv, st));
    ABILU_CUDA(cudaMemsetAsync(b->S, 0, sizeof(BState) * nsys, st));
    k_b_init<<<counted((nsys + 127) / 128), 128, 0, st>>>(b->S, nsys);
    k_b_flags_reset<<<counted(1), 32, 0, st>>>(b->bflag);
    launch_pdl(k_b_residual, b->nsc, RED_THREADS, 0, st, P, b->A, b->b, b->x, V, b->S, batch_tab(b),
        b->partials, cf, 1, b->hs_done, b->hs_fin, b->sys_done, b->bflag);
    launch_pdl(k_b_scale, nck, RED_THREADS, 0, st, V, V, v32, b->S, b->chunk_sys, ys.y0, ys.tk);
    ABILU_LAUNCH_CHECK("batch init");
    // the cycle graph: captured once per (restart, sweeps, mode, Gram-Schmidt
    // form, factor buffer, spin limit, tolerance, iteration limit: the kernels
    // take the last two by value), replayed for every cycle of every later solve
    unsigned long long rbits;
    memcpy(&rbits, &opts->rtol, sizeof rbits);
    const int key[12] = {m, opts->apply_sweeps_lower, opts->apply_sweeps_upper, opts->mode,
                         gs_form(opts), (int)b->fac->cur, (int)(opts->spin_limit >> 32),
                         (int)(opts->spin_limit & 0xffffffff), (int)(rbits >> 32),
                         (int)(rbits & 0xffffffff), opts->max_iters, 0};
    if (b->graph && memcmp(key, b->gkey, sizeof key) != 0) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    if (!b->graph && !b->no_graph) {
        apply_warm(b->fac->dtype);
        cudaGraph_t g = nullptr;
        if (capture_cycle(b, opts, cf, &g) == ABILU_OK &&
            cudaGraphInstantiate(&b->graph, g, 0) == cudaSuccess) {
            memcpy(b->gkey, key, sizeof key);
        } else {
            b->graph = nullptr;
            b->no_graph = 1;   // this runtime cannot: use the host-driven loop
        }
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
    }
    ABILU_CUDA(cudaMemsetAsync(b->bflag + 2, 0, sizeof(int), st));
    ABILU_CUDA(cudaStreamSynchronize(st));
    abilu_status ret = ABILU_OK;
    int cycles = 0, replays = 0;
    while (!all_set(b->hs_fin, nsys) && cycles <= opts->max_iters) {
        cycles++;
        cudaError_t e = cudaSuccess;
        if (b->graph) {
            e = cudaGraphLaunch(b->graph, st);
            replays++;
        } else {  // host-driven: look at step j-1 while step j runs
            cudaEvent_t ev[2];
            cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming);
            cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming);
            for (int j = 0; j < m; j++) {
                if ((ret = enqueue_step(b, opts, cf, j, st)) != ABILU_OK) break;
                if ((e = cudaEventRecord(ev[j & 1], st)) != cudaSuccess) break;
                if (j >= 1) {
                    if ((e = cudaEventSynchronize(ev[(j - 1) & 1])) != cudaSuccess) break;
                    if (all_set(b->hs_done, nsys)) break;
                }
            }
            cudaEventDestroy(ev[0]);
            cudaEventDestroy(ev[1]);
            if (ret != ABILU_OK) break;
            if (e != cudaSuccess) { ret = cuda_fail(e, "batch step wait"); break; }
            if ((ret = enqueue_restart(b, opts, cf, st)) != ABILU_OK) break;
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { ret = cuda_fail(e, "batch cycle"); break; }
    }
    if (replays) {
        int steps = 0;
        ABILU_CUDA(cudaMemcpy(&steps, b->bflag + 2, sizeof steps, cudaMemcpyDeviceToHost));
        note_launches(replays * b->g_fixed + (long long)steps * b->g_step);
    }
    std::vector<BState> hs(nsys);
    ABILU_CUDA(cudaMemcpy(hs.data(), b->S, sizeof(BState) * nsys, cudaMemcpyDeviceToHost));
    unsigned long long cv[5] = {0, 0, 0, 0, 0};
    ABILU_CUDA(cudaMemcpy(cv, b->fac->ctr, sizeof cv, cudaMemcpyDeviceToHost));
    const unsigned long long ns = cv[0];
    if (cv[4] && ret == ABILU_OK) {  // a staged sweep's bounded wait ran out: results invalid
        cudaMemset(b->fac->ctr + 4, 0, sizeof(unsigned long long));
        ret = fail(ABILU_ETIMEOUT, "batch_solve: %llu pipeline waits timed out", cv[4]);
    }
    int nconv = 0;
    for (int q = 0; q < nsys; q++) {
        res[q].iters = hs[q].iters;
        res[q].restarts = hs[q].restarts;
        res[q].rel_resid_est = hs[q].est;
        res[q].rel_resid_true = hs[q].bnorm > 0.0 ? hs[q].beta / hs[q].bnorm : 0.0;
        res[q].singular_blocks = (int64_t)ns;
        res[q].status = hs[q].converged ? (ns ? ABILU_WARN_SINGULAR : ABILU_OK) : ABILU_ENOCONV;
        nconv += hs[q].converged;
    }
    if (ret == ABILU_OK && nconv < nsys)
        ret = fail(ABILU_ENOCONV, "batch_solve: %d of %d systems did not converge", nsys - nconv, nsys);
    else if (ret == ABILU_OK && ns)
        ret = fail(ABILU_WARN_SINGULAR, "batch_solve: %llu singular diagonal blocks replaced", ns);
    return ret;
}

// ===================================================================== server
// Continuous batching (abilu_server_*): the systems of many requests share
// every launch of a step -- one batched solve of one value update of every
// admitted system -- and systems join and leave between steps.
//
// The server owns an arena: a batch allocated once for capacities (rows,
// blocks, L and U blocks, product pairs, work items, systems), so admission
// and departure allocate and free nothing in it.  Each admitted system's
// pattern is analysed once, at admission, into its own pattern handle (local
// indices).  Whenever the set of systems in a step differs from the arena's
// current layout, the systems are laid out packed, in the step's order: each
// local analysis is copied into the arena with its row, block, L, U, pair and
// work offsets added (k_relocate; plus the padding rows to a multiple of 64:
// identity diagonal blocks, b = 0, one diagonal work item each), and the
// factors of the systems that continue are moved from their old place in the
// current factor buffer to their new place in the other one (the warm start
// of Sec. 6 setup survives the move).  A departed system's share of the arena
// is free from the next layout on; its pattern handle is released at once.
namespace abilu {

struct Reloc {
    int R, n, np;          // row base, rows, padded rows
    int B, nnzb;           // block base, blocks (padding blocks follow)
    int Lb, nl, Ub, nu;    // bases and counts in the compact L and U arrays
    int Pb, npairs;        // product pairs
    int Wb, nwork;         // work items (padding diagonal items follow)
};

__global__ void k_relocate(PatternView s, Reloc o, int32_t *__restrict__ rowptr,
                           int32_t *__restrict__ colind, int32_t *__restrict__ diagpos,
                           int32_t *__restrict__ lrow, int32_t *__restrict__ urow,
                           int32_t *__restrict__ lcol, int32_t *__restrict__ ucol,
                           int32_t *__restrict__ pair_ptr, int2 *__restrict__ pairs,
                           WorkItem *__restrict__ work, int32_t *__restrict__ wpos,
                           double *__restrict__ A, double *__restrict__ b) {
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stp = (long long)gridDim.x * blockDim.x;
    const int npad = o.np - o.n;
    for (long long i = t0; i <= o.np; i += stp) {   // rows, and the terminal row entry
        const int r = o.R + (int)i;
        if (i < o.n) {
            rowptr[r] = o.B + s.rowptr[i];
            diagpos[r] = o.B + s.diagpos[i];
            lrow[r] = o.Lb + s.lrow[i];
            urow[r] = o.Ub + s.urow[i];
        } else {
            const int k = (int)i - o.n;
            rowptr[r] = o.B + o.nnzb + k;
            lrow[r] = o.Lb + o.nl;
            urow[r] = o.Ub + o.nu;
            if (i < o.np) {
                diagpos[r] = o.B + o.nnzb + k;
                for (int c = 0; c < BS; c++) b[(size_t)r * BS + c] = 0.0;
            }
        }
    }
    for (long long p = t0; p <= (long long)o.nnzb + npad; p += stp) {   // blocks, pair_ptr's end
        const int q = o.B + (int)p;
        if (p < o.nnzb) {
            colind[q] = o.R + s.colind[p];
            pair_ptr[q] = o.Pb + s.pair_ptr[p];
            const int w = s.wpos[p];
            wpos[q] = w >= 0 ? o.Wb + w : -1;
        } else if (p < (long long)o.nnzb + npad) {
            const int k = (int)(p - o.nnzb);
            colind[q] = o.R + o.n + k;
            pair_ptr[q] = o.Pb + o.npairs;
            wpos[q] = o.Wb + o.nwork + k;
            for (int e = 0; e < BB; e++) A[(size_t)q * BB + e] = (e % 5 == 0) ? 1.0 : 0.0;
        } else {
            pair_ptr[q] = o.Pb + o.npairs;
        }
    }
    for (long long l = t0; l < o.nl; l += stp) lcol[o.Lb + l] = o.R + s.lcol[l];
    for (long long u = t0; u < o.nu; u += stp) ucol[o.Ub + u] = o.R + s.ucol[u];
    for (long long t = t0; t < o.npairs; t += stp) {
        const int2 pr = s.pairs[t];
        pairs[o.Pb + t] = make_int2(pr.x + o.Lb, pr.y + o.Ub);
    }
    for (long long w = t0; w < (long long)o.nwork + npad; w += stp) {
        WorkItem it;
        if (w < o.nwork) {
            it = s.work[w];
            const int kind = it.kind_np & 3, np = it.kind_np >> 2;
            it.j += o.R;
            it.dst += kind == WORK_L ? o.Lb : (kind == WORK_D ? o.R : o.Ub);
            it.t0 += o.Pb;
            for (int k = 0; k < 2; k++)
                if (k < np) it.pr[k] = make_int2(it.pr[k].x + o.Lb, it.pr[k].y + o.Ub);
        } else {
            const int i = o.R + o.n + (int)(w - o.nwork);
            it.j = i;
            it.dst = i;
            it.kind_np = WORK_D;
            it.t0 = o.Pb + o.npairs;
            it.pr[0] = it.pr[1] = make_int2(0, 0);
        }
        work[o.Wb + w] = it;
    }
}

struct SrvMember {
    int id;
    abilu_pattern p;                       // local analysis, owned
    int n, nnzb, np, nl, nu, npairs, nwork, max_row;
    int R, B, Lb, Ub, Pb, Wb;              // offsets in the current layout
    int laid;                              // placed in the current layout
    int warm;                              // its factors in the arena are a previous update's
    long long blocks_p() const { return (long long)nnzb + (np - n); }
    long long work_p() const { return (long long)nwork + (np - n); }
};

struct SrvCaps {
    long long rows, blocks, nl, nu, pairs, work;
    int sys, restart;
    abilu_dtype dtype;
};

static inline long long rnd64(long long v) { return (v + 63) / 64 * 64; }

static abilu_status server_caps(const abilu_server_opts *o, SrvCaps *c) {
    if (!o) return fail(ABILU_EINVAL, "server: NULL options");
    if (o->max_cells < 64 || o->max_blocks < 64 || o->max_systems < 1 || o->restart < 1 ||
        o->restart > BMAXM || o->max_lower < 0 || o->max_upper < 0 || o->max_pairs < 0 ||
        o->max_work < 0)
        return fail(ABILU_EINVAL, "server: need max_cells, max_blocks >= 64, max_systems >= 1, "
                    "restart in 1..%d, non-negative optional capacities", BMAXM);
    if (o->factor_dtype != ABILU_F64 && o->factor_dtype != ABILU_F32 && o->factor_dtype != ABILU_BF16)
        return fail(ABILU_EINVAL, "server: bad factor dtype");
    c->rows = rnd64(o->max_cells);
    c->blocks = o->max_blocks + (c->rows - o->max_cells);
    // symmetric patterns (the grids' cell graphs) have as many L as U blocks
    c->nl = o->max_lower ? o->max_lower : c->blocks / 2;
    c->nu = o->max_upper ? o->max_upper : c->blocks / 2;
    c->pairs = o->max_pairs ? o->max_pairs : c->blocks;
    c->work = o->max_work ? o->max_work : c->blocks;
    c->sys = o->max_systems;
    c->restart = o->restart;
    c->dtype = (abilu_dtype)o->factor_dtype;
    if (c->rows + 256 > 0x7fffffffLL / BB || c->blocks + 256 > 0x7fffffffLL / BB ||
        c->pairs > 0x7fffffffLL || c->work > 0x7fffffffLL)
        return fail(ABILU_EINVAL, "server: capacities exceed 32-bit block indices");
    return ABILU_OK;
}

}  // namespace abilu

struct abilu_server_s {
    abilu_batch b;
    SrvCaps cap;
    std::vector<SrvMember> mem;   // admitted, in admission order
    std::vector<int> layout;      // ids in the current layout order
    int next_id;
    int *chunk_init;              // device, one per 64-row chunk
    int *staging;                 // pinned host: chunk_sys, sys_chunk0, chunk_init
    int device;
};

static void server_free(abilu_server sv) {
    if (!sv) return;
    for (auto &m : sv->mem)
        if (m.p) abilu_pattern_destroy(m.p);
    if (sv->b) batch_free(sv->b);
    if (sv->staging) cudaFreeHost(sv->staging);
    delete sv;
}

extern "C" void abilu_server_destroy(abilu_server sv) { server_free(sv); }

// device bytes of an arena with these capacities (the allocations below)
static long long arena_bytes(const SrvCaps &c) {
    auto r = [](long long b) { return (b + 255) / 256 * 256; };
    const long long chunks = c.rows / 64;
    const long long esz = c.dtype == ABILU_F64 ? 8 : (c.dtype == ABILU_F32 ? 4 : 2);
    const long long vt = c.dtype == ABILU_F64 ? 8 : 4;
    const bool narrow = c.dtype != ABILU_F64;
    long long b = 0;
    // batch arrays
    b += r(4 * (c.rows + 70)) + r(4 * (c.blocks + 4)) + r(8 * BB * c.blocks) + 2 * r(8 * BS * c.rows);
    b += r(4 * (chunks + 1)) + 2 * r(4 * (c.sys + 1)) + r((long long)sizeof(BState) * c.sys);
    b += r(8 * PSTRIDE * (chunks + 1)) + r(16) + r(4 * (chunks + 1));
    b += r(8 * BS * c.rows * (2 * (long long)c.restart + 2));   // Krylov workspace
    // pattern arrays
    b += r(4 * c.rows) + 2 * r(4 * (c.rows + 70)) + r(4 * (c.nl + 8)) + r(4 * (c.nu + 8));
    b += r(4 * (c.blocks + 2)) + r(8 * (c.pairs + 1)) + r(32 * (c.work + 1)) + r(4 * (c.blocks + 1));
    // factors (abilu_factors_create's single allocation)
    const long long bl = r(esz * BB * c.nl), bu = r(esz * BB * c.nu), bd = r(esz * BB * c.rows);
    const long long bv = r(vt * BS * c.rows);
    b += 2 * bl + 2 * bu + 3 * bd + 4 * bv + r(8 * 8) + r((long long)solve_state_bytes()) +
         r(8LL * 66 * red_ctas()) + (narrow ? r(4 * BB * c.blocks) + r(4 * BS * c.rows) : 0) +
         (c.dtype == ABILU_F32 ? bu : 0) + r(4 * ((c.work + 31) / 32 + 1));
    return b;
}

extern "C" abilu_status abilu_server_arena_bytes(const abilu_server_opts *o, int64_t *bytes) {
    if (!bytes) return fail(ABILU_EINVAL, "server_arena_bytes: NULL argument");
    SrvCaps c;
    abilu_status s = server_caps(o, &c);
    if (s != ABILU_OK) return s;
    *bytes = arena_bytes(c);
    return ABILU_OK;
}

extern "C" abilu_status abilu_server_create(const abilu_server_opts *o, abilu_stream stream,
                                            abilu_server *out) {
    if (!out) return fail(ABILU_EINVAL, "server_create: out is NULL");
    *out = nullptr;
    SrvCaps c;
    abilu_status s = server_caps(o, &c);
    if (s != ABILU_OK) return s;
    cudaStream_t st = S(stream);
    abilu_server sv = new abilu_server_s();
    sv->cap = c;
    sv->next_id = 0;
    cudaGetDevice(&sv->device);
    abilu_batch b = new abilu_batch_s();
    sv->b = b;
    b->arena = 1;
    b->no_graph = 1;   // the layout changes between steps; host-driven cycles
    b->nsys = 0;
    b->chunk0.push_back(0);
    const long long chunks = c.rows / 64;
    auto cu = [&](cudaError_t e, const char *w) -> abilu_status {
        return e == cudaSuccess ? ABILU_OK : cuda_fail(e, w);
    };
    auto alloc = [&](std::vector<void *> &v, void **p, size_t bytes) -> abilu_status {
        cudaError_t e = cudaMalloc(p, bytes < 16 ? 16 : bytes);
        if (e != cudaSuccess) return cuda_fail(e, "server_create: cudaMalloc");
        v.push_back(*p);
        return ABILU_OK;
    };
#define TRY(x)                                                  \
    do {                                                        \
        abilu_status s_ = (x);                                  \
        if (s_ != ABILU_OK) { server_free(sv); return s_; }     \
    } while (0)
    std::vector<void *> &ba = b->allocs;
    TRY(alloc(ba, (void **)&b->rowptr, sizeof(int32_t) * (c.rows + 70)));
    TRY(alloc(ba, (void **)&b->colind, sizeof(int32_t) * (c.blocks + 4)));
    TRY(alloc(ba, (void **)&b->A, sizeof(double) * BB * c.blocks));
    TRY(alloc(ba, (void **)&b->b, sizeof(double) * BS * c.rows));
    TRY(alloc(ba, (void **)&b->x, sizeof(double) * BS * c.rows));
    TRY(alloc(ba, (void **)&b->chunk_sys, sizeof(int) * (chunks + 1)));
    TRY(alloc(ba, (void **)&b->sys_chunk0, sizeof(int) * (c.sys + 1)));
    TRY(alloc(ba, (void **)&b->sc_tab, sizeof(int) * (2 * (size_t)chunks + c.sys + 2)));
    TRY(alloc(ba, (void **)&b->S, sizeof(BState) * c.sys));
    TRY(alloc(ba, (void **)&b->partials, sizeof(double) * PSTRIDE * (chunks + 1)));
    TRY(alloc(ba, (void **)&b->sys_done, sizeof(int) * (c.sys + 1)));
    TRY(alloc(ba, (void **)&b->bflag, sizeof(int) * 4));
    TRY(alloc(ba, (void **)&sv->chunk_init, sizeof(int) * (chunks + 1)));
    TRY(cu(cudaMalloc(&b->krylov, sizeof(double) * BS * c.rows * (2 * (size_t)c.restart + 2)),
           "server_create: Krylov workspace"));
    b->krylov_m = c.restart;
    TRY(cu(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking), "stream"));
    TRY(cu(cudaStreamCreateWithFlags(&b->body_stream, cudaStreamNonBlocking), "stream"));
    TRY(cu(cudaHostAlloc((void **)&b->hs_done, sizeof(int) * c.sys, cudaHostAllocMapped), "hostalloc"));
    TRY(cu(cudaHostAlloc((void **)&b->hs_fin, sizeof(int) * c.sys, cudaHostAllocMapped), "hostalloc"));
    // staging: chunk_sys [chunks], sys_chunk0 [systems + 1], chunk_init [chunks],
    // super-chunk tables [2 chunks + systems + 2]
    TRY(cu(cudaHostAlloc((void **)&sv->staging, sizeof(int) * (4 * chunks + 2 * c.sys + 3),
                         cudaHostAllocDefault), "hostalloc"));
    // the arena's pattern: arrays with the capacities, analysed by relocation
    abilu_pattern p = new abilu_pattern_s();
    memset(&p->v, 0, sizeof p->v);
    auto pv = new std::vector<void *>();
    p->mem = pv;
    p->device = sv->device;
    b->pat = p;
    int32_t *diagpos, *lrow, *urow, *lcol, *ucol, *pair_ptr, *wpos;
    int2 *pairs;
    WorkItem *work;
    TRY(alloc(*pv, (void **)&diagpos, sizeof(int32_t) * c.rows));
    TRY(alloc(*pv, (void **)&lrow, sizeof(int32_t) * (c.rows + 70)));
    TRY(alloc(*pv, (void **)&urow, sizeof(int32_t) * (c.rows + 70)));
    TRY(alloc(*pv, (void **)&lcol, sizeof(int32_t) * (c.nl + 8)));
    TRY(alloc(*pv, (void **)&ucol, sizeof(int32_t) * (c.nu + 8)));
    TRY(alloc(*pv, (void **)&pair_ptr, sizeof(int32_t) * (c.blocks + 2)));
    TRY(alloc(*pv, (void **)&pairs, sizeof(int2) * (c.pairs + 1)));
    TRY(alloc(*pv, (void **)&work, sizeof(WorkItem) * (c.work + 1)));
    TRY(alloc(*pv, (void **)&wpos, sizeof(int32_t) * (c.blocks + 1)));
    p->v.rowptr = b->rowptr;
    p->v.colind = b->colind;
    p->v.diagpos = diagpos;
    p->v.lrow = lrow;
    p->v.urow = urow;
    p->v.lcol = lcol;
    p->v.ucol = ucol;
    p->v.pair_ptr = pair_ptr;
    p->v.pairs = pairs;
    p->v.work = work;
    p->v.wpos = wpos;
    // factor storage for the capacities, then the pattern is empty until a step
    p->v.n = (int32_t)c.rows;
    p->v.nnzb = (int32_t)c.blocks;
    p->v.nl = (int32_t)c.nl;
    p->v.nu = (int32_t)c.nu;
    p->v.nwork = (int32_t)c.work;
    TRY(abilu_factors_create(p, c.dtype, &b->fac));
    p->v.n = p->v.nnzb = p->v.nl = p->v.nu = p->v.nwork = 0;
    p->v.npairs = 0;
    TRY(cu(cudaMemsetAsync(b->A, 0, sizeof(double) * BB * c.blocks, st), "memset A"));
    TRY(cu(cudaStreamSynchronize(st), "sync"));
#undef TRY
    *out = sv;
    return ABILU_OK;
}

static void server_totals(const abilu_server sv, long long t[7]) {
    for (int k = 0; k < 7; k++) t[k] = 0;
    for (const auto &m : sv->mem) {
        t[0] += m.np;
        t[1] += m.blocks_p();
        t[2] += m.nl;
        t[3] += m.nu;
        t[4] += m.npairs;
        t[5] += m.work_p();
        t[6] += 1;
    }
}

extern "C" abilu_status abilu_server_usage(abilu_server sv, int64_t *out) {
    if (!sv || !out) return fail(ABILU_EINVAL, "server_usage: NULL argument");
    const SrvCaps &c = sv->cap;
    const long long cap[7] = {c.rows, c.blocks, c.nl, c.nu, c.pairs, c.work, c.sys};
    long long t[7];
    server_totals(sv, t);
    for (int k = 0; k < 7; k++) {
        out[k] = cap[k];
        out[7 + k] = t[k];
    }
    return ABILU_OK;
}

// room in the arena for one more system of n cells and nnzb blocks (the
// counts that need no analysis)
static abilu_status server_room(abilu_server sv, long long n, long long nnzb, const char *who) {
    const SrvCaps &c = sv->cap;
    long long t[7];
    server_totals(sv, t);
    const long long np = rnd64(n), bp = nnzb + (np - n);
    if (t[6] + 1 > c.sys || t[0] + np > c.rows || t[1] + bp > c.blocks)
        return fail(ABILU_ENOMEM, "%s: the arena has no room for %lld cells / %lld blocks now "
                    "(%lld of %lld rows, %lld of %lld blocks, %lld of %d systems in use)", who, n,
                    nnzb, t[0], c.rows, t[1], c.blocks, t[6], c.sys);
    return ABILU_OK;
}

static abilu_status server_admit(abilu_server sv, abilu_pattern p, int32_t *id);

extern "C" abilu_status abilu_server_add(abilu_server sv, int32_t n, int32_t nnzb,
                                         const int32_t *rowptr, const int32_t *colind,
                                         abilu_stream stream, int32_t *id) {
    if (!sv || !rowptr || !colind || !id) return fail(ABILU_EINVAL, "server_add: NULL argument");
    if (n < 1 || nnzb < n) return fail(ABILU_EINVAL, "server_add: need n >= 1 and nnzb >= n");
    abilu_status s = server_room(sv, n, nnzb, "server_add");
    if (s != ABILU_OK) return s;
    abilu_pattern p = nullptr;
    s = abilu_pattern_create(n, nnzb, rowptr, colind, stream, &p);
    if (s != ABILU_OK) return s;
    s = server_admit(sv, p, id);
    if (s != ABILU_OK) abilu_pattern_destroy(p);
    return s;
}

extern "C" abilu_status abilu_server_add_pattern(abilu_server sv, abilu_pattern p, int32_t *id) {
    if (!sv || !p || !id) return fail(ABILU_EINVAL, "server_add_pattern: NULL argument");
    if (p->device != sv->device)
        return fail(ABILU_EINVAL, "server_add_pattern: the pattern lives on another device");
    abilu_status s = server_room(sv, p->v.n, p->v.nnzb, "server_add_pattern");
    if (s != ABILU_OK) return s;
    return server_admit(sv, p, id);
}

// admit an analysed pattern (the server owns it on success)
static abilu_status server_admit(abilu_server sv, abilu_pattern p, int32_t *id) {
    const SrvCaps &c = sv->cap;
    long long t[7];
    server_totals(sv, t);
    const int n = p->v.n, nnzb = p->v.nnzb;
    const long long np = rnd64(n);
    SrvMember m = {};
    m.id = sv->next_id;
    m.p = p;
    m.n = n;
    m.nnzb = nnzb;
    m.np = (int)np;
    m.nl = p->v.nl;
    m.nu = p->v.nu;
    m.npairs = (int)p->v.npairs;
    m.nwork = p->v.nwork;
    m.max_row = p->max_row;
    if (t[2] + m.nl > c.nl || t[3] + m.nu > c.nu || t[4] + m.npairs > c.pairs ||
        t[5] + m.work_p() > c.work)
        return fail(ABILU_ENOMEM, "server_add: the arena has no room for the system's L/U blocks, "
                    "product pairs or work items now");
    sv->next_id++;
    sv->mem.push_back(m);
    *id = m.id;
    return ABILU_OK;
}

extern "C" abilu_status abilu_server_remove(abilu_server sv, int32_t id) {
    if (!sv) return fail(ABILU_EINVAL, "server_remove: NULL server");
    for (size_t k = 0; k < sv->mem.size(); k++) {
        if (sv->mem[k].id != id) continue;
        abilu_pattern_destroy(sv->mem[k].p);
        sv->mem.erase(sv->mem.begin() + (long)k);
        return ABILU_OK;
    }
    return fail(ABILU_EINVAL, "server_remove: no system %d", id);
}

// Lay the systems `order` (indices into sv->mem) out packed, as described
// above.  Asynchronous on st.
static abilu_status server_relayout(abilu_server sv, const std::vector<int> &order,
                                    cudaStream_t st) {
    abilu_batch b = sv->b;
    abilu_factors f = b->fac;
    abilu_pattern P = b->pat;
    const int k = (int)order.size();
    std::vector<Reloc> rel(k);
    long long R = 0, B = 0, Lb = 0, Ub = 0, Pb = 0, Wb = 0;
    int maxrow = 0;
    for (int q = 0; q < k; q++) {
        const SrvMember &m = sv->mem[order[q]];
        rel[q] = Reloc{(int)R, m.n, m.np, (int)B, m.nnzb, (int)Lb, m.nl, (int)Ub, m.nu, (int)Pb,
                       m.npairs, (int)Wb, m.nwork};
        R += m.np;
        B += m.blocks_p();
        Lb += m.nl;
        Ub += m.nu;
        Pb += m.npairs;
        Wb += m.work_p();
        maxrow = m.max_row > maxrow ? m.max_row : maxrow;
    }
    // the warm factors of continuing systems: current buffer, old place ->
    // other buffer, new place
    const int c = f->cur, o = 1 - c;
    const size_t eb = f->esz * BB;
    char **L = reinterpret_cast<char **>(f->L), **U = reinterpret_cast<char **>(f->U);
    char **D = reinterpret_cast<char **>(f->D);
    for (int q = 0; q < k; q++) {
        const SrvMember &m = sv->mem[order[q]];
        if (!m.laid || !m.warm) continue;
        if (m.nl)
            ABILU_CUDA(cudaMemcpyAsync(L[o] + rel[q].Lb * eb, L[c] + (size_t)m.Lb * eb, m.nl * eb,
                                       cudaMemcpyDeviceToDevice, st));
        if (m.nu)
            ABILU_CUDA(cudaMemcpyAsync(U[o] + rel[q].Ub * eb, U[c] + (size_t)m.Ub * eb, m.nu * eb,
                                       cudaMemcpyDeviceToDevice, st));
        ABILU_CUDA(cudaMemcpyAsync(D[o] + (size_t)rel[q].R * eb, D[c] + (size_t)m.R * eb,
                                   (size_t)m.np * eb, cudaMemcpyDeviceToDevice, st));
    }
    f->cur = o;
    PatternView &v = P->v;
    for (int q = 0; q < k; q++) {
        const SrvMember &m = sv->mem[order[q]];
        const Reloc &r = rel[q];
        long long work = r.np + 1;
        if (r.nnzb + (r.np - r.n) + 1 > work) work = r.nnzb + (r.np - r.n) + 1;
        if (r.nwork + (r.np - r.n) > work) work = r.nwork + (r.np - r.n);
        if (r.npairs > work) work = r.npairs;
        int grid = (int)((work + 255) / 256);
        if (grid > 4 * red_ctas()) grid = 4 * red_ctas();
        k_relocate<<<counted(grid), 256, 0, st>>>(
            m.p->v, r, b->rowptr, b->colind, const_cast<int32_t *>(v.diagpos),
            const_cast<int32_t *>(v.lrow), const_cast<int32_t *>(v.urow),
            const_cast<int32_t *>(v.lcol), const_cast<int32_t *>(v.ucol),
            const_cast<int32_t *>(v.pair_ptr), const_cast<int2 *>(v.pairs),
            const_cast<WorkItem *>(v.work), const_cast<int32_t *>(v.wpos), b->A, b->b);
        ABILU_LAUNCH_CHECK("k_relocate");
    }
    // chunk tables
    const int nck = (int)(R / 64);
    int *h_chunk_sys = sv->staging, *h_c0 = sv->staging + sv->cap.rows / 64;
    for (int q = 0; q < k; q++) {
        const int c0 = rel[q].R / 64, c1 = c0 + rel[q].np / 64;
        for (int ch = c0; ch < c1; ch++) h_chunk_sys[ch] = q;
        h_c0[q] = c0;
    }
    h_c0[k] = nck;
    ABILU_CUDA(cudaMemcpyAsync(b->chunk_sys, h_chunk_sys, sizeof(int) * nck, cudaMemcpyHostToDevice, st));
    ABILU_CUDA(cudaMemcpyAsync(b->sys_chunk0, h_c0, sizeof(int) * (k + 1), cudaMemcpyHostToDevice, st));
    // the batch's sizes and per-system tables, the pattern's counts
    b->nsys = k;
    b->rows = (int)R;
    b->blocks = (int)B;
    b->nchunks = nck;
    b->n.assign(k, 0);
    b->nnzb.assign(k, 0);
    b->row_off.assign(k, 0);
    b->nnz_off.assign(k, 0);
    b->chunk0.assign(k + 1, nck);
    for (int q = 0; q < k; q++) {
        SrvMember &m = sv->mem[order[q]];
        const Reloc &r = rel[q];
        b->n[q] = m.n;
        b->nnzb[q] = m.nnzb;
        b->row_off[q] = r.R;
        b->nnz_off[q] = r.B;
        b->chunk0[q] = r.R / 64;
        m.R = r.R;
        m.B = r.B;
        m.Lb = r.Lb;
        m.Ub = r.Ub;
        m.Pb = r.Pb;
        m.Wb = r.Wb;
        m.laid = 1;
    }
    v.n = (int32_t)R;
    v.nnzb = (int32_t)B;
    v.nl = (int32_t)Lb;
    v.nu = (int32_t)Ub;
    v.npairs = Pb;
    v.nwork = (int32_t)Wb;
    P->max_row = maxrow;
    abilu_status sst = batch_super_chunks(b, sv->staging + 2 * (sv->cap.rows / 64) + sv->cap.sys + 1,
                                          st);
    if (sst != ABILU_OK) return sst;
    sv->layout.clear();
    for (int q = 0; q < k; q++) sv->layout.push_back(sv->mem[order[q]].id);
    return ABILU_OK;
}

extern "C" abilu_status abilu_server_step(abilu_server sv, int32_t k, const int32_t *ids,
                                          const double *const *A, const double *const *rhs,
                                          double *const *x, const fgmres_opts *opts,
                                          fgmres_result *res, abilu_stream stream) {
    if (!sv || !ids || !A || !rhs || !x || !opts || !res)
        return fail(ABILU_EINVAL, "server_step: NULL argument");
    if (k < 1 || k != (int)sv->mem.size())
        return fail(ABILU_EINVAL, "server_step: the step must list every admitted system once "
                    "(%d listed, %zu admitted)", k, sv->mem.size());
    if (!opts->build) return fail(ABILU_EINVAL, "server_step: every step builds (opts->build = 1)");
    cudaStream_t st = S(stream);
    std::vector<int> order(k);
    for (int q = 0; q < k; q++) {
        int idx = -1;
        for (size_t t = 0; t < sv->mem.size(); t++)
            if (sv->mem[t].id == ids[q]) idx = (int)t;
        if (idx < 0) return fail(ABILU_EINVAL, "server_step: system %d is not admitted", ids[q]);
        for (int t = 0; t < q; t++)
            if (order[t] == idx) return fail(ABILU_EINVAL, "server_step: system %d listed twice", ids[q]);
        if (!A[q] || !rhs[q] || !x[q]) return fail(ABILU_EINVAL, "server_step: NULL array of system %d", ids[q]);
        order[q] = idx;
    }
    bool same = (int)sv->layout.size() == k;
    for (int q = 0; same && q < k; q++) same = sv->layout[q] == ids[q];
    abilu_status s;
    if (!same && (s = server_relayout(sv, order, st)) != ABILU_OK) return s;
    abilu_batch b = sv->b;
    // this step's values and right-hand sides (device or pinned host memory)
    for (int q = 0; q < k; q++) {
        const SrvMember &m = sv->mem[order[q]];
        ABILU_CUDA(cudaMemcpyAsync(b->A + (size_t)m.B * BB, A[q], sizeof(double) * BB * m.nnzb,
                                   cudaMemcpyDefault, st));
        ABILU_CUDA(cudaMemcpyAsync(b->b + (size_t)m.R * BS, rhs[q], sizeof(double) * BS * m.n,
                                   cudaMemcpyDefault, st));
    }
    // new systems start from A, continuing ones from their factors (warm start)
    int *h_init = sv->staging + sv->cap.rows / 64 + sv->cap.sys + 1;
    for (int q = 0; q < k; q++) {
        const SrvMember &m = sv->mem[order[q]];
        for (int ch = m.R / 64; ch < (m.R + m.np) / 64; ch++) h_init[ch] = m.warm ? 0 : 1;
    }
    ABILU_CUDA(cudaMemcpyAsync(sv->chunk_init, h_init, sizeof(int) * b->nchunks,
                               cudaMemcpyHostToDevice, st));
    b->fac->chunk_init = sv->chunk_init;
    fgmres_opts o = *opts;
    o.init = ABILU_INIT_FROM_A;
    s = batch_solve_core(b, &o, res, st);
    b->fac->chunk_init = nullptr;
    if (s != ABILU_OK && s != ABILU_ENOCONV && s != ABILU_WARN_SINGULAR) return s;
    for (int q = 0; q < k; q++) {
        SrvMember &m = sv->mem[order[q]];
        ABILU_CUDA(cudaMemcpyAsync(x[q], b->x + (size_t)m.R * BS, sizeof(double) * BS * m.n,
                                   cudaMemcpyDefault, st));
        m.warm = 1;
    }
    ABILU_CUDA(cudaStreamSynchronize(st));
    return s;
}
