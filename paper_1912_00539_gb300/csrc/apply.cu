// Preconditioner application by block triangular sweeps (Sec. 4.1).
//
//   lower:  y_i <- b_i - sum_{j<i} L_ij y_j          (L_ii = I, Sec. 2)
//   upper:  x_i <- U_ii^{-1} (y_i - sum_{j>i} U_ij x_j)
//
// from zero initial guesses (Sec. 6 setup), n_L sweeps then n_U sweeps.  SYNC
// runs Jacobi sweeps (every read from the previous sweep's vector, double
// buffered); ASYNC runs in-place sweeps with no barrier between them
// (Algorithm 5; backward row order for U), chunks of rows handed out in order
// by a ticket counter.
//
// Shortcuts that do not change the result: from y^0 = 0 the first lower sweep
// gives y^1 = b exactly, so it is not run (the second sweep reads b as y^1);
// and x^1 = Dinv_i y_i needs only row i, so it is fused into the last lower
// sweep.  The last upper sweep writes the FP64 output directly.  In ASYNC mode
// the same first updates are taken: y = b and x^1 = Dinv y are the first
// update of every unknown with every read seeing the zero initial guess, one
// of the orders an asynchronous sweep may run in, and the in-place sweeps then
// perform the remaining n_L - 1 and n_U - 1 updates of each unknown.  With
// FP32/BF16 factors the FP64 right-hand side is converted to FP32 once per
// application (FGMRES hands over the FP32 copy it already wrote).  With FP32
// factors the upper sweeps run on the Dinv-scaled blocks Us_ij = Dinv_i U_ij
// formed once per build: x_i = yh_i - sum_{j>i} Us_ij x_j with yh = Dinv y (formed where
// x^1 = Dinv y is formed), the same iteration without re-reading Dinv in every
// sweep.
//
// Thread mapping: a quad per block row, thread q computes unknown q of the
// row: it reads row q of each factor block (one 16-byte load for FP32, 32 for
// FP64, 8 for BF16; contiguous across the quad) and the neighbour's 4 unknowns
// (one vector load, shared by the quad).  FP32 and BF16 factors run in FP32;
// FP64 factors in FP64.
#include <type_traits>

#include "common.cuh"
#include "pipe.cuh"

namespace abilu {

constexpr int APPLY_THREADS = 256;
constexpr int APPLY_ROWS = APPLY_THREADS / 4;
// The sweeps are bound by the latency of their dependent loads, so the FP32
// ones keep 8 CTAs (64 warps) resident per SM: 32 registers a thread (FP64
// ones, with twice the registers per value, 6).
template <typename VT> constexpr int sweep_min_ctas() { return sizeof(VT) == 4 ? 8 : 6; }

template <typename T> struct ApplyArith { using VT = float; };
template <> struct ApplyArith<double> { using VT = double; };

__device__ __forceinline__ double to_f64v(float v) { return to_f64(v); }
__device__ __forceinline__ double to_f64v(double v) { return v; }

static_assert(APPLY_ROWS == SKIP_CHUNK_ROWS, "one CTA (or ticket) per 64-row chunk");

template <typename VT>
__device__ __forceinline__ VT dot4(const VT a[4], const VT b[4]) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2] + a[3] * b[3];
}

// s - sum over blocks l0..l1-1 of (row q of factor block l) . v[col[l]].
// VOL: the vector is being updated in place by other threads.  (Prefetching
// the row's blocks before the arithmetic was measured slower here: the extra
// registers cost more occupancy than the shorter dependency chain gained.)
template <bool VOL, typename T, typename VT>
__device__ __forceinline__ VT row_sweep_sum(VT s, const T *__restrict__ F,
                                            const int32_t *__restrict__ col, int l0, int l1,
                                            const VT *v) {
    const int q = threadIdx.x & 3;
    for (int l = l0; l < l1; l++) {
        VT a[4], b[4];
        ld_row(F + (size_t)l * BB + q * BS, a);
        ld_row_sel<VOL>(v + (size_t)col[l] * BS, b);
        s -= dot4(a, b);
    }
    return s;
}

// x_i = Dinv_i t_i where thread q holds t_i[q]; returns x_i[q]
template <typename T, typename VT>
__device__ __forceinline__ VT dinv_times(const T *__restrict__ D, int i, VT t) {
    const int q = threadIdx.x & 3;
    VT d[4], tv[4];
    ld_row(D + (size_t)i * BB + q * BS, d);
    tv[0] = qshfl(t, 0); tv[1] = qshfl(t, 1); tv[2] = qshfl(t, 2); tv[3] = qshfl(t, 3);
    return dot4(d, tv);
}

// one Jacobi lower sweep; optionally x^1 = Dinv y fused (into x1 or, when
// it is the last upper result, into z as FP64)
template <typename T, typename VT>
__global__ void __launch_bounds__(APPLY_THREADS)
k_lower_sync(PatternView P, const T *__restrict__ L, const VT *__restrict__ r,
             const VT *__restrict__ yin, VT *__restrict__ yout, const T *__restrict__ D,
             VT *__restrict__ x1, double *__restrict__ z, Skip skip) {
    pdl_wait();
    pdl_trigger();
    if (skip_all(skip) || skip_chunk(skip, blockIdx.x)) return;
    const int i = blockIdx.x * APPLY_ROWS + (threadIdx.x >> 2), q = threadIdx.x & 3;
    if (i >= P.n) return;
    const VT s = row_sweep_sum<false>(r[(size_t)i * BS + q], L, P.lcol, P.lrow[i], P.lrow[i + 1], yin);
    if (yout) yout[(size_t)i * BS + q] = s;
    if (x1 || z) {
        VT x = dinv_times<T, VT>(D, i, s);
        if (x1) x1[(size_t)i * BS + q] = x;
        if (z) z[(size_t)i * BS + q] = to_f64v(x);
    }
}

// x^1 = Dinv y (used when fewer than two lower sweeps run)
template <typename T, typename VT>
__global__ void __launch_bounds__(APPLY_THREADS)
k_diag_apply(PatternView P, const T *__restrict__ D, const VT *__restrict__ y,
             VT *__restrict__ x1, double *__restrict__ z, Skip skip) {
    pdl_wait();
    pdl_trigger();
    if (skip_all(skip) || skip_chunk(skip, blockIdx.x)) return;
    const int i = blockIdx.x * APPLY_ROWS + (threadIdx.x >> 2), q = threadIdx.x & 3;
    if (i >= P.n) return;
    VT t = y[(size_t)i * BS + q];
    VT x = dinv_times<T, VT>(D, i, t);
    if (x1) x1[(size_t)i * BS + q] = x;
    if (z) z[(size_t)i * BS + q] = to_f64v(x);
}

// SCALED: U holds Us = Dinv U and y holds yh = Dinv y, so x = the row sum
template <typename T, typename VT, bool SCALED>
__global__ void __launch_bounds__(APPLY_THREADS, sweep_min_ctas<VT>())
k_upper_sync(PatternView P, const T *__restrict__ U, const T *__restrict__ D,
             const VT *__restrict__ y, const VT *__restrict__ xin, VT *__restrict__ xout,
             double *__restrict__ z, Skip skip) {
    pdl_wait();
    pdl_trigger();
    if (skip_all(skip) || skip_chunk(skip, blockIdx.x)) return;
    const int i = blockIdx.x * APPLY_ROWS + (threadIdx.x >> 2), q = threadIdx.x & 3;
    if (i >= P.n) return;
    const VT s = row_sweep_sum<false>(y[(size_t)i * BS + q], U, P.ucol, P.urow[i], P.urow[i + 1], xin);
    VT x;
    if constexpr (SCALED) x = s;
    else x = dinv_times<T, VT>(D, i, s);
    if (xout) xout[(size_t)i * BS + q] = x;
    if (z) z[(size_t)i * BS + q] = to_f64v(x);
}

// ---------------------------------------------------------------- async
template <typename VT> __device__ __forceinline__ void st_vol(VT *p, VT v);
template <> __device__ __forceinline__ void st_vol<float>(float *p, float v) {
    asm volatile("st.volatile.global.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}
template <> __device__ __forceinline__ void st_vol<double>(double *p, double v) {
    asm volatile("st.volatile.global.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}

// In-place lower sweeps (nsweeps more updates of every row); y holds the first
// update (y = b) on entry.  The last update of a row also forms x^1 = Dinv y
// (into x1, or into z as FP64 when it is the final upper result; with scaled
// upper blocks also into yh, the upper sweeps' right-hand side).
template <typename T, typename VT>
__global__ void __launch_bounds__(APPLY_THREADS, sweep_min_ctas<VT>())
k_lower_async(PatternView P, const T *__restrict__ L, const VT *__restrict__ r, VT *y,
              int nsweeps, const T *__restrict__ D, VT *__restrict__ x1, VT *__restrict__ yh,
              double *__restrict__ z, unsigned long long *ticket, Skip skip) {
    pdl_wait();
    pdl_trigger();
    if (skip_all(skip)) return;
    __shared__ unsigned long long s_t;
    const long long nchunks = (P.n + APPLY_ROWS - 1) / APPLY_ROWS;
    const long long total = nchunks * nsweeps;
    const int q = threadIdx.x & 3;
    for (;;) {
        if (threadIdx.x == 0) s_t = atomicAdd(ticket, 1ull);
        __syncthreads();
        const long long t = (long long)s_t;
        __syncthreads();
        if (t >= total) break;
        const bool last = t / nchunks == nsweeps - 1;
        const int chunk = (int)(t % nchunks);
        const int i = chunk * APPLY_ROWS + (threadIdx.x >> 2);
        if (i < P.n && !skip_chunk(skip, chunk)) {  // quads of a row stay together
            const VT s = row_sweep_sum<true>(r[(size_t)i * BS + q], L, P.lcol, P.lrow[i],
                                             P.lrow[i + 1], (const VT *)y);
            st_vol(y + (size_t)i * BS + q, s);
            if (last && (x1 || z)) {
                const VT x = dinv_times<T, VT>(D, i, s);
                if (x1) x1[(size_t)i * BS + q] = x;
                if (yh) yh[(size_t)i * BS + q] = x;
                if (z) z[(size_t)i * BS + q] = to_f64v(x);
            }
        }
    }
}

// First update of the asynchronous application: y = b, and when no further
// lower sweep runs also x^1 = Dinv b (into x1 or z); resets the two ticket
// counters of the in-place kernels that follow.
template <typename T, typename VT>
__global__ void __launch_bounds__(APPLY_THREADS)
k_async_start(PatternView P, const T *__restrict__ D, const VT *__restrict__ r,
              VT *__restrict__ y, VT *__restrict__ x1, VT *__restrict__ yh, double *__restrict__ z,
              unsigned long long *tickets, Skip skip) {
    pdl_wait();
    pdl_trigger();
    if (skip_all(skip)) return;
    if (blockIdx.x == 0 && threadIdx.x < 2) tickets[threadIdx.x] = 0ull;
    if (skip_chunk(skip, blockIdx.x)) return;
    const int i = blockIdx.x * APPLY_ROWS + (threadIdx.x >> 2), q = threadIdx.x & 3;
    if (i >= P.n) return;
    const VT b = r[(size_t)i * BS + q];
    y[(size_t)i * BS + q] = b;
    if (x1 || z) {
        const VT x = dinv_times<T, VT>(D, i, b);
        if (x1) x1[(size_t)i * BS + q] = x;
        if (yh) yh[(size_t)i * BS + q] = x;
        if (z) z[(size_t)i * BS + q] = to_f64v(x);
    }
}

// In-place upper sweeps (nsweeps more updates of every row), chunks in
// backward order; x holds x^1 on entry.  The last sweep of each chunk also
// writes the FP64 result z.
template <typename T, typename VT, bool SCALED>
__global__ void __launch_bounds__(APPLY_THREADS)
k_upper_async(PatternView P, const T *__restrict__ U, const T *__restrict__ D,
              const VT *__restrict__ y, VT *x, double *__restrict__ z, int nsweeps,
              unsigned long long *ticket, Skip skip) {
    pdl_wait();
    pdl_trigger();
    if (skip_all(skip)) return;
    __shared__ unsigned long long s_t;
    const long long nchunks = (P.n + APPLY_ROWS - 1) / APPLY_ROWS;
    const long long total = nchunks * nsweeps;
    const int q = threadIdx.x & 3;
    for (;;) {
        if (threadIdx.x == 0) s_t = atomicAdd(ticket, 1ull);
        __syncthreads();
        const long long t = (long long)s_t;
        __syncthreads();
        if (t >= total) break;
        const bool last = t / nchunks == nsweeps - 1;
        const int chunk = (int)(nchunks - 1 - t % nchunks);
        const int i = chunk * APPLY_ROWS + (threadIdx.x >> 2);
        if (i < P.n && !skip_chunk(skip, chunk)) {  // quads of a row stay together
            const VT s = row_sweep_sum<true>(y[(size_t)i * BS + q], U, P.ucol, P.urow[i],
                                             P.urow[i + 1], (const VT *)x);
            VT xi;
            if constexpr (SCALED) xi = s;
            else xi = dinv_times<T, VT>(D, i, s);
            st_vol(x + (size_t)i * BS + q, xi);
            if (last) z[(size_t)i * BS + q] = to_f64v(xi);
        }
    }
}

// ---------------------------------------------------------------- staged sweeps
// The sweeps with factors in FP32/BF16, as a warp-specialised pipeline: a
// producer warp picks the next chunk of 64 rows (ASYNC: the next ticket
// (chunk, sweep) from the queue; SYNC: this CTA's next chunk in a static
// round-robin) and copies the chunk's read-only data -- its rows' factor
// blocks and column indices (contiguous in the compact L/U arrays), its row
// pointers and right-hand side -- into one of two shared-memory stages with
// bulk asynchronous copies, while 8 consumer warps (a quad per row) sweep the
// chunk staged before it.  The swept vector is never staged: neighbour values
// are read from global memory at the moment of the update (ASYNC: in place,
// volatile, Algorithm 5; SYNC: from the previous iterate `vin`, written to
// `v`), so each mode computes exactly what its unstaged form computes; only
// the latency of the ticket, the row pointers and the factor rows leaves the
// critical path.  A chunk with more than PIPE_CAP factor blocks reads them
// from global memory.  Lower (UPPER = false): y_i = b_i - sum L_ij y_j; the
// last update of a row also forms x^1 = Dinv_i y_i into x1 / yh / z.  Upper:
// x_i = rhs_i - sum Us_ij x_j (SCALED) or Dinv_i (rhs_i - sum U_ij x_j),
// ASYNC chunks in backward order; the last update writes z.
constexpr int PIPE_CONSUMERS = 8;                          // warps
constexpr int PIPE_THREADS = (PIPE_CONSUMERS + 1) * 32;    // + the producer warp
constexpr int PIPE_CAP = 160;                              // factor blocks per stage
constexpr int PIPE_ROWP = 68;                              // row pointers copied per chunk

template <typename T> struct __align__(128) PipeStage {   // every field 16-byte aligned
    T F[PIPE_CAP * BB];
    int32_t col[PIPE_CAP + 8];
    float rhs[APPLY_ROWS * BS];
    int32_t rowp[PIPE_ROWP];
    long long ticket;     // -1: no more work
    int32_t fb, cb, staged;
    int32_t chunk, last;  // the ticket's chunk and whether it is the chunk's last sweep, formed
                          // once by the producer (a 64-bit division per chunk and consumer
                          // warp was a large share of the consumers' instructions)
    int32_t pad[3];
};

template <bool UPPER, bool SCALED, bool SYNC, typename T>
__global__ void __launch_bounds__(PIPE_THREADS, 7)   // 7 x 288 threads per SM: 32 registers
k_tri_staged(PatternView P, const T *__restrict__ F, const T *__restrict__ D,
             const float *__restrict__ rhs, const float *vin, float *v, int nsweeps, int sync_last,
             float *__restrict__ x1, float *__restrict__ yh, double *__restrict__ z,
             unsigned long long *ticket, unsigned long long *err, Skip skip,
             unsigned long long limit) {
    pdl_wait();
    pdl_trigger();
    if (skip_all(skip)) return;
    __shared__ __align__(128) PipeStage<T> st[2];
    __shared__ __align__(8) uint64_t full[2], empty[2];
    const int32_t *rowp = UPPER ? P.urow : P.lrow;
    const int32_t *colg = UPPER ? P.ucol : P.lcol;
    const long long nchunks = (P.n + APPLY_ROWS - 1) / APPLY_ROWS;
    const long long total = SYNC ? nchunks : nchunks * nsweeps;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        mbar_init(&empty[0], PIPE_CONSUMERS);
        mbar_init(&empty[1], PIPE_CONSUMERS);
        mbar_fence_init();
    }
    __syncthreads();

    if (warp == PIPE_CONSUMERS) {  // ---- producer (one lane)
        if (lane != 0) return;
        // phases armed per stage; before this lane retires (normally or after
        // a timed-out wait) it waits for the copies of the last ones, so the
        // CTA keeps its shared memory until every copy it issued has landed
        int armed[2] = {0, 0};
        // the next chunk's ticket is taken one chunk ahead, and a chunk's row
        // pointers are read before waiting for its stage, so the atomic's and
        // the loads' latency overlap the consumers' work on earlier chunks
        long long tn = SYNC ? (long long)blockIdx.x : (long long)atomicAdd(ticket, 1ull);
        for (int k = 0;; k++) {
            const int s = k & 1, u = k >> 1;
            const long long t = tn;
            const bool more = t < total;
            long long sw = 0;
            int chunk = 0, i0 = 0, i1 = 0, fb = 0, fe = 0;
            if (more) {
                tn = SYNC ? t + gridDim.x : (long long)atomicAdd(ticket, 1ull);
                sw = SYNC ? 0 : t / nchunks;   // SYNC: t < nchunks
                const int c = (int)(t - sw * nchunks);
                chunk = (UPPER && !SYNC) ? (int)(nchunks - 1 - c) : c;
                i0 = chunk * APPLY_ROWS;
                i1 = min(i0 + APPLY_ROWS, P.n);
                fb = rowp[i0];
                fe = rowp[i1];
            }
            if (u >= 1 && !mbar_wait(&empty[s], (u - 1) & 1, err, limit)) break;
            PipeStage<T> &S = st[s];
            if (!more) {
                S.ticket = -1;
                mbar_arrive(&full[s]);
                armed[s]++;
                break;
            }
            const bool staged = fe - fb <= PIPE_CAP;
            const int cb = fb & ~3, ce = (fe + 3) & ~3;
            S.ticket = t;
            S.fb = fb;
            S.cb = cb;
            S.staged = staged;
            S.chunk = chunk;
            S.last = SYNC ? (sync_last != 0) : (sw == nsweeps - 1);
            unsigned bytes = 0;
            const bool run = !skip_chunk(skip, chunk);
            if (run) {
                bytes = PIPE_ROWP * 4 + (unsigned)(i1 - i0) * 16;
                if (staged) bytes += (unsigned)(fe - fb) * BB * sizeof(T) + (unsigned)(ce - cb) * 4;
            }
            mbar_arrive_tx(&full[s], bytes);
            armed[s]++;
            if (run) {
                bulk_g2s(S.rowp, rowp + i0, PIPE_ROWP * 4, &full[s]);
                bulk_g2s(S.rhs, rhs + (size_t)i0 * BS, (unsigned)(i1 - i0) * 16, &full[s]);
                if (staged) {
                    if (fe > fb) bulk_g2s(S.F, F + (size_t)fb * BB, (unsigned)(fe - fb) * BB * sizeof(T), &full[s]);
                    if (ce > cb) bulk_g2s(S.col, colg + cb, (unsigned)(ce - cb) * 4, &full[s]);
                }
            }
        }
        mbar_drain(full, armed, 2, err, limit);
        return;
    }

    // ---- consumers: a quad per row of the staged chunk
    const int r = threadIdx.x >> 2, q = threadIdx.x & 3;
    for (int k = 0;; k++) {
        const int s = k & 1, u = k >> 1;
        if (!mbar_wait(&full[s], u & 1, err, limit)) return;
        const PipeStage<T> &S = st[s];
        if (S.ticket < 0) return;
        const int chunk = S.chunk;
        const bool last = S.last != 0;
        const int i = chunk * APPLY_ROWS + r;
        if (i < P.n && !skip_chunk(skip, chunk)) {
            const int l0 = S.rowp[r], l1 = S.rowp[r + 1];
            float acc = S.rhs[r * BS + q];
            for (int l = l0; l < l1; l++) {
                float a[4], b[4];
                int j;
                if (S.staged) {
                    ld_row(S.F + (size_t)(l - S.fb) * BB + q * BS, a);
                    j = S.col[l - S.cb];
                } else {
                    ld_row(F + (size_t)l * BB + q * BS, a);
                    j = colg[l];
                }
                if constexpr (SYNC) ld_row(vin + (size_t)j * BS, b);
                else ld_row_volatile(v + (size_t)j * BS, b);
                acc -= dot4(a, b);
            }
            float xi = acc;
            if constexpr (UPPER && !SCALED) xi = dinv_times<T, float>(D, i, acc);
            if constexpr (SYNC) {
                if (v) v[(size_t)i * BS + q] = xi;
            } else {
                st_vol(v + (size_t)i * BS + q, xi);
            }
            if (last) {
                if constexpr (UPPER) {
                    if (z) z[(size_t)i * BS + q] = to_f64v(xi);
                } else if (x1 || yh || z) {
                    const float x = dinv_times<T, float>(D, i, acc);
                    if (x1) x1[(size_t)i * BS + q] = x;
                    if (yh) yh[(size_t)i * BS + q] = x;
                    if (z) z[(size_t)i * BS + q] = to_f64v(x);
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
    }
}

// r32 = (float) r, once per application (the sweeps then read 16-byte FP32
// rows and do no FP64 conversions on the slow FP64 pipe)
__global__ void __launch_bounds__(APPLY_THREADS)
k_to_f32(const double *__restrict__ r, float *__restrict__ r32, long long n4) {
    const long long e = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (e >= n4) return;
    double v[4];
    ld_row(r + e, v);
    st_row(r32 + e, v);
}

// v = 0 (n values) unless the launch is skipped: the zero initial guess of the
// in-place sweeps, as a kernel so that a skipped FGMRES step costs no memset
template <typename VT>
__global__ void k_zero(VT *v, long long n, Skip skip) {
    if (skip_all(skip)) return;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) v[e] = (VT)0;
}

template <typename K>
static int resident_ctas(K kernel, int threads) {
    int dev = 0, per_sm = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int c = per_sm * sms;
    return c > 0 ? c : 1;
}

// resident CTAs of the persistent kernels, looked up once (before any stream
// capture: see apply_warm)
template <typename T, typename VT> static int lower_async_ctas() {
    static int c = resident_ctas(k_lower_async<T, VT>, APPLY_THREADS);
    return c;
}
template <typename T, typename VT> static int upper_async_ctas() {
    static int c = resident_ctas(k_upper_async<T, VT, std::is_same<T, float>::value>, APPLY_THREADS);
    return c;
}
template <bool UPPER, bool SCALED, bool SYNC, typename T> static int staged_ctas() {
    static int c = resident_ctas(k_tri_staged<UPPER, SCALED, SYNC, T>, PIPE_THREADS);
    return c;
}


// y_ready (asynchronous mode, FP32/BF16 factors, nl >= 2): the caller already
// wrote y[0] = the FP32 right-hand side and zeroed the two ticket counters in
// an earlier kernel on `st` (FGMRES does it where it writes that right-hand
// side), so k_async_start, which would only do the same, is not launched.
template <typename T>
static abilu_status apply_t(abilu_factors f, const double *r, const float *r32_in, double *z,
                            int nl, int nu, abilu_mode mode, cudaStream_t st, Skip skip,
                            bool y_ready = false) {
    using VT = typename ApplyArith<T>::VT;
    const PatternView &P = f->p->v;
    const int c = f->cur;
    const T *L = reinterpret_cast<const T *>(f->L[c]);
    const T *U = reinterpret_cast<const T *>(f->U[c]);
    const T *D = reinterpret_cast<const T *>(f->D[c]);
    VT *y[2] = {reinterpret_cast<VT *>(f->y[0]), reinterpret_cast<VT *>(f->y[1])};
    VT *x[2] = {reinterpret_cast<VT *>(f->x[0]), reinterpret_cast<VT *>(f->x[1])};
    const int grid = (P.n + APPLY_ROWS - 1) / APPLY_ROWS;

    // right-hand side in the compute type
    const VT *rv;
    if constexpr (sizeof(VT) == 8) {
        rv = r;
    } else {
        if (r32_in) {
            rv = r32_in;
        } else {
            const long long n4 = (long long)P.n * BS;
            k_to_f32<<<counted((int)((n4 / 4 + APPLY_THREADS - 1) / APPLY_THREADS)), APPLY_THREADS,
                       0, st>>>(r, reinterpret_cast<float *>(f->r32), n4);
            ABILU_LAUNCH_CHECK("k_to_f32");
            rv = reinterpret_cast<const float *>(f->r32);
        }
    }

    // FP32 factors: upper sweeps on Us = Dinv U with right-hand side yh = Dinv y
    // (BF16 would round Dinv U to 8 bits and save no bytes)
    constexpr bool SC = std::is_same<T, float>::value;
    const T *UU = SC ? reinterpret_cast<const T *>(f->Us) : U;
    const long long n4 = (long long)P.n * BS;
    if (nl == 0 || nu == 0) {  // y = 0, or no upper update: z = x^0 = 0
        k_zero<double><<<counted((int)((n4 + 255) / 256)), 256, 0, st>>>(z, n4, skip);
        ABILU_LAUNCH_CHECK("apply");
        return ABILU_OK;
    }

    if (mode == ABILU_ASYNC) {
        const long long nchunks = grid;
        unsigned long long *tk = f->ctr + 2;   // [0] lower, [1] upper tickets
        VT *x1 = nu >= 2 ? x[0] : nullptr;     // x^1, updated in place by the upper sweeps
        VT *yh = SC && nu >= 2 ? y[1] : nullptr;
        double *z1 = nu == 1 ? z : nullptr;
        if (!(y_ready && sizeof(VT) == 4 && nl >= 2)) {
            launch_pdl(k_async_start<T, VT>, grid, APPLY_THREADS, 0, st,
                P, D, rv, y[0], nl == 1 ? x1 : nullptr, nl == 1 ? yh : nullptr, nl == 1 ? z1 : nullptr,
                tk, skip);
            ABILU_LAUNCH_CHECK("k_async_start");
        }
        unsigned long long *err = f->ctr + 4;
        const unsigned long long lim = spin_limit_or_default(f->spin_limit);
        if (nl >= 2) {
            if constexpr (sizeof(VT) == 4) {  // staged pipeline (FP32/BF16 factors)
                const int c = staged_ctas<false, false, false, T>();
                const int g = (int)(c < nchunks ? c : nchunks);
                launch_pdl(k_tri_staged<false, false, false, T>, g, PIPE_THREADS, 0, st,
                    P, L, D, rv, nullptr, y[0], nl - 1, 0, x1, yh, z1, tk, err, skip, lim);
            } else {
                const int ctas_l = lower_async_ctas<T, VT>();
                const int g = (int)(ctas_l < nchunks ? ctas_l : nchunks);
                launch_pdl(k_lower_async<T, VT>, g, APPLY_THREADS, 0, st, P, L, rv, y[0], nl - 1, D,
                    x1, yh, z1, tk, skip);
            }
            ABILU_LAUNCH_CHECK("lower async");
        }
        if (nu >= 2) {
            if constexpr (sizeof(VT) == 4) {
                const int c = staged_ctas<true, SC, false, T>();
                const int g = (int)(c < nchunks ? c : nchunks);
                launch_pdl(k_tri_staged<true, SC, false, T>, g, PIPE_THREADS, 0, st,
                    P, UU, D, SC ? y[1] : y[0], nullptr, x[0], nu - 1, 0, nullptr, nullptr, z, tk + 1,
                    err, skip, lim);
            } else {
                const int ctas_u = upper_async_ctas<T, VT>();
                const int g = (int)(ctas_u < nchunks ? ctas_u : nchunks);
                launch_pdl(k_upper_async<T, VT, SC>, g, APPLY_THREADS, 0, st,
                    P, UU, D, SC ? y[1] : y[0], x[0], z, nu - 1, tk + 1, skip);
            }
            ABILU_LAUNCH_CHECK("upper async");
        }
        return ABILU_OK;
    }

    // ---- synchronous: y^1 = r (the first sweep from y = 0), y^s in y[s & 1];
    // x^1 = Dinv y^{n_L} fused into the last lower sweep.  Scaled: that sweep
    // writes only yh = x^1 (in place of y^{n_L}), and the first upper sweep
    // reads x^1 from it.
    const VT *yfin;     // the upper sweeps' right-hand side (y, or yh when scaled)
    const VT *xfirst;   // x^1
    if (nl == 1) {      // no lower sweep runs: x^1 = Dinv r
        VT *x1 = nu >= 2 ? (SC ? y[0] : x[1]) : nullptr;
        launch_pdl(k_diag_apply<T, VT>, grid, APPLY_THREADS, 0, st, P, D, rv, x1,
            nu == 1 ? z : nullptr, skip);
        ABILU_LAUNCH_CHECK("k_diag_apply");
        yfin = SC ? y[0] : rv;
        xfirst = x1;
    } else {
        const VT *yprev = rv;
        VT *x1 = nullptr;
        for (int s = 2; s <= nl; s++) {
            const bool last = s == nl;
            VT *yout = y[s & 1];
            if (last) x1 = nu >= 2 ? (SC ? yout : x[1]) : nullptr;
            // (the staged form was measured slower for this sweep: 19.3 vs 17.1 us)
            launch_pdl(k_lower_sync<T, VT>, grid, APPLY_THREADS, 0, st,
                P, L, rv, yprev, (last && SC) ? nullptr : yout, D, last ? x1 : nullptr,
                (last && nu == 1) ? z : nullptr, skip);
            ABILU_LAUNCH_CHECK("lower sync");
            yprev = yout;
        }
        yfin = yprev;   // y^{n_L}, or yh when scaled (written as x1 into the same buffer)
        xfirst = x1;
    }
    for (int s = 2; s <= nu; s++) {  // x^s in x[s & 1], the last one to z
        const bool last = s == nu;
        const VT *xin = s == 2 ? xfirst : x[(s - 1) & 1];
        if constexpr (sizeof(VT) == 4) {
            const int c = staged_ctas<true, SC, true, T>();
            const int g = c < grid ? c : grid;
            launch_pdl(k_tri_staged<true, SC, true, T>, g, PIPE_THREADS, 0, st,
                P, UU, D, yfin, xin, last ? nullptr : x[s & 1], 1, last ? 1 : 0, nullptr, nullptr,
                last ? z : nullptr, nullptr, f->ctr + 4, skip, spin_limit_or_default(f->spin_limit));
        } else {
            launch_pdl(k_upper_sync<T, VT, SC>, grid, APPLY_THREADS, 0, st,
                P, UU, D, yfin, xin, last ? nullptr : x[s & 1], last ? z : nullptr, skip);
        }
        ABILU_LAUNCH_CHECK("upper sync");
    }
    return ABILU_OK;
}

// Performs the one-time occupancy lookups of the apply kernels of a dtype, so
// that later calls make no such API call (needed inside stream capture).
void apply_warm(abilu_dtype dt) {
    switch (dt) {
    case ABILU_F64: lower_async_ctas<double, double>(); upper_async_ctas<double, double>(); break;
    case ABILU_F32:
        staged_ctas<false, false, false, float>();
        staged_ctas<true, true, false, float>();
        staged_ctas<true, true, true, float>();
        break;
    case ABILU_BF16:
        staged_ctas<false, false, false, __nv_bfloat16>();
        staged_ctas<true, false, false, __nv_bfloat16>();
        staged_ctas<true, false, true, __nv_bfloat16>();
        break;
    }
}

abilu_status scalar_apply(abilu_factors f, const double *r, double *z, int nl, int nu,
                          abilu_mode mode, cudaStream_t st, Skip skip);

abilu_status apply_dispatch(abilu_factors f, const double *r, const float *r32, double *z,
                            int nl, int nu, abilu_mode mode, cudaStream_t st, Skip skip) {
    if (f->scalar) return scalar_apply(f, r, z, nl, nu, mode, st, skip);
    switch (f->dtype) {
    case ABILU_F64: return apply_t<double>(f, r, r32, z, nl, nu, mode, st, skip);
    case ABILU_F32: return apply_t<float>(f, r, r32, z, nl, nu, mode, st, skip);
    case ABILU_BF16: return apply_t<__nv_bfloat16>(f, r, r32, z, nl, nu, mode, st, skip);
    }
    return fail(ABILU_EINVAL, "apply: bad dtype");
}

// The application when apply_y_ready(f, nl, mode) holds and the caller wrote
// y[0] and zeroed the tickets (see apply_t)
abilu_status apply_dispatch_ready(abilu_factors f, const double *r, const float *r32, double *z,
                                  int nl, int nu, abilu_mode mode, cudaStream_t st, Skip skip) {
    if (f->dtype == ABILU_F32)
        return apply_t<float>(f, r, r32, z, nl, nu, mode, st, skip, true);
    return apply_t<__nv_bfloat16>(f, r, r32, z, nl, nu, mode, st, skip, true);
}

// Whether an application can start from a y[0] and tickets prepared by the
// caller: asynchronous block factors in FP32/BF16 with at least two lower
// updates (with one, the start kernel also forms x^1)
bool apply_y_ready(abilu_factors f, int nl, int nu, abilu_mode mode) {
    return !f->scalar && f->dtype != ABILU_F64 && mode == ABILU_ASYNC && nl >= 2 && nu >= 1;
}

}  // namespace abilu
