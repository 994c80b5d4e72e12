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
#include <atomic>

#include "common.cuh"
#include "pipe.cuh"

namespace abilu {

template <typename T> struct BuildArith { using C = float; };
template <> struct BuildArith<double> { using C = double; };

constexpr int BUILD_THREADS = 256;
constexpr int BUILD_ROWS = BUILD_THREADS / 4;  // rows per CTA (= chunk of the async queue)
static_assert(BUILD_ROWS == SKIP_CHUNK_ROWS, "a build CTA's rows are one 64-row chunk");

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

// Inverse of a 4x4 FP32 block accurate to FP32 rounding without FP64
// instructions (FP64 and FP64<->FP32 conversions share this GPU's slow FP64
// pipe).  The quad holding the block (thread q owns row q) computes
//   X0 = adj(U)/det(U) in FP32 (thread q: row q of adj(U), the cofactors of
//        column q),
//   R  = I - U X0 with error-free products and sums (TwoProd by FMA, TwoSum),
//   X1 = X0 + X0 R  (one Newton step),
// so X1 carries an error of about (cond(U) u)^2 + u, u = 2^-24: the FP32
// rounding of the exact inverse for every block with cond(U) << 1/sqrt(u).
// Thread q's cofactors are the 3x3 minors of the other three columns, taken
// in the cyclic order q+1, q+2, q+3 (an even permutation of their natural
// order, so every minor keeps its sign): the same instructions in all four
// threads, no branch on q.  det(U) is thread 0's expansion along column 0,
// shared by the quad, so all four threads reach the same singular decision
// (det == 0 or non-finite: replaced by the identity, modified iteration,
// Sec. 4.2).  `sh` is this quad's scratch of QUAD_SCRATCH floats (U, X0, R);
// the stride of 52 floats puts the 8 quads of a warp on distinct banks.
// refine = false returns X0 (the intermediate sweeps of a synchronous build:
// their inverses only feed the next sweep; its last sweep refines the Dinv
// that the application uses).
constexpr int QUAD_SCRATCH = 52;
__device__ __forceinline__ bool quad_inv4_refined(const float u_row[4], float x_row[4],
                                                  float *sh, bool refine = true) {
    const int q = threadIdx.x & 3;
    const unsigned m = quad_mask();
    float *shU = sh, *shX = sh + 16, *shR = sh + 32;
    reinterpret_cast<float4 *>(shU)[q] = make_float4(u_row[0], u_row[1], u_row[2], u_row[3]);
    __syncwarp(m);
    const int k0 = (q + 1) & 3, k1 = (q + 2) & 3, k2 = (q + 3) & 3;
    float b0[4], b1[4], b2[4], cq[4];   // columns k0, k1, k2 and q of U
#pragma unroll
    for (int r = 0; r < 4; r++) {
        b0[r] = shU[4 * r + k0];
        b1[r] = shU[4 * r + k1];
        b2[r] = shU[4 * r + k2];
        cq[r] = shU[4 * r + q];
    }
    // 2x2 minors of columns (k1, k2), rows (a, b)
    const float m01 = b1[0] * b2[1] - b2[0] * b1[1], m02 = b1[0] * b2[2] - b2[0] * b1[2];
    const float m03 = b1[0] * b2[3] - b2[0] * b1[3], m12 = b1[1] * b2[2] - b2[1] * b1[2];
    const float m13 = b1[1] * b2[3] - b2[1] * b1[3], m23 = b1[2] * b2[3] - b2[2] * b1[3];
    // minor of (row r, column q), then cofactor sign (-1)^(r+q)
    const float sg = (q & 1) ? -1.0f : 1.0f;
    float x0[4];
    x0[0] = sg * (b0[1] * m23 - b0[2] * m13 + b0[3] * m12);
    x0[1] = -sg * (b0[0] * m23 - b0[2] * m03 + b0[3] * m02);
    x0[2] = sg * (b0[0] * m13 - b0[1] * m03 + b0[3] * m01);
    x0[3] = -sg * (b0[0] * m12 - b0[1] * m02 + b0[2] * m01);
    const float det_q = cq[0] * x0[0] + cq[1] * x0[1] + cq[2] * x0[2] + cq[3] * x0[3];
    const float det = __shfl_sync(m, det_q, (threadIdx.x & 31) & ~3);
    if (det == 0.0f || !isfinite(det)) {
#pragma unroll
        for (int c = 0; c < 4; c++) x_row[c] = (c == q) ? 1.0f : 0.0f;
        __syncwarp(m);
        return true;
    }
    const float id = 1.0f / det;
#pragma unroll
    for (int c = 0; c < 4; c++) x0[c] *= id;
    if (!refine) {   // the FP32 adjugate alone (relative error about cond(U) u)
#pragma unroll
        for (int c = 0; c < 4; c++) x_row[c] = x0[c];
        return false;
    }
    reinterpret_cast<float4 *>(shX)[q] = make_float4(x0[0], x0[1], x0[2], x0[3]);
    __syncwarp(m);
    float X[16];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        float4 t = reinterpret_cast<const float4 *>(shX)[k];
        X[4 * k] = t.x; X[4 * k + 1] = t.y; X[4 * k + 2] = t.z; X[4 * k + 3] = t.w;
    }
    // R[q][c] = delta_qc - sum_k U[q][k] X0[k][c], accumulated error-free
    float r[4];
#pragma unroll
    for (int c = 0; c < 4; c++) {
        float acc = (c == q) ? 1.0f : 0.0f, comp = 0.0f;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const float uq = u_row[k], xk = X[4 * k + c];
            const float p = __fmul_rn(uq, xk);
            const float pe = __fmaf_rn(uq, xk, -p);          // uq*xk = p + pe exactly
            const float t = __fsub_rn(acc, p);                // TwoSum(acc, -p)
            const float bp = __fsub_rn(t, acc);
            const float err = __fadd_rn(__fsub_rn(acc, __fsub_rn(t, bp)), __fsub_rn(-p, bp));
            acc = t;
            comp = __fsub_rn(__fadd_rn(comp, err), pe);
        }
        r[c] = acc + comp;
    }
    reinterpret_cast<float4 *>(shR)[q] = make_float4(r[0], r[1], r[2], r[3]);
    __syncwarp(m);
    float R[16];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        float4 t = reinterpret_cast<const float4 *>(shR)[k];
        R[4 * k] = t.x; R[4 * k + 1] = t.y; R[4 * k + 2] = t.z; R[4 * k + 3] = t.w;
    }
#pragma unroll
    for (int c = 0; c < 4; c++) {
        float corr = 0.0f;
#pragma unroll
        for (int k = 0; k < 4; k++) corr += x0[k] * R[4 * k + c];
        x_row[c] = x0[c] + corr;
    }
    __syncwarp(m);
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
        st_row(p, v);
    }
}

// One block row i handled by one quad.  Writes the row's L and U blocks and
// returns row q of U_ii in udiag.
template <typename T, bool VOL, typename AT>
__device__ __forceinline__ void build_row_products(const PatternView &P, int i,
                                                   const AT *__restrict__ A, const T *Lin,
                                                   const T *Uin, const T *Din, T *Lout, T *Uout,
                                                   typename BuildArith<T>::C udiag[4]) {
    using C = typename BuildArith<T>::C;
    const int q = threadIdx.x & 3;
    const int p0 = P.rowptr[i], p1 = P.rowptr[i + 1], dp = P.diagpos[i];
    const int lb = P.lrow[i], ub = P.urow[i];
    for (int p = p0; p < p1; p++) {
        const int t0 = P.pair_ptr[p], t1 = P.pair_ptr[p + 1];
        // U_ij with no product pair equals A_ij in every sweep: written once
        // per build by k_build_prepare into every buffer, skipped here
        if (p > dp && t0 == t1) continue;
        const int j = P.colind[p];
        C s[4];
        ld_row(A + (size_t)p * BB + q * BS, s);
        for (int t = t0; t < t1; t++) {
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
            udiag[0] = s[0]; udiag[1] = s[1]; udiag[2] = s[2]; udiag[3] = s[3];
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

// Dinv_i = inv(U_ii) for the CTA's rows and (if Udiag) U_ii, from row q of
// U_ii held by thread q of each row's quad.  Every thread of the CTA calls it.
template <typename T, bool VOL>
__device__ __forceinline__ void build_finish_rows(int row0, int n, const typename BuildArith<T>::C u[4],
                                                  T *Dout, T *Udiag, double *sh_u, double *sh_d,
                                                  float *sh_q, unsigned long long *nsing) {
    const int i = row0 + (threadIdx.x >> 2), q = threadIdx.x & 3;
    if constexpr (sizeof(T) < 8) {
        if (i < n) {
            float d[4];
            // refined where the inverse is final (Udiag passed: the last sweep,
            // or a prepare pass that no sweep follows)
            if (quad_inv4_refined(u, d, sh_q + (threadIdx.x >> 2) * QUAD_SCRATCH, Udiag != nullptr) &&
                q == 0)
                atomicAdd(nsing, 1ull);
            st_row_sel<VOL>(Dout + (size_t)i * BB + q * BS, d);
            if (Udiag) st_row_sel<false>(Udiag + (size_t)i * BB + q * BS, u);
        }
    } else {
        if (i < n) {
            double *su = sh_u + (threadIdx.x >> 2) * BB + q * BS;
            su[0] = u[0]; su[1] = u[1]; su[2] = u[2]; su[3] = u[3];
        }
        build_cta_invert<T, VOL>(row0, n, Dout, Udiag, sh_u, sh_d, nsing);
    }
}

// shared memory of the build kernels: FP64 inversion scratch or FP32 quad scratch
template <typename T> struct BuildShared {
    static constexpr int D = sizeof(T) == 8 ? BUILD_ROWS * BB : 1;
    static constexpr int F = sizeof(T) == 8 ? 1 : BUILD_ROWS * QUAD_SCRATCH;
};

// ---- block work items (FP32/BF16 factors)
// The block-asynchronous iteration updates one block per step (Eq.
// async_blockilu_fp: the update function ranges over the blocks), so a work
// item here is one block of the pattern's work list, handled by one quad.  Its
// dependency chain is two loads deep: the 32-byte record and the item's FP32 A
// row (stored at the item's index) are read together, then Dinv_j or the rows
// of L_ik and U_kj that the record's inline pairs name (a third level only for
// blocks with more than two pairs).  There are four times more items in
// flight than block rows, which is what hides memory latency on this GPU.
constexpr int WORK_PER_CTA = BUILD_THREADS / 4;
static_assert(WORK_PER_CTA == WORK_CHUNK, "work list chunks are sorted per CTA");
static_assert(sizeof(WorkItem) == 32, "work records are two 16-byte loads");

// s -= L_ik U_kj for the quad's block (thread q: row q); u's row k lives in thread k
__device__ __forceinline__ void sub_product(float s[4], const float l[4], const float u[4]) {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 4; k++)
#pragma unroll
        for (int c = 0; c < 4; c++) acc[c] += l[k] * qshfl(u[c], k);
#pragma unroll
    for (int c = 0; c < 4; c++) s[c] -= acc[c];
}

template <typename T, bool VOL>
__device__ __forceinline__ void build_block(const PatternView &P, int w,
                                            const float *__restrict__ A32, const T *Lin,
                                            const T *Uin, const T *Din, T *Lout, T *Uout, T *Dout,
                                            T *Udiag, float *sh_q, unsigned long long *nsing) {
    const int q = threadIdx.x & 3;
    const WorkItem it = P.work[w];
    float s[4], d[4];
    ld_row(A32 + (size_t)w * BB + q * BS, s);
    const int kind = it.kind_np & 3, np = it.kind_np >> 2, dst = it.dst;
    if (kind == WORK_L) ld_row_sel<VOL>(Din + (size_t)it.j * BB + q * BS, d);
    if (np > 0) {  // products in pair order (ascending k)
        float l0[4], u0[4], l1[4], u1[4];
        ld_row_sel<VOL>(Lin + (size_t)it.pr[0].x * BB + q * BS, l0);  // row q of L_ik
        ld_row_sel<VOL>(Uin + (size_t)it.pr[0].y * BB + q * BS, u0);  // row q of U_kj
        if (np > 1) {
            ld_row_sel<VOL>(Lin + (size_t)it.pr[1].x * BB + q * BS, l1);
            ld_row_sel<VOL>(Uin + (size_t)it.pr[1].y * BB + q * BS, u1);
        }
        sub_product(s, l0, u0);
        if (np > 1) sub_product(s, l1, u1);
        for (int t = 2; t < np; t++) {
            const int2 pr = P.pairs[it.t0 + t];
            ld_row_sel<VOL>(Lin + (size_t)pr.x * BB + q * BS, l0);
            ld_row_sel<VOL>(Uin + (size_t)pr.y * BB + q * BS, u0);
            sub_product(s, l0, u0);
        }
    }
    if (kind == WORK_L) {  // L_ij = S Dinv_j; row k of Dinv_j lives in thread k
        float o[4];
#pragma unroll
        for (int c = 0; c < 4; c++) {
            float d0 = qshfl(d[c], 0), d1 = qshfl(d[c], 1), d2 = qshfl(d[c], 2), d3 = qshfl(d[c], 3);
            o[c] = s[0] * d0 + s[1] * d1 + s[2] * d2 + s[3] * d3;
        }
        st_row_sel<VOL>(Lout + (size_t)dst * BB + q * BS, o);
    } else if (kind == WORK_U) {
        st_row_sel<VOL>(Uout + (size_t)dst * BB + q * BS, s);
    } else {  // U_ii = S, Dinv_i = inv(U_ii), refined only in a build's last sweep, in
              // either mode (Udiag passed): earlier inverses only feed the next updates
        float x[4];
        if (quad_inv4_refined(s, x, sh_q, Udiag != nullptr) && q == 0) atomicAdd(nsing, 1ull);
        st_row_sel<VOL>(Dout + (size_t)dst * BB + q * BS, x);
        if (Udiag) st_row_sel<false>(Udiag + (size_t)dst * BB + q * BS, s);
    }
}

template <typename T>
__global__ void __launch_bounds__(BUILD_THREADS, 6)   // 40 registers: measured fastest
k_build_blocks_sync(PatternView P, const float *__restrict__ A32, const T *__restrict__ Lin,
                    const T *__restrict__ Uin, const T *__restrict__ Din, T *__restrict__ Lout,
                    T *__restrict__ Uout, T *__restrict__ Dout, T *__restrict__ Udiag,
                    unsigned long long *nsing) {
    pdl_wait();
    pdl_trigger();
    __shared__ __align__(16) float sh_q[WORK_PER_CTA * QUAD_SCRATCH];
    const int w = blockIdx.x * WORK_PER_CTA + (threadIdx.x >> 2);
    if (w >= P.nwork) return;  // whole quads leave together
    build_block<T, false>(P, w, A32, Lin, Uin, Din, Lout, Uout, Dout, Udiag,
                          sh_q + (threadIdx.x >> 2) * QUAD_SCRATCH, nsing);
}

// In place.  Each warp takes tickets t = 0 .. nsweeps*nchunks-1 in order from
// one counter (no CTA barrier, so warps never wait for each other); ticket t
// is chunk c = t mod nchunks of sweep t / nchunks.  A chunk is `wchunk` work
// blocks in sub-chunks of `sub` consecutive blocks (64, one kind-sorted group
// of the list, or 32 for sizes that are not multiples of 64) taken at a stride
// of nchunks sub-chunks: sub-chunks c, c + nchunks, c + 2 nchunks, ...  Each
// sub-chunk is done in steps of 8 blocks (one block per quad, consecutive
// blocks, so a step stays within one kind).
//
// Why the stride: the ILU fixed-point residual after a given number of sweeps
// falls as the blocks in flight (resident warps x blocks per ticket) span
// fewer consecutive blocks, because then more of the rows a block reads were
// already updated in the current sweep (the in-place iteration's Gauss-Seidel
// effect).  At 512x512 (1.31 M work blocks, 6,080 warps), 6 sweeps, tickets
// of 128 consecutive blocks left an ILU residual of 44 in 437.7 us, of 64
// blocks 4.1 in 442-444 us (twice the atomics on the one contended counter).
// A 128-block ticket made of two 64-block sub-chunks half the list apart (the
// default) keeps the 128-block atomic count while each half of the list sees
// the 64-block span: 4.9 in 429.7 us.
//
// ORDERED (with `done`): the sweeps of one chunk run in order.  Tickets of
// the same chunk in consecutive sweeps are nchunks apart, so when chunks are
// few against warps one warp could still be updating chunk c in sweep s while
// another takes it in sweep s + 1, and the older update's Dinv could land
// after the newer U_ii.  Then a warp first waits (at most `limit` polls; a
// timeout is counted in *err and the warp stops) until done[c] records s
// completed sweeps, and publishes s + 1 after its writes.  A wait points only
// to a smaller ticket, held by a resident warp, so every wait ends.  No bulk
// copy is in flight in this kernel, so a warp that gives up can simply return.
constexpr int WARP_CHUNK = 128;   // default work blocks per ticket (abilu_factors_set_build_chunk)

// Sub-chunk size of a ticket of `wchunk` blocks (a multiple of 32) and the
// number of tickets per sweep: the kernel and its launcher share this.
__host__ __device__ __forceinline__ int build_sub(int wchunk) { return wchunk % 64 == 0 ? 64 : 32; }
__host__ __device__ __forceinline__ long long build_tickets(int nwork, int wchunk) {
    const int sub = build_sub(wchunk);
    const long long nsub = (nwork + sub - 1) / sub;
    const int per = wchunk / sub;
    return (nsub + per - 1) / per;
}

template <typename T, bool ORDERED, int SUB>
__global__ void __launch_bounds__(BUILD_THREADS, 5)   // 48 registers: measured fastest (4, 6 slower)
k_build_blocks_async(PatternView P, const float *__restrict__ A32, T *L, T *U, T *D, T *Udiag,
                     int nsweeps, int max_warps, unsigned long long *nsing,
                     unsigned long long *ticket, unsigned long long *err, int *done,
                     unsigned long long limit, int wchunk) {
    pdl_wait();
    pdl_trigger();
    __shared__ __align__(16) float sh_q[WORK_PER_CTA * QUAD_SCRATCH];
    // at most one warp per chunk: more would sweep the same blocks at once
    if (blockIdx.x * (BUILD_THREADS / 32) + (threadIdx.x >> 5) >= max_warps) return;
    const long long nchunks = build_tickets(P.nwork, wchunk);
    const long long total = nchunks * nsweeps;
    const int stride = (int)nchunks * SUB;   // blocks between a ticket's sub-chunks
    const int lane = threadIdx.x & 31;
    float *myq = sh_q + (threadIdx.x >> 2) * QUAD_SCRATCH;
    for (;;) {
        unsigned long long tk = 0;
        if (lane == 0) tk = atomicAdd(ticket, 1ull);
        const long long t = (long long)__shfl_sync(0xffffffffu, tk, 0);
        if (t >= total) break;
        const int sweep = (int)(t / nchunks), chunk = (int)(t % nchunks);
        const bool last = sweep == nsweeps - 1;
        if constexpr (ORDERED) {  // wait for this chunk's previous sweep
            int ok = 1;
            if (lane == 0) {
                unsigned long long it = 0;
                bool ready;
                while (!(ready = *reinterpret_cast<volatile int *>(done + chunk) >= sweep) && ++it < limit) {}
                ok = ready;
                if (!ok) atomicAdd(err, 1ull);
                __threadfence();
            }
            if (!__shfl_sync(0xffffffffu, ok, 0)) return;
        }
        // step k: sub-chunk chunk + (k / steps) nchunks, its 8 blocks k mod
        // steps (32-bit: block indices stay below (nsub + wchunk / 32) * 64,
        // and nwork <= nnzb < 2^31 - 2^16)
        constexpr int SSH = SUB == 64 ? 3 : 2;   // log2(steps per sub-chunk)
        const int base = chunk * SUB + (lane >> 2);
#pragma unroll 1
        for (int k = 0; k < wchunk / 8; k++) {
            const int w = base + (k >> SSH) * stride + ((k & ((1 << SSH) - 1)) << 3);
            if (w < P.nwork)
                build_block<T, true>(P, w, A32, L, U, D, L, U, D, last ? Udiag : nullptr, myq, nsing);
        }
        if constexpr (ORDERED) __threadfence();   // this lane's factor writes, before the flag
        __syncwarp();
        if (ORDERED && lane == 0) *reinterpret_cast<volatile int *>(done + chunk) = sweep + 1;
    }
}

template <typename T, typename AT>
__global__ void __launch_bounds__(BUILD_THREADS)
k_build_sync(PatternView P, const AT *__restrict__ A, const T *__restrict__ Lin,
             const T *__restrict__ Uin, const T *__restrict__ Din, T *__restrict__ Lout,
             T *__restrict__ Uout, T *__restrict__ Dout, T *__restrict__ Udiag,
             unsigned long long *nsing) {
    pdl_wait();
    pdl_trigger();
    __shared__ double sh_u[BuildShared<T>::D];
    __shared__ double sh_d[BuildShared<T>::D];
    __shared__ __align__(16) float sh_q[BuildShared<T>::F];
    const int row0 = blockIdx.x * BUILD_ROWS;
    const int i = row0 + (threadIdx.x >> 2);
    typename BuildArith<T>::C u[4] = {0, 0, 0, 0};
    if (i < P.n) build_row_products<T, false>(P, i, A, Lin, Uin, Din, Lout, Uout, u);
    build_finish_rows<T, false>(row0, P.n, u, Dout, Udiag, sh_u, sh_d, sh_q, nsing);
}

// Persistent in-place kernel: tickets t = 0 .. nsweeps*nchunks-1 taken in
// order from ctr; ticket t is chunk (t mod nchunks) in sweep (t / nchunks).
template <typename T, typename AT>
__global__ void __launch_bounds__(BUILD_THREADS)
k_build_async(PatternView P, const AT *__restrict__ A, T *L, T *U, T *D, T *Udiag,
              int nsweeps, unsigned long long *nsing, unsigned long long *ticket) {
    pdl_wait();
    pdl_trigger();
    __shared__ double sh_u[BuildShared<T>::D];
    __shared__ double sh_d[BuildShared<T>::D];
    __shared__ __align__(16) float sh_q[BuildShared<T>::F];
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
        typename BuildArith<T>::C u[4] = {0, 0, 0, 0};
        if (i < P.n) build_row_products<T, true>(P, i, A, L, U, D, L, U, u);
        build_finish_rows<T, true>(row0, P.n, u, D, sweep == nsweeps - 1 ? Udiag : nullptr,
                                   sh_u, sh_d, sh_q, nsing);
    }
}

// Once per build, one pass over the FP64 A:
//  * the constant blocks (U_ij, i < j, with no product pair: U_ij = A_ij in
//    every sweep) go into U[cur] and, for synchronous builds, U[other];
//  * for FP32/BF16 factors every other block is stored as FP32 in A32, which
//    the sweeps read instead of A (they compute in FP32; same values);
//  * from A (init_from_a): X^0 = A, i.e. L^0 = strictly lower blocks of A
//    (unscaled), U^0 = upper blocks, Dinv^0 = inv(A_ii), U_ii stored (Sec. 6
//    setup: the initial guess of the factorisation is the matrix itself).
template <typename T>
__global__ void __launch_bounds__(BUILD_THREADS, sizeof(T) == 8 ? 3 : 4)
k_build_prepare(PatternView P, const double *__restrict__ A, float *__restrict__ A32,
                T *__restrict__ L, T *__restrict__ U, T *__restrict__ Uother, T *__restrict__ D,
                T *__restrict__ Udiag, int init_all, const int *__restrict__ chunk_init,
                unsigned long long *nsing) {
    pdl_wait();
    pdl_trigger();
    // a CTA's 64 rows are one chunk of a server's arena (BUILD_ROWS = 64)
    const int init_from_a = chunk_init ? chunk_init[blockIdx.x] : init_all;
    __shared__ double sh_u[BuildShared<T>::D];
    __shared__ double sh_d[BuildShared<T>::D];
    __shared__ __align__(16) float sh_q[BuildShared<T>::F];
    const int row0 = blockIdx.x * BUILD_ROWS;
    const int i = row0 + (threadIdx.x >> 2), q = threadIdx.x & 3;
    typename BuildArith<T>::C ud[4] = {0, 0, 0, 0};
    if (i < P.n) {
        const int p0 = P.rowptr[i], p1 = P.rowptr[i + 1], dp = P.diagpos[i];
        const int lb = P.lrow[i], ub = P.urow[i];
        // four blocks of the row at a time, every load issued before any store
        for (int pb = p0; pb < p1; pb += 4) {
            double a[4][4];
            int wp[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                if (pb + k < p1) {
                    ld_row(A + (size_t)(pb + k) * BB + q * BS, a[k]);
                    wp[k] = P.wpos[pb + k];
                }
            }
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const int p = pb + k;
                if (p >= p1) break;
                if (p > dp && wp[k] < 0) {  // not a work item: a constant U block
                    st_row(U + (size_t)(ub + p - dp - 1) * BB + q * BS, a[k]);
                    if (Uother) st_row(Uother + (size_t)(ub + p - dp - 1) * BB + q * BS, a[k]);
                    continue;
                }
                if (A32) st_row(A32 + (size_t)wp[k] * BB + q * BS, a[k]);  // work order
                if (!init_from_a) continue;
                if (p < dp) st_row(L + (size_t)(lb + p - p0) * BB + q * BS, a[k]);
                else if (p > dp) st_row(U + (size_t)(ub + p - dp - 1) * BB + q * BS, a[k]);
                else {
#pragma unroll
                    for (int c = 0; c < 4; c++) {
                        if constexpr (sizeof(T) == 8) ud[c] = a[k][c];
                        else ud[c] = to_f32(a[k][c]);
                    }
                }
            }
        }
    }
    if (init_from_a) build_finish_rows<T, false>(row0, P.n, ud, D, Udiag, sh_u, sh_d, sh_q, nsing);
}

// Us_ij = Dinv_i U_ij for every strictly upper block (FP32 factors), once per
// build: the upper sweeps then read x_i = Dinv_i y_i - sum_j Us_ij x_j
// (the same iteration as x_i = Dinv_i (y_i - sum_j U_ij x_j), Sec. 4.1) and
// no longer re-read Dinv_i in every sweep.  A quad per block row, thread q
// forms row q: sum_k Dinv_i[q][k] U_ij[k][:] with U's rows from the quad.
template <typename T>
__global__ void __launch_bounds__(BUILD_THREADS)
k_scale_upper(PatternView P, const T *__restrict__ U, const T *__restrict__ D, T *__restrict__ Us) {
    pdl_wait();
    pdl_trigger();
    const int i = blockIdx.x * BUILD_ROWS + (threadIdx.x >> 2), q = threadIdx.x & 3;
    if (i >= P.n) return;
    float d[4];
    ld_row(D + (size_t)i * BB + q * BS, d);
    for (int l = P.urow[i]; l < P.urow[i + 1]; l++) {
        float u[4], o[4] = {0.f, 0.f, 0.f, 0.f};
        ld_row(U + (size_t)l * BB + q * BS, u);
#pragma unroll
        for (int k = 0; k < 4; k++)
#pragma unroll
            for (int c = 0; c < 4; c++) o[c] += d[k] * qshfl(u[c], k);
        st_row(Us + (size_t)l * BB + q * BS, o);
    }
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
static abilu_status block_sweeps_t(abilu_factors f, const float *A32, int nsweeps,
                                   abilu_mode mode, cudaStream_t st) {
    const PatternView &P = f->p->v;
    const int grid = (P.nwork + WORK_PER_CTA - 1) / WORK_PER_CTA;
    T **L = reinterpret_cast<T **>(f->L), **U = reinterpret_cast<T **>(f->U);
    T **D = reinterpret_cast<T **>(f->D);
    T *Ud = reinterpret_cast<T *>(f->Udiag);
    if (grid == 0) return ABILU_OK;
    if (mode == ABILU_SYNC) {
        for (int s = 0; s < nsweeps; s++) {
            const int c = f->cur, o = 1 - f->cur;
            launch_pdl(k_build_blocks_sync<T>, grid, BUILD_THREADS, 0, st,
                P, A32, L[c], U[c], D[c], L[o], U[o], D[o], s == nsweeps - 1 ? Ud : nullptr, f->ctr);
            ABILU_LAUNCH_CHECK("k_build_blocks_sync");
            f->cur = o;
        }
    } else {
        static std::atomic<int> per_sm_cache{-1};
        int dev = 0, sms = 0, per_sm = per_sm_cache.load(std::memory_order_relaxed);
        cudaGetDevice(&dev);
        if (per_sm < 0) {   // the ordered variant is held to the same occupancy
            ABILU_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &per_sm, k_build_blocks_async<T, false, 64>, BUILD_THREADS, 0));
            per_sm_cache.store(per_sm, std::memory_order_relaxed);
        }
        ABILU_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const int wc = f->build_chunk ? f->build_chunk : WARP_CHUNK;
        const int wchunks = (int)build_tickets(P.nwork, wc);
        int warps = per_sm * sms * (BUILD_THREADS / 32);
        if (warps > wchunks) warps = wchunks;
        if (warps < 1) warps = 1;
        const int ctas = (warps + BUILD_THREADS / 32 - 1) / (BUILD_THREADS / 32);
        ABILU_CUDA(cudaMemsetAsync(f->ctr + 1, 0, sizeof(unsigned long long), st));
        // fewer than 4 chunks per warp: keep each chunk's sweeps in order (see
        // the kernel); with more, an overlap needs one warp stalled for the
        // time the others take to process several chunks each
        int *done = nullptr;
        if ((long long)wchunks < 4LL * warps) {
            done = f->chunk_done;
            // failure injection (tests of the bounded wait): every flag at -1,
            // one sweep behind, which no warp ever publishes, so the first
            // wait of every chunk runs out after the spin limit
            const int fill = f->stall_flags ? 0xff : 0;
            f->stall_flags = 0;
            ABILU_CUDA(cudaMemsetAsync(done, fill, sizeof(int) * (size_t)wchunks, st));
        }
        const int c = f->cur;
        const unsigned long long lim = spin_limit_or_default(f->spin_limit);
        auto kern = done ? (build_sub(wc) == 64 ? k_build_blocks_async<T, true, 64>
                                                : k_build_blocks_async<T, true, 32>)
                         : (build_sub(wc) == 64 ? k_build_blocks_async<T, false, 64>
                                                : k_build_blocks_async<T, false, 32>);
        launch_pdl(kern, ctas, BUILD_THREADS, 0, st,
            P, A32, L[c], U[c], D[c], Ud, nsweeps, warps, f->ctr, f->ctr + 1, f->ctr + 4, done,
            lim, wc);
        ABILU_LAUNCH_CHECK("k_build_blocks_async");
    }
    return ABILU_OK;
}

template <typename T, typename AT>
static abilu_status sweeps_t(abilu_factors f, const AT *Asrc, int nsweeps, abilu_mode mode,
                             cudaStream_t st) {
    const PatternView &P = f->p->v;
    const int grid = (P.n + BUILD_ROWS - 1) / BUILD_ROWS;
    T **L = reinterpret_cast<T **>(f->L), **U = reinterpret_cast<T **>(f->U);
    T **D = reinterpret_cast<T **>(f->D);
    T *Ud = reinterpret_cast<T *>(f->Udiag);
    if (mode == ABILU_SYNC) {
        for (int s = 0; s < nsweeps; s++) {
            const int c = f->cur, o = 1 - f->cur;
            launch_pdl(k_build_sync<T, AT>, grid, BUILD_THREADS, 0, st,
                P, Asrc, L[c], U[c], D[c], L[o], U[o], D[o], s == nsweeps - 1 ? Ud : nullptr,
                f->ctr);
            ABILU_LAUNCH_CHECK("k_build_sync");
            f->cur = o;
        }
    } else {
        static std::atomic<int> per_sm_cache{-1};
        int dev = 0, sms = 0, per_sm = per_sm_cache.load(std::memory_order_relaxed);
        cudaGetDevice(&dev);
        if (per_sm < 0) {
            ABILU_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_build_async<T, AT>,
                                                                     BUILD_THREADS, 0));
            per_sm_cache.store(per_sm, std::memory_order_relaxed);
        }
        ABILU_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        // at most one CTA per chunk: more would sweep the same rows at once
        int ctas = per_sm * sms;
        if (ctas > grid) ctas = grid;
        if (ctas < 1) ctas = 1;
        ABILU_CUDA(cudaMemsetAsync(f->ctr + 1, 0, sizeof(unsigned long long), st));
        const int c = f->cur;
        launch_pdl(k_build_async<T, AT>, ctas, BUILD_THREADS, 0, st, P, Asrc, L[c], U[c], D[c], Ud,
            nsweeps, f->ctr, f->ctr + 1);
        ABILU_LAUNCH_CHECK("k_build_async");
    }
    return ABILU_OK;
}

// With timing enabled on the handle, a build records tev[0] before its sweep
// kernels and tev[1] after them on its stream (abilu_factors_sweep_time).
static abilu_status timing_mark(abilu_factors f, int k, cudaStream_t st) {
    if (!f->timing) return ABILU_OK;
    if (k == 0) f->timed = 0;   // a build that fails between the marks leaves no time
    ABILU_CUDA(cudaEventRecord(static_cast<cudaEvent_t>(f->tev[k]), st));
    if (k == 1) f->timed = 1;
    return ABILU_OK;
}

template <typename T>
static abilu_status build_t(abilu_factors f, const double *A, int nsweeps, abilu_mode mode,
                            abilu_init init, cudaStream_t st) {
    const PatternView &P = f->p->v;
    const int grid = (P.n + BUILD_ROWS - 1) / BUILD_ROWS;
    T **L = reinterpret_cast<T **>(f->L), **U = reinterpret_cast<T **>(f->U);
    T **D = reinterpret_cast<T **>(f->D);
    T *Ud = reinterpret_cast<T *>(f->Udiag);
    constexpr bool narrow = sizeof(T) < 8;
    float *A32 = narrow ? reinterpret_cast<float *>(f->A32) : nullptr;
    const int c = f->cur;
    // U_ii of the initial guess only when no sweep follows: the last sweep
    // stores the build's U_ii (33.5 MB fewer writes at 512x512)
    launch_pdl(k_build_prepare<T>, grid, BUILD_THREADS, 0, st,
        P, A, A32, L[c], U[c], mode == ABILU_SYNC ? U[1 - c] : nullptr, D[c], nsweeps > 0 ? nullptr : Ud,
        init == ABILU_INIT_FROM_A ? 1 : 0, f->chunk_init, f->ctr);
    ABILU_LAUNCH_CHECK("k_build_prepare");
    if constexpr (narrow) {
        if (nsweeps > 0) {
            abilu_status s = timing_mark(f, 0, st);
            if (s == ABILU_OK) s = block_sweeps_t<T>(f, A32, nsweeps, mode, st);
            if (s == ABILU_OK) s = timing_mark(f, 1, st);
            if (s != ABILU_OK) return s;
        }
        const int cf = f->cur;
        if (f->Us && P.nu > 0) {
            launch_pdl(k_scale_upper<T>, grid, BUILD_THREADS, 0, st,
                P, reinterpret_cast<const T *>(f->U[cf]), reinterpret_cast<const T *>(f->D[cf]),
                reinterpret_cast<T *>(f->Us));
            ABILU_LAUNCH_CHECK("k_scale_upper");
        }
        return ABILU_OK;
    } else {
        if (nsweeps == 0) return ABILU_OK;
        abilu_status s = timing_mark(f, 0, st);
        if (s == ABILU_OK) s = sweeps_t<T, double>(f, A, nsweeps, mode, st);
        if (s == ABILU_OK) s = timing_mark(f, 1, st);
        return s;
    }
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

abilu_status scalar_build(abilu_factors f, const double *A, int nsweeps, abilu_mode mode,
                          abilu_init init, cudaStream_t st);
abilu_status scalar_export(abilu_factors f, double *X, cudaStream_t st);

// Us = Dinv U for FP32 factors whose L, U and Dinv were written directly
// (imported factors), as a build forms it at its end
abilu_status form_scaled_upper(abilu_factors f, cudaStream_t st) {
    const PatternView &P = f->p->v;
    if (f->dtype != ABILU_F32 || !f->Us || P.nu == 0) return ABILU_OK;
    const int cf = f->cur;
    launch_pdl(k_scale_upper<float>, (P.n + BUILD_ROWS - 1) / BUILD_ROWS, BUILD_THREADS, 0, st,
        P, reinterpret_cast<const float *>(f->U[cf]), reinterpret_cast<const float *>(f->D[cf]),
        reinterpret_cast<float *>(f->Us));
    ABILU_LAUNCH_CHECK("k_scale_upper");
    return ABILU_OK;
}

abilu_status build_dispatch(abilu_factors f, const double *A, int nsweeps, abilu_mode mode,
                            abilu_init init, cudaStream_t st) {
    if (f->scalar) return scalar_build(f, A, nsweeps, mode, init, st);
    switch (f->dtype) {
    case ABILU_F64: return build_t<double>(f, A, nsweeps, mode, init, st);
    case ABILU_F32: return build_t<float>(f, A, nsweeps, mode, init, st);
    case ABILU_BF16: return build_t<__nv_bfloat16>(f, A, nsweeps, mode, init, st);
    }
    return fail(ABILU_EINVAL, "build: bad dtype");
}

abilu_status export_dispatch(abilu_factors f, double *X, double *Dinv, cudaStream_t st) {
    if (f->scalar) return scalar_export(f, X, st);   // no Dinv: scalar pivots
    switch (f->dtype) {
    case ABILU_F64: return export_t<double>(f, X, Dinv, st);
    case ABILU_F32: return export_t<float>(f, X, Dinv, st);
    case ABILU_BF16: return export_t<__nv_bfloat16>(f, X, Dinv, st);
    }
    return fail(ABILU_EINVAL, "export: bad dtype");
}

}  // namespace abilu
