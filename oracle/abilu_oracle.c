/*
 * CPU oracle for the asynchronous block ILU(0) preconditioner with FGMRES
 * (Kashi & Nadarajah, "An asynchronous incomplete block LU preconditioner for
 * computational fluid dynamics on unstructured grids").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, single-threaded FP64
 * statement of what the method computes.  It shares no code with the CUDA
 * library; only the test suite, the smoke check and the benchmark's CPU-baseline
 * leg load it.  The product path never calls it.
 *
 * Storage: block CSR with b = 4 (Sec. 2: all d+2 = 4 unknowns of a cell
 * contiguous), rowptr/colind int32, colind sorted inside each row, the diagonal
 * block present in every row, each 4x4 block row-major (16 doubles).
 * The factors X are held in a copy of A's pattern: positions with column < row
 * hold L_ij (L_ii = I is implicit), positions with column >= row hold U_ij.
 * Dinv holds one 4x4 block per row, the inverse of U_ii.
 *
 * Every sum runs in ascending column order and accumulates in a local FP64
 * variable that is written once (Sec. 4.2 notes that accumulating a partial sum
 * in place slows the asynchronous iteration; a local accumulator is the form the
 * paper uses).  Build with -O2 -ffp-contract=off so no FMA contraction changes
 * the rounding between machines.
 *
 * Parity status: every function below is pinned by tests against an
 * independent statement (dense numpy elimination, numpy.linalg, scipy, closed
 * forms, the paper's theorems); see tests/test_oracle_*.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define BS 4
#define BB 16

typedef int32_t idx_t;

/* ---------------------------------------------------------------- 4x4 blocks */

/* S -= X * Y  (4x4 row-major) */
static void blk_sub_mul(double *S, const double *X, const double *Y)
{
    for (int r = 0; r < BS; r++)
        for (int c = 0; c < BS; c++) {
            double acc = 0.0;
            for (int k = 0; k < BS; k++)
                acc += X[r * BS + k] * Y[k * BS + c];
            S[r * BS + c] -= acc;
        }
}

/* out = X * Y */
static void blk_mul(double *out, const double *X, const double *Y)
{
    for (int r = 0; r < BS; r++)
        for (int c = 0; c < BS; c++) {
            double acc = 0.0;
            for (int k = 0; k < BS; k++)
                acc += X[r * BS + k] * Y[k * BS + c];
            out[r * BS + c] = acc;
        }
}

/* s -= X * v  (4x4 times 4-vector) */
static void blk_sub_matvec(double *s, const double *X, const double *v)
{
    for (int r = 0; r < BS; r++) {
        double acc = 0.0;
        for (int k = 0; k < BS; k++)
            acc += X[r * BS + k] * v[k];
        s[r] -= acc;
    }
}

/* out = X * v */
static void blk_matvec(double *out, const double *X, const double *v)
{
    for (int r = 0; r < BS; r++) {
        double acc = 0.0;
        for (int k = 0; k < BS; k++)
            acc += X[r * BS + k] * v[k];
        out[r] = acc;
    }
}

/*
 * Exact inverse of a 4x4 block by Gauss-Jordan elimination with partial
 * pivoting (the paper inverts diagonal blocks exactly, Sec. 4.1 / Eq. (bilu)).
 * Pivot: the first row of largest |entry| in the column.  A zero or non-finite
 * pivot marks the block singular; then, following the "modified iteration" of
 * Sec. 4.2 (a singular diagonal block is replaced by an arbitrary non-singular
 * one), the block is replaced by the identity and out = I.
 * Returns 1 if the block was singular, else 0.
 */
int orc_inv4(const double *a, double *out)
{
    double m[BS][2 * BS];
    for (int r = 0; r < BS; r++)
        for (int c = 0; c < BS; c++) {
            m[r][c] = a[r * BS + c];
            m[r][BS + c] = (r == c) ? 1.0 : 0.0;
        }
    for (int c = 0; c < BS; c++) {
        int p = c;
        for (int r = c + 1; r < BS; r++)
            if (fabs(m[r][c]) > fabs(m[p][c]))
                p = r;
        double piv = m[p][c];
        if (piv == 0.0 || !isfinite(piv)) {
            for (int r = 0; r < BS; r++)
                for (int k = 0; k < BS; k++)
                    out[r * BS + k] = (r == k) ? 1.0 : 0.0;
            return 1;
        }
        if (p != c)
            for (int k = 0; k < 2 * BS; k++) {
                double t = m[p][k];
                m[p][k] = m[c][k];
                m[c][k] = t;
            }
        for (int k = 0; k < 2 * BS; k++)
            m[c][k] = m[c][k] / piv;
        for (int r = 0; r < BS; r++) {
            if (r == c)
                continue;
            double f = m[r][c];
            for (int k = 0; k < 2 * BS; k++)
                m[r][k] = m[r][k] - f * m[c][k];
        }
    }
    for (int r = 0; r < BS; r++)
        for (int c = 0; c < BS; c++)
            out[r * BS + c] = m[r][BS + c];
    return 0;
}

/* Position of block (i, j) in the pattern, or -1 (linear search in row i). */
static long find_block(const idx_t *rowptr, const idx_t *colind, idx_t i, idx_t j)
{
    for (long p = rowptr[i]; p < rowptr[i + 1]; p++)
        if (colind[p] == j)
            return p;
    return -1;
}

static long diag_pos(const idx_t *rowptr, const idx_t *colind, idx_t i)
{
    return find_block(rowptr, colind, i, i);
}

/*
 * S = A_ij - sum_{k < min(i,j), (i,k),(k,j) in S_B} Xsrc_ik Xsrc_kj, the common
 * part of both lines of Eq. (bilu) / H_ij.  k runs in ascending order over the
 * blocks of row i.
 */
static void bilu_residual_block(idx_t i, idx_t j, long p, const idx_t *rowptr,
                                const idx_t *colind, const double *A,
                                const double *Xsrc, double *S)
{
    memcpy(S, A + p * BB, sizeof(double) * BB);
    idx_t kmax = i < j ? i : j;
    for (long q = rowptr[i]; q < rowptr[i + 1]; q++) {
        idx_t k = colind[q];
        if (k >= kmax)
            break;
        long r = find_block(rowptr, colind, k, j);
        if (r < 0)
            continue;
        blk_sub_mul(S, Xsrc + q * BB, Xsrc + r * BB);
    }
}

/*
 * Sequential block ILU(0): Eq. (bilu) evaluated in the block Gaussian
 * elimination (row-major) ordering, each block from the values already
 * computed.  This is the unique fixed point of h (Sec. 4.2, uniqueness
 * theorem) and what one thread running one sweep of the asynchronous
 * iteration produces (Sec. 3.3 / Sec. 6 setup).
 * X (nnzb*16) and Dinv (n*16) are outputs.  Returns the number of singular
 * diagonal blocks that were replaced.
 */
int orc_bilu0_seq(idx_t n, const idx_t *rowptr, const idx_t *colind,
                  const double *A, double *X, double *Dinv)
{
    int nsing = 0;
    double S[BB];
    for (idx_t i = 0; i < n; i++) {
        for (long p = rowptr[i]; p < rowptr[i + 1]; p++) {
            idx_t j = colind[p];
            bilu_residual_block(i, j, p, rowptr, colind, A, X, S);
            if (j < i) {
                blk_mul(X + p * BB, S, Dinv + (long)j * BB);
            } else {
                memcpy(X + p * BB, S, sizeof S);
                if (j == i)
                    nsing += orc_inv4(S, Dinv + (long)i * BB);
            }
        }
    }
    return nsing;
}

/*
 * Initial guess of the factorisation (Sec. 6 setup: "the Jacobian itself"):
 * X^0 = A on S_B, L^0 unscaled, and Dinv^0 = inv(A_ii).
 */
int orc_bilu_init(idx_t n, const idx_t *rowptr, const idx_t *colind,
                  const double *A, double *X, double *Dinv)
{
    long nnzb = rowptr[n];
    int nsing = 0;
    memcpy(X, A, sizeof(double) * BB * nnzb);
    for (idx_t i = 0; i < n; i++) {
        long d = diag_pos(rowptr, colind, i);
        nsing += orc_inv4(A + d * BB, Dinv + (long)i * BB);
    }
    return nsing;
}

/*
 * One synchronous (Jacobi-type) sweep x^{n+1} = h(x^n), Eq. (seq_blockilu_fp)
 * with H_ij of Eq. (blockH): every block from the previous iterate; the L
 * update multiplies by inv(U_jj^n) = Dinv_in[j].  After U_ii^{n+1} is formed
 * its inverse becomes Dinv_out[i].  Returns the number of singular blocks.
 */
int orc_bilu_sync_sweep(idx_t n, const idx_t *rowptr, const idx_t *colind,
                        const double *A, const double *Xin, const double *Dinv_in,
                        double *Xout, double *Dinv_out)
{
    int nsing = 0;
    double S[BB];
    for (idx_t i = 0; i < n; i++) {
        for (long p = rowptr[i]; p < rowptr[i + 1]; p++) {
            idx_t j = colind[p];
            bilu_residual_block(i, j, p, rowptr, colind, A, Xin, S);
            if (j < i) {
                blk_mul(Xout + p * BB, S, Dinv_in + (long)j * BB);
            } else {
                memcpy(Xout + p * BB, S, sizeof S);
                if (j == i)
                    nsing += orc_inv4(S, Dinv_out + (long)i * BB);
            }
        }
    }
    return nsing;
}

/*
 * Deterministic emulation of the asynchronous in-place sweep (Algorithm 4 with
 * blocks): the rows are cut into chunks of `chunk` consecutive rows; the chunks
 * are visited in the order chunk_order[0..nchunks-1]; each chunk's rows are
 * processed in ascending order, blocks of a row in ascending column order,
 * every read taking the latest value in memory (in place).  This is what one
 * thread taking chunks in that order does.  Returns singular count.
 */
int orc_bilu_chunked_sweep(idx_t n, const idx_t *rowptr, const idx_t *colind,
                           const double *A, double *X, double *Dinv,
                           idx_t chunk, const idx_t *chunk_order, idx_t nchunks)
{
    int nsing = 0;
    double S[BB];
    for (idx_t c = 0; c < nchunks; c++) {
        idx_t i0 = chunk_order[c] * chunk;
        idx_t i1 = i0 + chunk < n ? i0 + chunk : n;
        for (idx_t i = i0; i < i1; i++) {
            for (long p = rowptr[i]; p < rowptr[i + 1]; p++) {
                idx_t j = colind[p];
                bilu_residual_block(i, j, p, rowptr, colind, A, X, S);
                if (j < i) {
                    blk_mul(X + p * BB, S, Dinv + (long)j * BB);
                } else {
                    memcpy(X + p * BB, S, sizeof S);
                    if (j == i)
                        nsing += orc_inv4(S, Dinv + (long)i * BB);
                }
            }
        }
    }
    return nsing;
}

/* ------------------------------------------------------- triangular apply */

/*
 * One synchronous (Jacobi) sweep of the lower block triangular solve L y = r
 * (Algorithm 5 with every read from the previous iterate; L_ii = I):
 *   y_out_i = r_i - sum_{j<i} L_ij y_in_j.
 */
void orc_lower_sweep(idx_t n, const idx_t *rowptr, const idx_t *colind,
                     const double *X, const double *r, const double *y_in,
                     double *y_out)
{
    for (idx_t i = 0; i < n; i++) {
        double s[BS];
        memcpy(s, r + (long)i * BS, sizeof s);
        for (long p = rowptr[i]; p < rowptr[i + 1]; p++) {
            idx_t j = colind[p];
            if (j >= i)
                break;
            blk_sub_matvec(s, X + p * BB, y_in + (long)j * BS);
        }
        memcpy(y_out + (long)i * BS, s, sizeof s);
    }
}

/*
 * One synchronous (Jacobi) sweep of the upper block triangular solve U x = y
 * (the backward analogue of Algorithm 5):
 *   x_out_i = U_ii^{-1} (y_i - sum_{j>i} U_ij x_in_j).
 */
void orc_upper_sweep(idx_t n, const idx_t *rowptr, const idx_t *colind,
                     const double *X, const double *Dinv, const double *y,
                     const double *x_in, double *x_out)
{
    for (idx_t i = 0; i < n; i++) {
        double s[BS];
        memcpy(s, y + (long)i * BS, sizeof s);
        for (long p = rowptr[i]; p < rowptr[i + 1]; p++) {
            idx_t j = colind[p];
            if (j <= i)
                continue;
            blk_sub_matvec(s, X + p * BB, x_in + (long)j * BS);
        }
        blk_matvec(x_out + (long)i * BS, Dinv + (long)i * BB, s);
    }
}

/* Exact forward substitution L y = r with unit diagonal blocks (Algorithm 1). */
void orc_lower_solve(idx_t n, const idx_t *rowptr, const idx_t *colind,
                     const double *X, const double *r, double *y)
{
    for (idx_t i = 0; i < n; i++) {
        double s[BS];
        memcpy(s, r + (long)i * BS, sizeof s);
        for (long p = rowptr[i]; p < rowptr[i + 1]; p++) {
            idx_t j = colind[p];
            if (j >= i)
                break;
            blk_sub_matvec(s, X + p * BB, y + (long)j * BS);
        }
        memcpy(y + (long)i * BS, s, sizeof s);
    }
}

/* Exact backward substitution U x = y, rows in descending order. */
void orc_upper_solve(idx_t n, const idx_t *rowptr, const idx_t *colind,
                     const double *X, const double *Dinv, const double *y, double *x)
{
    for (idx_t i = n - 1; i >= 0; i--) {
        double s[BS];
        memcpy(s, y + (long)i * BS, sizeof s);
        for (long p = rowptr[i]; p < rowptr[i + 1]; p++) {
            idx_t j = colind[p];
            if (j <= i)
                continue;
            blk_sub_matvec(s, X + p * BB, x + (long)j * BS);
        }
        blk_matvec(x + (long)i * BS, Dinv + (long)i * BB, s);
    }
}

/*
 * Preconditioner application z = (LU)^{-1} r, approximately: n_lower Jacobi
 * sweeps on L y = r from y = 0, then n_upper Jacobi sweeps on U z = y from
 * z = 0 (zero initial guesses every application, Sec. 6 setup).  A negative
 * sweep count means the exact substitution.  work: 2*n*4 doubles.
 */
void orc_apply(idx_t n, const idx_t *rowptr, const idx_t *colind,
               const double *X, const double *Dinv, const double *r, double *z,
               int n_lower, int n_upper, double *work)
{
    long nv = (long)n * BS;
    double *y = work, *t = work + nv;
    if (n_lower < 0) {
        orc_lower_solve(n, rowptr, colind, X, r, y);
    } else {
        memset(y, 0, sizeof(double) * nv);
        for (int s = 0; s < n_lower; s++) {
            orc_lower_sweep(n, rowptr, colind, X, r, y, t);
            memcpy(y, t, sizeof(double) * nv);
        }
    }
    if (n_upper < 0) {
        orc_upper_solve(n, rowptr, colind, X, Dinv, y, z);
    } else {
        memset(z, 0, sizeof(double) * nv);
        for (int s = 0; s < n_upper; s++) {
            orc_upper_sweep(n, rowptr, colind, X, Dinv, y, z, t);
            memcpy(z, t, sizeof(double) * nv);
        }
    }
}

/* ------------------------------------------------------------------ SpMV */

/* y = A x, block rows independent, j ascending within a row. */
void orc_spmv(idx_t n, const idx_t *rowptr, const idx_t *colind,
              const double *A, const double *x, double *y)
{
    for (idx_t i = 0; i < n; i++) {
        double s[BS] = {0.0, 0.0, 0.0, 0.0};
        for (long p = rowptr[i]; p < rowptr[i + 1]; p++) {
            const double *a = A + p * BB;
            const double *xj = x + (long)colind[p] * BS;
            for (int r = 0; r < BS; r++) {
                double acc = 0.0;
                for (int k = 0; k < BS; k++)
                    acc += a[r * BS + k] * xj[k];
                s[r] += acc;
            }
        }
        memcpy(y + (long)i * BS, s, sizeof s);
    }
}

/* --------------------------------------------------------------- FGMRES */

static double dot(long nv, const double *a, const double *b)
{
    double s = 0.0;
    for (long k = 0; k < nv; k++)
        s += a[k] * b[k];
    return s;
}

typedef struct {
    int iters;             /* Arnoldi steps over all restarts */
    int restarts;          /* completed restart cycles */
    int converged;         /* 1 if the true relative residual <= rtol */
    double rel_resid_est;  /* last Givens estimate |g_{j+1}| / ||b|| */
    double rel_resid_true; /* ||b - A x|| / ||b|| at exit */
} orc_fgmres_result;

/*
 * Right-preconditioned flexible GMRES(m) (Saad's FGMRES, used by the paper
 * through PETSc, Sec. 2 / Sec. 6 setup), with modified Gram-Schmidt and Givens
 * rotations.  orc_fgmres_pc takes the preconditioner as a callback; in
 * orc_fgmres it is the block ILU given by (X, Dinv), applied with n_lower /
 * n_upper Jacobi sweeps (negative: exact), or with Dinv == NULL the scalar ILU
 * held in X (orc_silu_apply).  x holds x0 on entry
 * and the solution on exit.  Stops when the Givens residual estimate drops to
 * rtol*||b||, confirmed at the end of the cycle by the explicit residual; an
 * unconfirmed estimate restarts.  Stops at max_iters Arnoldi steps.
 * hist (may be NULL, max_iters+1 entries) receives |g_{j+1}| / ||b|| per step.
 */
void orc_silu_apply(idx_t n, const idx_t *rowptr, const idx_t *colind, const double *X,
                    const double *r, double *z, int n_lower, int n_upper, double *work);

/* A right preconditioner z = M^{-1} r as a callback (FGMRES allows it to vary
 * from one application to the next). */
typedef void (*orc_precond)(void *ctx, const double *r, double *z);

int orc_fgmres_pc(idx_t n, const idx_t *rowptr, const idx_t *colind, const double *A,
                  orc_precond pc, void *ctx, const double *b, double *x, int m,
                  int max_iters, double rtol, orc_fgmres_result *res, double *hist)
{
    long nv = (long)n * BS;
    double *V = calloc((size_t)(m + 1) * nv, sizeof(double));
    double *Z = calloc((size_t)m * nv, sizeof(double));
    double *w = calloc((size_t)nv, sizeof(double));
    double *H = calloc((size_t)(m + 1) * m, sizeof(double)); /* H[i*m + j] */
    double *cs = calloc((size_t)m, sizeof(double));
    double *sn = calloc((size_t)m, sizeof(double));
    double *g = calloc((size_t)m + 1, sizeof(double));
    double *yv = calloc((size_t)m, sizeof(double));
    if (!V || !Z || !w || !H || !cs || !sn || !g || !yv) {
        free(V); free(Z); free(w); free(H); free(cs); free(sn); free(g); free(yv);
        return -1;
    }
    memset(res, 0, sizeof *res);
    double bnorm = sqrt(dot(nv, b, b));
    if (bnorm == 0.0) {
        memset(x, 0, sizeof(double) * nv);
        res->converged = 1;
        goto done;
    }
    /* r0 = b - A x0 */
    orc_spmv(n, rowptr, colind, A, x, w);
    for (long k = 0; k < nv; k++)
        w[k] = b[k] - w[k];
    double beta = sqrt(dot(nv, w, w));
    res->rel_resid_true = beta / bnorm;
    res->rel_resid_est = res->rel_resid_true;
    if (hist)
        hist[0] = res->rel_resid_est;
    if (beta <= rtol * bnorm) {
        res->converged = 1;
        goto done;
    }
    while (res->iters < max_iters) {
        for (long k = 0; k < nv; k++)
            V[k] = w[k] / beta;
        memset(g, 0, sizeof(double) * (m + 1));
        g[0] = beta;
        int kdim = 0;
        for (int j = 0; j < m; j++) {
            double *vj = V + (long)j * nv, *zj = Z + (long)j * nv;
            pc(ctx, vj, zj);
            orc_spmv(n, rowptr, colind, A, zj, w);
            for (int i = 0; i <= j; i++) { /* modified Gram-Schmidt */
                double hij = dot(nv, w, V + (long)i * nv);
                H[i * m + j] = hij;
                const double *vi = V + (long)i * nv;
                for (long k = 0; k < nv; k++)
                    w[k] -= hij * vi[k];
            }
            double hn = sqrt(dot(nv, w, w));
            H[(j + 1) * m + j] = hn;
            for (int i = 0; i < j; i++) { /* previous rotations */
                double a = H[i * m + j], c = H[(i + 1) * m + j];
                H[i * m + j] = cs[i] * a + sn[i] * c;
                H[(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
            }
            double a = H[j * m + j], c = H[(j + 1) * m + j];
            double d = sqrt(a * a + c * c);
            if (d == 0.0) { cs[j] = 1.0; sn[j] = 0.0; }
            else { cs[j] = a / d; sn[j] = c / d; }
            H[j * m + j] = cs[j] * a + sn[j] * c;
            H[(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            res->iters++;
            kdim = j + 1;
            res->rel_resid_est = fabs(g[j + 1]) / bnorm;
            if (hist)
                hist[res->iters] = res->rel_resid_est;
            if (fabs(g[j + 1]) <= rtol * bnorm || hn == 0.0 || res->iters >= max_iters)
                break;
            double *vn = V + (long)(j + 1) * nv;
            for (long k = 0; k < nv; k++)
                vn[k] = w[k] / hn;
        }
        /* y = H^{-1} g (upper triangular, back substitution), x += Z y */
        for (int i = kdim - 1; i >= 0; i--) {
            double s = g[i];
            for (int k = i + 1; k < kdim; k++)
                s -= H[i * m + k] * yv[k];
            yv[i] = s / H[i * m + i];
        }
        for (int i = 0; i < kdim; i++) {
            const double *zi = Z + (long)i * nv;
            for (long k = 0; k < nv; k++)
                x[k] += yv[i] * zi[k];
        }
        res->restarts++;
        orc_spmv(n, rowptr, colind, A, x, w);
        for (long k = 0; k < nv; k++)
            w[k] = b[k] - w[k];
        beta = sqrt(dot(nv, w, w));
        res->rel_resid_true = beta / bnorm;
        if (beta <= rtol * bnorm) {
            res->converged = 1;
            break;
        }
    }
done:
    free(V); free(Z); free(w); free(H); free(cs); free(sn); free(g); free(yv);
    return res->converged ? 0 : 1;
}

/* the block (or, with Dinv == NULL, scalar) ILU preconditioner of orc_fgmres */
typedef struct {
    idx_t n;
    const idx_t *rowptr, *colind;
    const double *X, *Dinv;
    int n_lower, n_upper;
    double *work;
} ilu_pc_ctx;

static void ilu_pc(void *p, const double *r, double *z)
{
    const ilu_pc_ctx *c = p;
    if (c->Dinv)
        orc_apply(c->n, c->rowptr, c->colind, c->X, c->Dinv, r, z, c->n_lower, c->n_upper, c->work);
    else
        orc_silu_apply(c->n, c->rowptr, c->colind, c->X, r, z, c->n_lower, c->n_upper, c->work);
}

int orc_fgmres(idx_t n, const idx_t *rowptr, const idx_t *colind, const double *A,
               const double *X, const double *Dinv, int n_lower, int n_upper,
               const double *b, double *x, int m, int max_iters, double rtol,
               orc_fgmres_result *res, double *hist)
{
    ilu_pc_ctx c = {n, rowptr, colind, X, Dinv, n_lower, n_upper, NULL};
    c.work = calloc((size_t)2 * n * BS, sizeof(double));
    if (!c.work)
        return -1;
    int rc = orc_fgmres_pc(n, rowptr, colind, A, ilu_pc, &c, b, x, m, max_iters, rtol, res, hist);
    free(c.work);
    return rc;
}

/* ------------------------------------------------------------ diagnostics */

/*
 * ||x - h(x)||_1 over all entries of L and U (the ILU fixed-point residual of
 * Sec. 6.2, whose ratio to the initial one the paper plots).  h uses the
 * inverses of x's own diagonal blocks.  work: nnzb*16 + n*16 doubles.
 */
double orc_ilu_residual_l1(idx_t n, const idx_t *rowptr, const idx_t *colind,
                           const double *A, const double *X, double *work)
{
    long nnzb = rowptr[n];
    double *Xh = work, *Dx = work + nnzb * BB;
    double *Dunused = malloc(sizeof(double) * BB * (size_t)(n > 0 ? n : 1));
    for (idx_t i = 0; i < n; i++)
        orc_inv4(X + diag_pos(rowptr, colind, i) * BB, Dx + (long)i * BB);
    orc_bilu_sync_sweep(n, rowptr, colind, A, X, Dx, Xh, Dunused);
    free(Dunused);
    double s = 0.0;
    for (long k = 0; k < nnzb * BB; k++)
        s += fabs(X[k] - Xh[k]);
    return s;
}

/*
 * Largest |(LU)_ij - A_ij| over (i,j) in S_B and over the 16 entries, with
 * L_ii = I: (LU)_ij = sum_{k<min(i,j)} L_ik U_kj + (L_ij U_jj if i>j, U_ij if
 * i<=j).  Zero at the fixed point, Eq. (bilu).
 */
double orc_lu_defect_max(idx_t n, const idx_t *rowptr, const idx_t *colind,
                         const double *A, const double *X)
{
    double worst = 0.0, S[BB];
    for (idx_t i = 0; i < n; i++)
        for (long p = rowptr[i]; p < rowptr[i + 1]; p++) {
            idx_t j = colind[p];
            bilu_residual_block(i, j, p, rowptr, colind, A, X, S); /* A - sum */
            if (j < i)
                blk_sub_mul(S, X + p * BB, X + diag_pos(rowptr, colind, j) * BB);
            else
                for (int k = 0; k < BB; k++)
                    S[k] -= X[p * BB + k];
            for (int k = 0; k < BB; k++)
                if (fabs(S[k]) > worst)
                    worst = fabs(S[k]);
        }
    return worst;
}

/*
 * Max-norms of the block-Jacobi iteration matrices of the triangular solves
 * (the "diagonal dominance" measure of Sec. 6): for L (unit diagonal blocks)
 * || L - I ||_inf; for U, || D_U^{-1} (U - D_U) ||_inf with D_U the block
 * diagonal, i.e. the largest scalar row sum of |Dinv_i U_ij| over j > i.
 */
void orc_jacobi_norms(idx_t n, const idx_t *rowptr, const idx_t *colind,
                      const double *X, const double *Dinv, double *lnorm, double *unorm)
{
    double ln = 0.0, un = 0.0, P[BB];
    for (idx_t i = 0; i < n; i++) {
        double rl[BS] = {0, 0, 0, 0}, ru[BS] = {0, 0, 0, 0};
        for (long p = rowptr[i]; p < rowptr[i + 1]; p++) {
            idx_t j = colind[p];
            if (j < i) {
                for (int r = 0; r < BS; r++)
                    for (int c = 0; c < BS; c++)
                        rl[r] += fabs(X[p * BB + r * BS + c]);
            } else if (j > i) {
                blk_mul(P, Dinv + (long)i * BB, X + p * BB);
                for (int r = 0; r < BS; r++)
                    for (int c = 0; c < BS; c++)
                        ru[r] += fabs(P[r * BS + c]);
            }
        }
        for (int r = 0; r < BS; r++) {
            if (rl[r] > ln) ln = rl[r];
            if (ru[r] > un) un = ru[r];
        }
    }
    *lnorm = ln;
    *unorm = un;
}

/* ------------------------------------------------ scalar ILU(0) (Chow-Patel) */

/*
 * The scalar variant the paper compares against (Sec. 3.2, Eq.
 * scalarilu_fp_detail, Algorithm 3): ILU(0) of A taken entry by entry on the
 * scalar pattern S = every entry of every block of S_B,
 *   L_ij = (A_ij - sum_{k<j} L_ik U_kj) / U_jj   (i > j),
 *   U_ij =  A_ij - sum_{k<i} L_ik U_kj           (i <= j),
 * sums over k with (i,k) and (k,j) in S, ascending k, in a local accumulator.
 * L has a unit diagonal.  The factors are returned in A's block layout: blocks
 * left of the diagonal hold L entries, blocks right of it U entries, and a
 * diagonal block holds its strictly lower entries of L and the rest of U.
 * A zero pivot U_jj is replaced by 1 ("modified Jacobi-type iteration" of
 * Chow and Patel, Sec. 3.2) and counted.
 *
 * The oracle works on the plain scalar CSR expansion of the block pattern:
 * scalar row 4I+a holds the columns 4J+b of every block (I,J), ascending.
 */
typedef struct {
    idx_t ns;       /* scalar rows */
    long *ptr;      /* [ns+1] */
    idx_t *col;     /* [nnz] scalar columns, ascending per row */
    long *bpos;     /* [nnz] index into the block values: 16*p + 4*a + b */
    long *dpos;     /* [ns] position of the diagonal entry in the scalar row */
} scsr;

static void scsr_free(scsr *s) { free(s->ptr); free(s->col); free(s->bpos); free(s->dpos); }

static int scsr_from_blocks(idx_t n, const idx_t *rowptr, const idx_t *colind, scsr *s)
{
    s->ns = n * BS;
    long nnz = (long)rowptr[n] * BB;
    s->ptr = malloc(sizeof(long) * ((size_t)s->ns + 1));
    s->col = malloc(sizeof(idx_t) * (size_t)nnz);
    s->bpos = malloc(sizeof(long) * (size_t)nnz);
    s->dpos = malloc(sizeof(long) * (size_t)s->ns);
    if (!s->ptr || !s->col || !s->bpos || !s->dpos) { scsr_free(s); return -1; }
    long o = 0;
    for (idx_t I = 0; I < n; I++)
        for (int a = 0; a < BS; a++) {
            idx_t i = I * BS + a;
            s->ptr[i] = o;
            s->dpos[i] = -1;
            for (idx_t p = rowptr[I]; p < rowptr[I + 1]; p++)
                for (int b = 0; b < BS; b++) {
                    idx_t j = colind[p] * BS + b;
                    s->col[o] = j;
                    s->bpos[o] = (long)p * BB + a * BS + b;
                    if (j == i) s->dpos[i] = o;
                    o++;
                }
        }
    s->ptr[s->ns] = o;
    return 0;
}

/* position of scalar entry (i, j) in the expansion, or -1 */
static long scsr_find(const scsr *s, idx_t i, idx_t j)
{
    long lo = s->ptr[i], hi = s->ptr[i + 1];
    while (lo < hi) {
        long mid = (lo + hi) / 2;
        if (s->col[mid] < j) lo = mid + 1;
        else hi = mid;
    }
    return (lo < s->ptr[i + 1] && s->col[lo] == j) ? lo : -1;
}

/* A_ij - sum_{k < min(i,j)} L_ik U_kj for the entry at position o of row i,
 * reading the factors from F (block layout) */
static double silu_residual(const scsr *s, const double *A, const double *F, idx_t i, long o)
{
    idx_t j = s->col[o];
    idx_t kmax = i < j ? i : j;
    double acc = A[s->bpos[o]];
    for (long q = s->ptr[i]; q < s->ptr[i + 1] && s->col[q] < kmax; q++) {
        idx_t k = s->col[q];
        long r = scsr_find(s, k, j);
        if (r >= 0) acc -= F[s->bpos[q]] * F[s->bpos[r]];
    }
    return acc;
}

/* the pivot U_jj as used by an L update: 1 if zero or non-finite (counted) */
static double silu_pivot(const scsr *s, const double *F, idx_t j, int *nsing)
{
    double u = F[s->bpos[s->dpos[j]]];
    if (u == 0.0 || !isfinite(u)) { (*nsing)++; return 1.0; }
    return u;
}

/* Sequential scalar ILU(0): every entry once, scalar rows in order, columns
 * ascending (the Gaussian-elimination order, Algorithm 3 with one thread).
 * Returns the number of replaced pivots (or -1: out of memory). */
int orc_silu0_seq(idx_t n, const idx_t *rowptr, const idx_t *colind, const double *A, double *X)
{
    scsr s;
    if (scsr_from_blocks(n, rowptr, colind, &s)) return -1;
    int nsing = 0;
    memcpy(X, A, sizeof(double) * (size_t)rowptr[n] * BB);
    for (idx_t i = 0; i < s.ns; i++)
        for (long o = s.ptr[i]; o < s.ptr[i + 1]; o++) {
            idx_t j = s.col[o];
            double v = silu_residual(&s, A, X, i, o);
            X[s.bpos[o]] = j < i ? v / silu_pivot(&s, X, j, &nsing) : v;
        }
    scsr_free(&s);
    return nsing;
}

/* One synchronous (Jacobi-type) sweep of Eq. (scalarilu_fp): every entry of
 * Xout from Xin.  The initial guess of the iteration is A itself (Sec. 6
 * setup: L^0 = strictly lower part of A unscaled, U^0 = the rest). */
int orc_silu_sync_sweep(idx_t n, const idx_t *rowptr, const idx_t *colind, const double *A,
                        const double *Xin, double *Xout)
{
    scsr s;
    if (scsr_from_blocks(n, rowptr, colind, &s)) return -1;
    int nsing = 0;
    for (idx_t i = 0; i < s.ns; i++)
        for (long o = s.ptr[i]; o < s.ptr[i + 1]; o++) {
            idx_t j = s.col[o];
            double v = silu_residual(&s, A, Xin, i, o);
            Xout[s.bpos[o]] = j < i ? v / silu_pivot(&s, Xin, j, &nsing) : v;
        }
    scsr_free(&s);
    return nsing;
}

/* One Jacobi sweep of the scalar lower solve (unit diagonal, Algorithm 2):
 * y_out_i = r_i - sum_{j<i} L_ij y_in_j */
void orc_silu_lower_sweep(idx_t n, const idx_t *rowptr, const idx_t *colind, const double *X,
                          const double *r, const double *y_in, double *y_out)
{
    scsr s;
    if (scsr_from_blocks(n, rowptr, colind, &s)) return;
    for (idx_t i = 0; i < s.ns; i++) {
        double acc = r[i];
        for (long o = s.ptr[i]; o < s.ptr[i + 1] && s.col[o] < i; o++)
            acc -= X[s.bpos[o]] * y_in[s.col[o]];
        y_out[i] = acc;
    }
    scsr_free(&s);
}

/* One Jacobi sweep of the scalar upper solve (Algorithm 2, backward):
 * x_out_i = (y_i - sum_{j>i} U_ij x_in_j) / U_ii (a zero U_ii taken as 1) */
void orc_silu_upper_sweep(idx_t n, const idx_t *rowptr, const idx_t *colind, const double *X,
                          const double *y, const double *x_in, double *x_out)
{
    scsr s;
    if (scsr_from_blocks(n, rowptr, colind, &s)) return;
    for (idx_t i = 0; i < s.ns; i++) {
        double acc = y[i];
        for (long o = s.dpos[i] + 1; o < s.ptr[i + 1]; o++)
            acc -= X[s.bpos[o]] * x_in[s.col[o]];
        double u = X[s.bpos[s.dpos[i]]];
        if (u == 0.0 || !isfinite(u)) u = 1.0;
        x_out[i] = acc / u;
    }
    scsr_free(&s);
}

/* z ~= (L U)^{-1} r: n_lower Jacobi sweeps on L y = r from y = 0, then n_upper
 * on U z = y from z = 0 (n_lower/n_upper < 0: exact substitution).
 * work: 2 * n * 4 doubles. */
void orc_silu_apply(idx_t n, const idx_t *rowptr, const idx_t *colind, const double *X,
                    const double *r, double *z, int n_lower, int n_upper, double *work)
{
    long nv = (long)n * BS;
    double *y = work, *t = work + nv;
    if (n_lower < 0) {  /* forward substitution: the Jacobi sweep run in row order in place */
        scsr s;
        if (scsr_from_blocks(n, rowptr, colind, &s)) return;
        for (idx_t i = 0; i < s.ns; i++) {
            double acc = r[i];
            for (long o = s.ptr[i]; o < s.ptr[i + 1] && s.col[o] < i; o++)
                acc -= X[s.bpos[o]] * y[s.col[o]];
            y[i] = acc;
        }
        scsr_free(&s);
    } else {
        memset(y, 0, sizeof(double) * nv);
        for (int k = 0; k < n_lower; k++) {
            orc_silu_lower_sweep(n, rowptr, colind, X, r, y, t);
            memcpy(y, t, sizeof(double) * nv);
        }
    }
    if (n_upper < 0) {  /* back substitution */
        scsr s;
        if (scsr_from_blocks(n, rowptr, colind, &s)) return;
        for (idx_t i = s.ns - 1; i >= 0; i--) {
            double acc = y[i];
            for (long o = s.dpos[i] + 1; o < s.ptr[i + 1]; o++)
                acc -= X[s.bpos[o]] * z[s.col[o]];
            double u = X[s.bpos[s.dpos[i]]];
            if (u == 0.0 || !isfinite(u)) u = 1.0;
            z[i] = acc / u;
        }
        scsr_free(&s);
    } else {
        memset(z, 0, sizeof(double) * nv);
        for (int k = 0; k < n_upper; k++) {
            orc_silu_upper_sweep(n, rowptr, colind, X, y, z, t);
            memcpy(z, t, sizeof(double) * nv);
        }
    }
}

/* ------------------------------------------------------ multigrid smoother */
/*
 * Block ILU sweeps as the smoother of an aggregation multigrid cycle.  The
 * paper's closing section names asynchronous block ILU as a fine-grain
 * parallel multigrid smoother (and the study of its smoothing property) as
 * future work; it fixes no cycle, so this is the plain statement of the one
 * the library runs: unsmoothed aggregation (piecewise-constant transfer
 * between a cell and its aggregate), Galerkin coarse operators, and on every
 * level the smoother x += M^{-1} (b - A x) with M = L U the block ILU of that
 * level's matrix applied by triangular sweeps.
 */

/* squared Frobenius norm of a block, entries summed in storage order */
static double blk_norm2(const double *a)
{
    double s = 0.0;
    for (int e = 0; e < BB; e++)
        s += a[e] * a[e];
    return s;
}

/*
 * Greedy aggregation by strong couplings.  In row i, column j != i is a strong
 * coupling when ||A_ij||^2 > 0 and ||A_ij||^2 >= theta^2 * max_{k != i}
 * ||A_ik||^2 (Frobenius norms, compared squared).
 *   Pass 1, i ascending: a cell that is not yet placed, has at least one
 *     strong coupling, and none of whose strong neighbours is placed, roots a
 *     new aggregate made of itself and its strong neighbours.
 *   Pass 2, i ascending: a cell left over joins the pass-1 aggregate of its
 *     strongest neighbour (largest norm, the lowest column on ties) that pass
 *     1 placed; with no such neighbour it becomes an aggregate of its own.
 * Aggregates are numbered in the order they are made.  agg[n] receives each
 * cell's aggregate; returns the number of aggregates (-1: out of memory).
 */
idx_t orc_mg_aggregate(idx_t n, const idx_t *rowptr, const idx_t *colind, const double *A,
                       double theta, idx_t *agg)
{
    double *w = malloc(sizeof(double) * (size_t)(rowptr[n] > 0 ? rowptr[n] : 1));
    double *rmax = malloc(sizeof(double) * (size_t)n);
    idx_t *agg1 = malloc(sizeof(idx_t) * (size_t)n);
    if (!w || !rmax || !agg1) {
        free(w); free(rmax); free(agg1);
        return -1;
    }
    const double t2 = theta * theta;
    for (idx_t i = 0; i < n; i++) {
        rmax[i] = 0.0;
        for (long p = rowptr[i]; p < rowptr[i + 1]; p++) {
            w[p] = blk_norm2(A + p * BB);
            if (colind[p] != i && w[p] > rmax[i])
                rmax[i] = w[p];
        }
        agg[i] = -1;
    }
#define STRONG(i, p) (colind[p] != (i) && w[p] > 0.0 && w[p] >= t2 * rmax[i])
    idx_t nc = 0;
    for (idx_t i = 0; i < n; i++) {
        if (agg[i] >= 0)
            continue;
        int nstrong = 0, free_nbrs = 1;
        for (long p = rowptr[i]; p < rowptr[i + 1]; p++)
            if (STRONG(i, p)) {
                nstrong++;
                if (agg[colind[p]] >= 0)
                    free_nbrs = 0;
            }
        if (nstrong == 0 || !free_nbrs)
            continue;
        agg[i] = nc;
        for (long p = rowptr[i]; p < rowptr[i + 1]; p++)
            if (STRONG(i, p))
                agg[colind[p]] = nc;
        nc++;
    }
#undef STRONG
    memcpy(agg1, agg, sizeof(idx_t) * (size_t)n);
    for (idx_t i = 0; i < n; i++) {
        if (agg1[i] >= 0)
            continue;
        long best = -1;
        for (long p = rowptr[i]; p < rowptr[i + 1]; p++) {
            idx_t j = colind[p];
            if (j == i || agg1[j] < 0)
                continue;
            if (best < 0 || w[p] > w[best])
                best = p;
        }
        agg[i] = best >= 0 ? agg1[colind[best]] : nc++;
    }
    free(w); free(rmax); free(agg1);
    return nc;
}

/*
 * Pattern of the Galerkin coarse operator A_c = P^T A P, P the
 * piecewise-constant prolongation (P_{i,I} = I_4 when agg[i] = I): block (I,J)
 * is present when some block (i,j) of A has agg[i] = I and agg[j] = J.
 * rowptr_c[nc+1], colind_c (capacity rowptr[n]) sorted per row.  Returns the
 * number of coarse blocks (-1: out of memory).
 */
long orc_galerkin_pattern(idx_t n, const idx_t *rowptr, const idx_t *colind, const idx_t *agg,
                          idx_t nc, idx_t *rowptr_c, idx_t *colind_c)
{
    /* cells of each aggregate, by counting sort */
    idx_t *mptr = calloc((size_t)nc + 1, sizeof(idx_t));
    idx_t *mem = malloc(sizeof(idx_t) * (size_t)n);
    idx_t *mark = malloc(sizeof(idx_t) * (size_t)(nc > 0 ? nc : 1));
    if (!mptr || !mem || !mark) {
        free(mptr); free(mem); free(mark);
        return -1;
    }
    for (idx_t i = 0; i < n; i++)
        mptr[agg[i] + 1]++;
    for (idx_t I = 0; I < nc; I++)
        mptr[I + 1] += mptr[I];
    {
        idx_t *pos = malloc(sizeof(idx_t) * (size_t)(nc > 0 ? nc : 1));
        if (!pos) {
            free(mptr); free(mem); free(mark);
            return -1;
        }
        memcpy(pos, mptr, sizeof(idx_t) * (size_t)nc);
        for (idx_t i = 0; i < n; i++)
            mem[pos[agg[i]]++] = i;
        free(pos);
    }
    for (idx_t I = 0; I < nc; I++)
        mark[I] = -1;
    long nnz = 0;
    rowptr_c[0] = 0;
    for (idx_t I = 0; I < nc; I++) {
        long start = nnz;
        for (idx_t m = mptr[I]; m < mptr[I + 1]; m++) {
            idx_t i = mem[m];
            for (long p = rowptr[i]; p < rowptr[i + 1]; p++) {
                idx_t J = agg[colind[p]];
                if (mark[J] != I) {
                    mark[J] = I;
                    colind_c[nnz++] = J;
                }
            }
        }
        /* insertion sort of the row's columns */
        for (long a = start + 1; a < nnz; a++) {
            idx_t v = colind_c[a];
            long b = a - 1;
            while (b >= start && colind_c[b] > v) {
                colind_c[b + 1] = colind_c[b];
                b--;
            }
            colind_c[b + 1] = v;
        }
        rowptr_c[I + 1] = (idx_t)nnz;
    }
    free(mptr); free(mem); free(mark);
    return nnz;
}

/*
 * Values of A_c = P^T A P: every block of A, in ascending position, is added
 * entry by entry to coarse block (agg[i], agg[j]).
 */
void orc_galerkin_values(idx_t n, const idx_t *rowptr, const idx_t *colind, const double *A,
                         const idx_t *agg, idx_t nc, const idx_t *rowptr_c,
                         const idx_t *colind_c, double *Ac)
{
    memset(Ac, 0, sizeof(double) * (size_t)rowptr_c[nc] * BB);
    for (idx_t i = 0; i < n; i++)
        for (long p = rowptr[i]; p < rowptr[i + 1]; p++) {
            long c = find_block(rowptr_c, colind_c, agg[i], agg[colind[p]]);
            for (int e = 0; e < BB; e++)
                Ac[c * BB + e] += A[p * BB + e];
        }
}

/* one level of the hierarchy: its matrix, its block ILU factors and (except on
 * the coarsest level) each cell's aggregate on the next level */
typedef struct {
    idx_t n;
    const idx_t *rowptr, *colind;
    const double *A, *X, *Dinv;
    const idx_t *agg;
} orc_mg_level;

typedef struct {
    int nlevels;
    const orc_mg_level *lv;
    int n_lower, n_upper;      /* triangular sweeps per smoothing step (negative: exact) */
    int pre, post, coarse;     /* smoothing steps: before / after the coarse correction, coarsest level */
} orc_mg;

/* `steps` smoothing steps x += M^{-1} (b - A x) on level l */
static void mg_smooth(const orc_mg_level *L, int n_lower, int n_upper, int steps,
                      const double *b, double *x, double *r, double *z, double *work)
{
    long nv = (long)L->n * BS;
    for (int s = 0; s < steps; s++) {
        orc_spmv(L->n, L->rowptr, L->colind, L->A, x, r);
        for (long k = 0; k < nv; k++)
            r[k] = b[k] - r[k];
        orc_apply(L->n, L->rowptr, L->colind, L->X, L->Dinv, r, z, n_lower, n_upper, work);
        for (long k = 0; k < nv; k++)
            x[k] += z[k];
    }
}

/* x = V-cycle on level l applied to b, from x = 0 */
static int mg_vcycle_level(const orc_mg *mg, int l, const double *b, double *x)
{
    const orc_mg_level *L = mg->lv + l;
    long nv = (long)L->n * BS;
    double *r = malloc(sizeof(double) * (size_t)nv);
    double *z = malloc(sizeof(double) * (size_t)nv);
    double *work = malloc(sizeof(double) * (size_t)(2 * nv));
    if (!r || !z || !work) {
        free(r); free(z); free(work);
        return -1;
    }
    memset(x, 0, sizeof(double) * (size_t)nv);
    int rc = 0;
    if (l == mg->nlevels - 1) {
        mg_smooth(L, mg->n_lower, mg->n_upper, mg->coarse, b, x, r, z, work);
    } else {
        const orc_mg_level *Lc = mg->lv + l + 1;
        long nvc = (long)Lc->n * BS;
        double *bc = calloc((size_t)nvc, sizeof(double));
        double *xc = malloc(sizeof(double) * (size_t)nvc);
        if (!bc || !xc) {
            free(bc); free(xc); free(r); free(z); free(work);
            return -1;
        }
        mg_smooth(L, mg->n_lower, mg->n_upper, mg->pre, b, x, r, z, work);
        /* restriction of the residual: b_c = P^T (b - A x), cells in ascending order */
        orc_spmv(L->n, L->rowptr, L->colind, L->A, x, r);
        for (long k = 0; k < nv; k++)
            r[k] = b[k] - r[k];
        for (idx_t i = 0; i < L->n; i++)
            for (int c = 0; c < BS; c++)
                bc[(long)L->agg[i] * BS + c] += r[(long)i * BS + c];
        rc = mg_vcycle_level(mg, l + 1, bc, xc);
        /* prolongation of the correction: x_i += x_c[agg(i)] */
        for (idx_t i = 0; i < L->n; i++)
            for (int c = 0; c < BS; c++)
                x[(long)i * BS + c] += xc[(long)L->agg[i] * BS + c];
        mg_smooth(L, mg->n_lower, mg->n_upper, mg->post, b, x, r, z, work);
        free(bc); free(xc);
    }
    free(r); free(z); free(work);
    return rc;
}

/* z = one V-cycle applied to r (the multigrid preconditioner); 0 on success */
int orc_mg_vcycle(const orc_mg *mg, const double *r, double *z)
{
    return mg_vcycle_level(mg, 0, r, z);
}

static void mg_pc(void *p, const double *r, double *z)
{
    orc_mg_vcycle((const orc_mg *)p, r, z);
}

/* FGMRES(m) on level 0's matrix, right-preconditioned by one V-cycle */
int orc_fgmres_mg(const orc_mg *mg, const double *b, double *x, int m, int max_iters,
                  double rtol, orc_fgmres_result *res, double *hist)
{
    const orc_mg_level *L = mg->lv;
    return orc_fgmres_pc(L->n, L->rowptr, L->colind, L->A, mg_pc, (void *)mg, b, x, m, max_iters,
                         rtol, res, hist);
}

/* --------------------------------------------------- threshold block ILU */
/*
 * Building blocks of a threshold block ILU computed by fixed-point sweeps (the
 * paper's closing section names a parallel threshold ILU, ParILUT, as the
 * next extension of its sweeps).  The loop itself (oracle/__init__.py,
 * parilut) alternates: add the fill of L U to the pattern, one synchronous
 * sweep, keep the largest blocks, one synchronous sweep.
 */

static int cmp_idx(const void *a, const void *b)
{
    idx_t x = *(const idx_t *)a, y = *(const idx_t *)b;
    return (x > y) - (x < y);
}

/*
 * Block pattern of L U for factors on the pattern (rowptr, colind), L unit
 * lower (its diagonal blocks are identities) and U upper: row i holds every
 * column j >= k of row k, for k = i and for every column k < i of row i.
 * rowptr_out[n+1]; colind_out (NULL: count only) sorted per row.  Returns the
 * number of blocks (-1: out of memory).
 */
long orc_lu_pattern(idx_t n, const idx_t *rowptr, const idx_t *colind, idx_t *rowptr_out,
                    idx_t *colind_out)
{
    idx_t *mark = malloc(sizeof(idx_t) * (size_t)n);
    idx_t *buf = malloc(sizeof(idx_t) * (size_t)n);
    if (!mark || !buf) {
        free(mark); free(buf);
        return -1;
    }
    for (idx_t i = 0; i < n; i++)
        mark[i] = -1;
    long nnz = 0;
    rowptr_out[0] = 0;
    for (idx_t i = 0; i < n; i++) {
        idx_t cnt = 0;
        for (long p = rowptr[i]; p < rowptr[i + 1]; p++) {
            idx_t k = colind[p];
            if (k > i)
                break;
            /* k = i (the unit diagonal of L) or k < i: the upper part of row k */
            for (long q = rowptr[k]; q < rowptr[k + 1]; q++) {
                idx_t j = colind[q];
                if (j < k || mark[j] == i)
                    continue;
                mark[j] = i;
                buf[cnt++] = j;
            }
        }
        qsort(buf, (size_t)cnt, sizeof(idx_t), cmp_idx);
        if (colind_out)
            memcpy(colind_out + nnz, buf, sizeof(idx_t) * (size_t)cnt);
        nnz += cnt;
        rowptr_out[i + 1] = (idx_t)nnz;
    }
    free(mark); free(buf);
    return nnz;
}

static int cmp_desc(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x < y) - (x > y);
}

/*
 * keep[t] = 1 for the entries whose key exceeds the (budget+1)-th largest key
 * (every entry when there are at most `budget`): at most `budget` entries,
 * and of two entries with equal keys both or neither.  Returns the number kept.
 */
long orc_keep_largest(long m, const double *key, long budget, unsigned char *keep)
{
    if (m <= budget) {
        memset(keep, 1, (size_t)m);
        return m;
    }
    double *s = malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    if (!s)
        return -1;
    memcpy(s, key, sizeof(double) * (size_t)m);
    qsort(s, (size_t)m, sizeof(double), cmp_desc);
    const double v = s[budget];
    long kept = 0;
    for (long t = 0; t < m; t++) {
        keep[t] = key[t] > v;
        kept += keep[t];
    }
    free(s);
    return kept;
}

/* FGMRES on A (pattern rowptr/colind) preconditioned by block ILU factors on
 * their own pattern (rowptr_f/colind_f), e.g. the filled pattern of the
 * threshold ILU */
int orc_fgmres_ilu_pattern(idx_t n, const idx_t *rowptr, const idx_t *colind, const double *A,
                           const idx_t *rowptr_f, const idx_t *colind_f, const double *X,
                           const double *Dinv, int n_lower, int n_upper, const double *b,
                           double *x, int m, int max_iters, double rtol, orc_fgmres_result *res,
                           double *hist)
{
    ilu_pc_ctx c = {n, rowptr_f, colind_f, X, Dinv, n_lower, n_upper, NULL};
    c.work = calloc((size_t)2 * n * BS, sizeof(double));
    if (!c.work)
        return -1;
    int rc = orc_fgmres_pc(n, rowptr, colind, A, ilu_pc, &c, b, x, m, max_iters, rtol, res, hist);
    free(c.work);
    return rc;
}

/*
 * X[p] = A[p] for every strictly upper block (i,j) of the pattern with no
 * product pair (no k < i with (i,k) and (k,j) in the pattern): its update is
 * the constant A_ij, and a build sets such blocks to that value before its
 * first sweep, whatever the initial guess held (a choice of initial guess).
 */
void orc_fix_constant_upper(idx_t n, const idx_t *rowptr, const idx_t *colind, const double *A,
                            double *X)
{
    for (idx_t i = 0; i < n; i++)
        for (long p = rowptr[i]; p < rowptr[i + 1]; p++) {
            idx_t j = colind[p];
            if (j <= i)
                continue;
            int has_pair = 0;
            for (long q = rowptr[i]; q < rowptr[i + 1] && !has_pair; q++) {
                idx_t k = colind[q];
                if (k >= i)
                    break;
                if (find_block(rowptr, colind, k, j) >= 0)
                    has_pair = 1;
            }
            if (!has_pair)
                memcpy(X + p * BB, A + p * BB, sizeof(double) * BB);
        }
}
