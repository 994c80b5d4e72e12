// Block sparse matrix-vector product y = alpha A x + beta y, FP64, 4x4 blocks
// (the public bsr_spmv).
//
// FGMRES needs one product per iteration plus the residual at each restart
// (Sec. 6 setup); inside the solve those run in the kernel that also takes the
// Gram-Schmidt dot products (k_spmv_dots, fgmres.cu) and in the residual
// kernels, all with this kernel's row product (spmv.cuh).  Bytes dominate:
// every block is 128 bytes of FP64 values
// plus a 4-byte column index, read exactly once; x (4N doubles) is gathered
// through L1/L2.  A quad of threads handles one block row: thread q reads row q
// of every block of the row (32 contiguous bytes; the quad together reads each
// 128-byte block as one fully used line), forms the 4-term dot product with
// x_j, and writes y_i[q].  The first four blocks of a row are loaded before
// any arithmetic so each thread keeps up to 8 independent 16-byte loads in
// flight.  FP64 work is the minimum, 16 FMA per block: one running FMA chain
// per output entry (FP64 throughput on this GPU is ~1.2 TFLOP/s, so at
// 0.25 flop per byte the FP64 pipe, not only HBM, bounds this kernel).
#include "common.cuh"
#include "spmv.cuh"

namespace abilu {

constexpr int SPMV_THREADS = 256;
constexpr int SPMV_ROWS = SPMV_THREADS / 4;

// PLAIN: y = A x (alpha = 1, beta = 0, decided on the host), the form FGMRES
// uses: no FP64 instruction beyond the 16 FMA per block (a compare and a
// multiply per output would add ~12% to this FP64-pipe-bound kernel).
// Otherwise y = alpha A x + beta y, and beta == 0 never reads y (which may
// hold NaN).
template <bool PLAIN>
__global__ void __launch_bounds__(SPMV_THREADS)
k_spmv(PatternView P, const double *__restrict__ A, double alpha, const double *__restrict__ x,
       double beta, double *__restrict__ y, Skip skip) {
    pdl_wait();
    pdl_trigger();
    if (skip_all(skip) || skip_chunk(skip, blockIdx.x)) return;
    const int i = blockIdx.x * SPMV_ROWS + (threadIdx.x >> 2), q = threadIdx.x & 3;
    if (i >= P.n) return;
    const double s = row_dot_blocks(P, A, x, i, q);
    const size_t o = (size_t)i * BS + q;
    if constexpr (PLAIN) y[o] = s;
    else y[o] = beta == 0.0 ? alpha * s : alpha * s + beta * y[o];
}

abilu_status spmv_launch(const PatternView &P, const double *A, double alpha, const double *x,
                         double beta, double *y, cudaStream_t st, Skip skip) {
    static_assert(SPMV_ROWS == SKIP_CHUNK_ROWS, "one CTA per 64-row chunk");
    const int grid = (P.n + SPMV_ROWS - 1) / SPMV_ROWS;
    if (alpha == 1.0 && beta == 0.0)
        launch_pdl(k_spmv<true>, grid, SPMV_THREADS, 0, st, P, A, alpha, x, beta, y, skip);
    else
        launch_pdl(k_spmv<false>, grid, SPMV_THREADS, 0, st, P, A, alpha, x, beta, y, skip);
    ABILU_LAUNCH_CHECK("k_spmv");
    return ABILU_OK;
}

}  // namespace abilu
