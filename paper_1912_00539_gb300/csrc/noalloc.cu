// abilu_apply_noalloc: the synchronous FP64 preconditioner application for
// callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running inside another library's
// allocator hooks or memory pools, callers whose device memory is entirely
// pre-reserved by a framework, and code that must not allocate while a CUDA
// graph is being built.  They still need z ~= (LU)^{-1} r.  abilu_apply keeps
// its sweep vectors in a factors handle, which abilu_factors_create obtains
// with cudaMalloc; this entry point takes the factors as plain arrays instead
// and keeps its sweep vectors in a file-scope __device__ array of fixed size,
// so it allocates nothing.
//
// The scratch array holds three vectors of at most NOALLOC_MAX_CELLS cells
// (3 x 65,536 x 4 doubles = 6 MiB).  Every GPU that loads the library holds
// it until the process exits.  Every call shares it: two calls whose work
// overlaps on the GPU (different streams, or different host threads) race on
// it and produce wrong results; serialise them on one stream.  Nothing in the
// array has to start at zero: each call writes every scratch entry it reads.
//
// The pattern is trusted as far as abilu_pattern_create would accept it; the
// sweep only skips a column outside [0, n), so a malformed column index reads
// nothing out of bounds (the result of such a row is then meaningless).
#include <mutex>

#include "common.cuh"

namespace abilu {

constexpr int NOALLOC_MAX_CELLS = 65536;
constexpr int NOALLOC_THREADS = 256;
constexpr int NOALLOC_ROWS = NOALLOC_THREADS / 4;

// three FP64 vectors of NOALLOC_MAX_CELLS cells
static __device__ __align__(256) double g_noalloc_scratch[3 * NOALLOC_MAX_CELLS * BS];

// One Jacobi sweep on the factors in A's pattern layout (X: L_ij at column <
// row, U_ij at column > row; Dinv separate).  lower: out_i = r_i - sum_{j<i}
// L_ij in_j (in == nullptr means in = 0);  upper: out_i = Dinv_i (y_i -
// sum_{j>i} U_ij in_j).  A quad of threads per block row, thread q computes
// entry q; the row's blocks are scanned in column order.
__global__ void __launch_bounds__(NOALLOC_THREADS)
k_noalloc_sweep(int n, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colind,
                const double *__restrict__ X, const double *__restrict__ Dinv,
                const double *__restrict__ rhs, const double *__restrict__ in,
                double *__restrict__ out, int upper) {
    const int i = blockIdx.x * NOALLOC_ROWS + (threadIdx.x >> 2), q = threadIdx.x & 3;
    if (i >= n) return;
    double s = rhs ? rhs[(size_t)i * BS + q] : 0.0;
    if (in) {
        const int p1 = rowptr[i + 1];
        for (int p = rowptr[i]; p < p1; p++) {
            const int j = colind[p];
            if (j < 0 || j >= n || (upper ? j <= i : j >= i)) continue;
            double a[4], v[4];
            ld_row(X + (size_t)p * BB + q * BS, a);
            ld_row(in + (size_t)j * BS, v);
            s -= a[0] * v[0] + a[1] * v[1] + a[2] * v[2] + a[3] * v[3];
        }
    }
    if (upper) {
        double d[4], t[4];
        ld_row(Dinv + (size_t)i * BB + q * BS, d);
        t[0] = qshfl(s, 0); t[1] = qshfl(s, 1); t[2] = qshfl(s, 2); t[3] = qshfl(s, 3);
        s = d[0] * t[0] + d[1] * t[1] + d[2] * t[2] + d[3] * t[3];
    }
    out[(size_t)i * BS + q] = s;
}

// Device address of the scratch array, looked up once per device with that
// device current (the array's host-side name is only a stand-in).  The cache
// is never invalidated: after cudaDeviceReset the device's context, and with
// it this address, is gone, so the entry point must not be used on that
// device again in this process.
static double *scratch_for_current_device(abilu_status *st) {
    static std::mutex mu;
    static double *addr[128] = {nullptr};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 128) {
        *st = e != cudaSuccess ? cuda_fail(e, "apply_noalloc: cudaGetDevice")
                               : fail(ABILU_EINVAL, "apply_noalloc: device index %d", dev);
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            *st = cuda_fail(e, "apply_noalloc: cudaGetSymbolAddress");
            return nullptr;
        }
        addr[dev] = static_cast<double *>(p);
    }
    *st = ABILU_OK;
    return addr[dev];
}

}  // namespace abilu

using namespace abilu;

extern "C" abilu_status abilu_apply_noalloc(int32_t n, const int32_t *rowptr,
                                            const int32_t *colind, const double *X,
                                            const double *Dinv, const double *r, double *z,
                                            int nsweeps_lower, int nsweeps_upper,
                                            abilu_stream stream) {
    if (n < 1) return fail(ABILU_EINVAL, "apply_noalloc: n must be >= 1");
    if (n > NOALLOC_MAX_CELLS)
        return fail(ABILU_EINVAL, "apply_noalloc: n = %d exceeds the fixed scratch limit of %d cells",
                    n, NOALLOC_MAX_CELLS);
    if (!rowptr || !colind || !X || !Dinv || !r || !z)
        return fail(ABILU_EINVAL, "apply_noalloc: NULL argument");
    if (r == z) return fail(ABILU_EINVAL, "apply_noalloc: r and z must be distinct");
    // the sweeps read X, Dinv and r with 16-byte vector loads: reject a view
    // that starts off that boundary here, on the host, before any launch
    auto al16 = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    if (!al16(X) || !al16(Dinv) || !al16(r) || !al16(z))
        return fail(ABILU_EINVAL, "apply_noalloc: X, Dinv, r and z must be 16-byte aligned");
    if ((reinterpret_cast<uintptr_t>(rowptr) & 3u) || (reinterpret_cast<uintptr_t>(colind) & 3u))
        return fail(ABILU_EINVAL, "apply_noalloc: rowptr and colind must be 4-byte aligned");
    if (nsweeps_lower < 0 || nsweeps_upper < 0)
        return fail(ABILU_EINVAL, "apply_noalloc: negative sweep count");
    abilu_status st;
    double *scr = scratch_for_current_device(&st);
    if (!scr) return st;
    cudaStream_t cs = S(stream);
    const size_t nv = (size_t)n * BS;
    double *B[3] = {scr, scr + (size_t)NOALLOC_MAX_CELLS * BS, scr + 2 * (size_t)NOALLOC_MAX_CELLS * BS};
    const int grid = (n + NOALLOC_ROWS - 1) / NOALLOC_ROWS;
    // lower sweeps from y^0 = 0: y^1 = r, y^s in B[s & 1]; y == nullptr means y = 0
    const double *y = nullptr;
    if (nsweeps_lower >= 1) y = r;
    for (int s = 2; s <= nsweeps_lower; s++) {
        k_noalloc_sweep<<<counted(grid), NOALLOC_THREADS, 0, cs>>>(n, rowptr, colind, X, Dinv, r, y,
                                                                   B[s & 1], 0);
        ABILU_LAUNCH_CHECK("k_noalloc_sweep lower");
        y = B[s & 1];
    }
    // upper sweeps from x^0 = 0 in the two buffers y does not occupy
    double *xb[2];
    if (y == B[0]) { xb[0] = B[1]; xb[1] = B[2]; }
    else if (y == B[1]) { xb[0] = B[0]; xb[1] = B[2]; }
    else { xb[0] = B[0]; xb[1] = B[1]; }
    const double *x = nullptr;  // nullptr means x = 0
    for (int s = 1; s <= nsweeps_upper; s++) {
        double *out = s == nsweeps_upper ? z : xb[s & 1];
        k_noalloc_sweep<<<counted(grid), NOALLOC_THREADS, 0, cs>>>(n, rowptr, colind, X, Dinv, y, x,
                                                                   out, 1);
        ABILU_LAUNCH_CHECK("k_noalloc_sweep upper");
        x = out;
    }
    if (nsweeps_upper == 0) ABILU_CUDA(cudaMemsetAsync(z, 0, sizeof(double) * nv, cs));
    return ABILU_OK;
}
