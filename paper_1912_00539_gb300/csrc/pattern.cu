// Pattern analysis of the block sparsity pattern S_B (Sec. 4.2).
//
// For every block (i,j) of S_B the fixed-point map H_ij of Eq. (blockH) needs
// the products X_ik X_kj with k < min(i,j) and both (i,k) and (k,j) in S_B.
// These pair lists depend only on the pattern, so they are computed once per
// pattern and reused by every sweep of every build (values change per
// pseudo-time step, the pattern does not; Sec. 5 reorders the grid once).
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "common.cuh"

namespace abilu {

static thread_local char g_msg[512] = "";

abilu_status fail(abilu_status s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof g_msg, fmt, ap);
    va_end(ap);
    return s;
}

abilu_status cuda_fail(cudaError_t e, const char *what) {
    return fail(e == cudaErrorMemoryAllocation ? ABILU_ENOMEM : ABILU_ECUDA, "%s: %s (%s)", what,
                cudaGetErrorString(e), cudaGetErrorName(e));
}

const char *last_error() { return g_msg; }

static unsigned long long g_launches = 0;
void note_launch() { __atomic_add_fetch(&g_launches, 1ull, __ATOMIC_RELAXED); }
void note_launches(long long d) {
    __atomic_add_fetch(&g_launches, (unsigned long long)d, __ATOMIC_RELAXED);
}
unsigned long long launches() { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

// ------------------------------------------------------------------ scan
// Exclusive prefix sum of int32 counts into int32 offsets (out has n+1
// entries; out[n] = total).  Three passes: tile scans, a one-CTA scan of the
// tile totals, then the tile offsets are added.
constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__global__ void k_scan_tiles(const int32_t *__restrict__ in, int32_t *__restrict__ out,
                             long long *__restrict__ tile_sum, int n) {
    __shared__ long long sh[SCAN_THREADS];
    long long base = (long long)blockIdx.x * SCAN_TILE + (long long)threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS];
    long long s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        long long idx = base + k;
        v[k] = idx < n ? in[idx] : 0;
        s += v[k];
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < SCAN_THREADS; off <<= 1) {  // Hillis-Steele, inclusive
        long long t = threadIdx.x >= (unsigned)off ? sh[threadIdx.x - off] : 0;
        __syncthreads();
        sh[threadIdx.x] += t;
        __syncthreads();
    }
    long long run = sh[threadIdx.x] - s;  // exclusive prefix of this thread
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        long long idx = base + k;
        if (idx < n) out[idx] = (int32_t)run;
        run += v[k];
    }
    if (threadIdx.x == SCAN_THREADS - 1) tile_sum[blockIdx.x] = sh[threadIdx.x];
}

__global__ void k_scan_top(long long *tile_sum, int ntiles, int32_t *out_total_slot,
                           unsigned *err) {
    // one CTA: exclusive scan of the tile totals in chunks, carrying the sum
    __shared__ long long sh[SCAN_THREADS];
    long long carry = 0;
    for (int c0 = 0; c0 < ntiles; c0 += SCAN_THREADS) {
        int i = c0 + threadIdx.x;
        long long v = i < ntiles ? tile_sum[i] : 0;
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < SCAN_THREADS; off <<= 1) {
            long long t = threadIdx.x >= (unsigned)off ? sh[threadIdx.x - off] : 0;
            __syncthreads();
            sh[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < ntiles) tile_sum[i] = carry + sh[threadIdx.x] - v;
        long long tot = sh[SCAN_THREADS - 1];
        __syncthreads();
        carry += tot;
    }
    if (threadIdx.x == 0) {
        if (carry > 0x7fffffffLL) atomicOr(err, 1u << 8);
        *out_total_slot = (int32_t)carry;
    }
}

__global__ void k_scan_add(int32_t *out, const long long *tile_off, int n) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < n) out[idx] += (int32_t)tile_off[idx / SCAN_TILE];
}

// out[0..n] = exclusive scan of in[0..n-1]; scratch >= ceil(n/TILE) long longs;
// a total above 2^31 - 1 sets bit 8 of *err
abilu_status scan_i32(const int32_t *in, int32_t *out, int n, long long *scratch, unsigned *err,
                      cudaStream_t st) {
    int ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (ntiles < 1) ntiles = 1;
    k_scan_tiles<<<counted(ntiles), SCAN_THREADS, 0, st>>>(in, out, scratch, n);
    k_scan_top<<<counted(1), SCAN_THREADS, 0, st>>>(scratch, ntiles, out + n, err);
    const int add_grid = n > 0 ? (n + 255) / 256 : 1;
    k_scan_add<<<counted(add_grid), 256, 0, st>>>(out, scratch, n);
    ABILU_LAUNCH_CHECK("scan");
    return ABILU_OK;
}

// ------------------------------------------------------------ row analysis
// error bits
enum : unsigned {
    PAT_BAD_ROWPTR = 1u, PAT_BAD_COL = 2u, PAT_UNSORTED = 4u, PAT_NO_DIAG = 8u,
};

__global__ void k_pat_rows(int n, int nnzb, const int32_t *__restrict__ rowptr,
                           const int32_t *__restrict__ colind, int32_t *__restrict__ diagpos,
                           int32_t *__restrict__ lcnt, int32_t *__restrict__ ucnt,
                           unsigned *err, int *max_row) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int p0 = rowptr[i], p1 = rowptr[i + 1];
    if ((i == 0 && p0 != 0) || (i == n - 1 && p1 != nnzb) || p0 < 0 || p1 < p0 || p1 > nnzb) {
        atomicOr(err, PAT_BAD_ROWPTR);
        diagpos[i] = 0; lcnt[i] = 0; ucnt[i] = 0;
        return;
    }
    int dp = -1, prev = -1;
    unsigned e = 0;
    for (int p = p0; p < p1; p++) {
        int j = colind[p];
        if (j < 0 || j >= n) e |= PAT_BAD_COL;
        if (j <= prev) e |= PAT_UNSORTED;
        if (j == i) dp = p;
        prev = j;
    }
    if (dp < 0) e |= PAT_NO_DIAG;
    if (e) atomicOr(err, e);
    if (dp < 0) dp = p0;
    diagpos[i] = dp;
    lcnt[i] = dp - p0;
    ucnt[i] = p1 - dp - (dp < p1 ? 1 : 0);
    atomicMax(max_row, p1 - p0);
}

__global__ void k_pat_cols(int n, const int32_t *__restrict__ rowptr,
                           const int32_t *__restrict__ colind, const int32_t *__restrict__ diagpos,
                           const int32_t *__restrict__ lrow, const int32_t *__restrict__ urow,
                           int32_t *__restrict__ lcol, int32_t *__restrict__ ucol) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int p0 = rowptr[i], p1 = rowptr[i + 1], dp = diagpos[i];
    int l = lrow[i], u = urow[i];
    for (int p = p0; p < dp; p++) lcol[l++] = colind[p];
    for (int p = dp + 1; p < p1; p++) ucol[u++] = colind[p];
}

// position of column j among the strictly-upper blocks of row k, or -1
__device__ __forceinline__ int find_upper(const int32_t *__restrict__ colind, int lo, int hi,
                                          int j) {
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        int c = colind[mid];
        if (c == j) return mid;
        if (c < j) lo = mid + 1; else hi = mid;
    }
    return -1;
}

// FILL = false: count the pairs of each block; FILL = true: write them.
template <bool FILL>
__global__ void k_pat_pairs(int n, const int32_t *__restrict__ rowptr,
                            const int32_t *__restrict__ colind, const int32_t *__restrict__ diagpos,
                            const int32_t *__restrict__ lrow, const int32_t *__restrict__ urow,
                            int32_t *__restrict__ pair_cnt, const int32_t *__restrict__ pair_ptr,
                            int2 *__restrict__ pairs) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int p0 = rowptr[i], p1 = rowptr[i + 1], dp = diagpos[i];
    for (int p = p0; p < p1; p++) {
        int j = colind[p];
        int kmax = i < j ? i : j;
        int c = 0;
        int out = FILL ? pair_ptr[p] : 0;
        for (int q = p0; q < dp; q++) {  // L blocks (i,k), k ascending
            int k = colind[q];
            if (k >= kmax) break;
            int r = find_upper(colind, diagpos[k] + 1, rowptr[k + 1], j);
            if (r < 0) continue;
            if (FILL)
                pairs[out + c] = make_int2(lrow[i] + (q - p0), urow[k] + (r - diagpos[k] - 1));
            c++;
        }
        if (!FILL) pair_cnt[p] = c;
    }
}

// FILL = false: count the row's work blocks; FILL = true: write them
template <bool FILL>
__global__ void k_pat_work(int n, const int32_t *__restrict__ rowptr,
                           const int32_t *__restrict__ colind, const int32_t *__restrict__ diagpos,
                           const int32_t *__restrict__ lrow, const int32_t *__restrict__ urow,
                           const int32_t *__restrict__ pair_ptr, int32_t *__restrict__ wcnt,
                           const int32_t *__restrict__ wptr, int4 *__restrict__ work) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int p0 = rowptr[i], p1 = rowptr[i + 1], dp = diagpos[i];
    int c = 0, out = FILL ? wptr[i] : 0;
    for (int p = p0; p < p1; p++) {
        if (p > dp && pair_ptr[p] == pair_ptr[p + 1]) continue;  // constant U block
        if (FILL) {
            int kind = p < dp ? WORK_L : (p == dp ? WORK_D : WORK_U);
            int dst = p < dp ? lrow[i] + (p - p0) : (p == dp ? i : urow[i] + (p - dp - 1));
            work[out + c] = make_int4(p, colind[p], dst, kind);
        }
        c++;
    }
    if (!FILL) wcnt[i] = c;
}

// Inside each chunk of `chunk` consecutive work blocks, put the diagonal
// blocks first, then the L blocks, then the U blocks (stable).  The blocks of a
// chunk are processed concurrently by one CTA, so the order inside a chunk
// changes no result; grouping the kinds keeps the warps of a CTA on one code
// path (the diagonal path also inverts U_ii).
__global__ void k_pat_work_sort(int nwork, int chunk, int4 *work) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int w0 = c * chunk;
    if (w0 >= nwork) return;
    const int w1 = w0 + chunk < nwork ? w0 + chunk : nwork;
    int4 buf[64];
    for (int w = w0; w < w1; w++) buf[w - w0] = work[w];
    int out = w0;
    const int order[3] = {WORK_D, WORK_L, WORK_U};
    for (int o = 0; o < 3; o++)
        for (int k = 0; k < w1 - w0; k++)
            if (buf[k].w == order[o]) work[out++] = buf[k];
}

// After the sort: the 32-byte records the sweeps read (pair range and the
// first two pairs inline) and wpos[p] = w, where the FP32 copy of A_p goes.
__global__ void k_pat_work_items(int nwork, const int4 *__restrict__ work,
                                 const int32_t *__restrict__ pair_ptr,
                                 const int2 *__restrict__ pairs, int32_t *__restrict__ wpos,
                                 WorkItem *__restrict__ items) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nwork) return;
    const int4 r = work[w];
    const int t0 = pair_ptr[r.x], np = pair_ptr[r.x + 1] - t0;
    WorkItem it;
    it.j = r.y;
    it.dst = r.z;
    it.kind_np = r.w | (np << 2);
    it.t0 = t0;
    it.pr[0] = np > 0 ? pairs[t0] : make_int2(0, 0);
    it.pr[1] = np > 1 ? pairs[t0 + 1] : make_int2(0, 0);
    items[w] = it;
    wpos[r.x] = w;
}

}  // namespace abilu

using namespace abilu;

extern "C" const char *abilu_last_error(void) { return last_error(); }
extern "C" const char *abilu_version(void) { return "abilu-gb300 0.1"; }
extern "C" uint64_t abilu_kernel_launches(void) { return launches(); }

static void pattern_free(abilu_pattern p) {
    if (!p) return;
    std::vector<void *> *allocs = reinterpret_cast<std::vector<void *> *>(p->mem);
    if (allocs) {
        for (void *a : *allocs) cudaFree(a);
        delete allocs;
    }
    delete p;
}

extern "C" void abilu_pattern_destroy(abilu_pattern p) { pattern_free(p); }

extern "C" abilu_status abilu_pattern_create(int32_t n, int32_t nnzb, const int32_t *rowptr,
                                             const int32_t *colind, abilu_stream stream,
                                             abilu_pattern *out) {
    if (!out) return fail(ABILU_EINVAL, "pattern_create: out is NULL");
    *out = nullptr;
    if (n < 1 || nnzb < n) return fail(ABILU_EINVAL, "pattern_create: need n >= 1 and nnzb >= n (n=%d nnzb=%d)", n, nnzb);
    // block indices of the build's work list stay 32-bit with slack for its
    // last ticket (far beyond any system that fits the device: 2^31 blocks of
    // A alone are 275 GB)
    if (nnzb > INT32_MAX - (1 << 16))
        return fail(ABILU_EINVAL, "pattern_create: nnzb=%d above 2^31 - 2^16", nnzb);
    if (!rowptr || !colind) return fail(ABILU_EINVAL, "pattern_create: NULL rowptr/colind");
    cudaStream_t st = S(stream);
    abilu_pattern p = new abilu_pattern_s();
    memset(&p->v, 0, sizeof p->v);
    auto allocs = new std::vector<void *>();
    p->mem = allocs;
    cudaGetDevice(&p->device);
    auto alloc = [&](void **ptr, size_t bytes) -> abilu_status {
        cudaError_t e = cudaMalloc(ptr, bytes < 16 ? 16 : bytes);
        if (e != cudaSuccess) return cuda_fail(e, "pattern_create: cudaMalloc");
        allocs->push_back(*ptr);
        return ABILU_OK;
    };
#define TRY(x)                                   \
    do {                                         \
        abilu_status s_ = (x);                   \
        if (s_ != ABILU_OK) { pattern_free(p); return s_; } \
    } while (0)
    int32_t *d_rowptr, *d_colind, *diagpos, *lcnt, *ucnt, *lrow, *urow, *pair_cnt, *pair_ptr;
    long long *scratch;
    unsigned *err;
    int *max_row;
    int ntiles = (nnzb + SCAN_TILE - 1) / SCAN_TILE + 1;
    TRY(alloc((void **)&d_rowptr, sizeof(int32_t) * (n + 1)));
    TRY(alloc((void **)&d_colind, sizeof(int32_t) * nnzb));
    TRY(alloc((void **)&diagpos, sizeof(int32_t) * n));
    TRY(alloc((void **)&lcnt, sizeof(int32_t) * n));
    TRY(alloc((void **)&ucnt, sizeof(int32_t) * n));
    // +68 entries: a sweep copies rowptr windows of 68 entries per 64-row chunk
    TRY(alloc((void **)&lrow, sizeof(int32_t) * (n + 1 + 68)));
    TRY(alloc((void **)&urow, sizeof(int32_t) * (n + 1 + 68)));
    TRY(alloc((void **)&pair_cnt, sizeof(int32_t) * nnzb));
    TRY(alloc((void **)&pair_ptr, sizeof(int32_t) * (nnzb + 1)));
    TRY(alloc((void **)&scratch, sizeof(long long) * ntiles));
    TRY(alloc((void **)&err, sizeof(unsigned) * 4));
    max_row = reinterpret_cast<int *>(err + 2);
    auto cu = [&](cudaError_t e, const char *w) -> abilu_status {
        return e == cudaSuccess ? ABILU_OK : cuda_fail(e, w);
    };
    TRY(cu(cudaMemcpyAsync(d_rowptr, rowptr, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToDevice, st), "copy rowptr"));
    TRY(cu(cudaMemcpyAsync(d_colind, colind, sizeof(int32_t) * nnzb, cudaMemcpyDeviceToDevice, st), "copy colind"));
    TRY(cu(cudaMemsetAsync(err, 0, sizeof(unsigned) * 4, st), "memset"));
    int gb = (n + 255) / 256;
    k_pat_rows<<<counted(gb), 256, 0, st>>>(n, nnzb, d_rowptr, d_colind, diagpos, lcnt, ucnt, err, max_row);
    TRY(cu(cudaGetLastError(), "k_pat_rows"));
    unsigned herr[4];
    TRY(cu(cudaMemcpyAsync(herr, err, sizeof herr, cudaMemcpyDeviceToHost, st), "read err"));
    TRY(cu(cudaStreamSynchronize(st), "sync"));
    if (herr[0]) {
        pattern_free(p);
        return fail(ABILU_EINVAL, "pattern_create: malformed pattern (%s%s%s%s)",
                    herr[0] & PAT_BAD_ROWPTR ? "bad rowptr " : "",
                    herr[0] & PAT_BAD_COL ? "column out of range " : "",
                    herr[0] & PAT_UNSORTED ? "columns not strictly increasing " : "",
                    herr[0] & PAT_NO_DIAG ? "missing diagonal block" : "");
    }
    TRY(scan_i32(lcnt, lrow, n, scratch, err, st));
    TRY(scan_i32(ucnt, urow, n, scratch, err, st));
    int32_t nl_nu[2];
    TRY(cu(cudaMemcpyAsync(&nl_nu[0], lrow + n, 4, cudaMemcpyDeviceToHost, st), "read nl"));
    TRY(cu(cudaMemcpyAsync(&nl_nu[1], urow + n, 4, cudaMemcpyDeviceToHost, st), "read nu"));
    TRY(cu(cudaStreamSynchronize(st), "sync"));
    int32_t *lcol, *ucol;
    // padded to whole 16-byte groups (+16 bytes): the sweeps copy index ranges
    // rounded out to 16-byte boundaries with bulk asynchronous copies
    TRY(alloc((void **)&lcol, sizeof(int32_t) * ((nl_nu[0] + 3) / 4 * 4 + 4)));
    TRY(alloc((void **)&ucol, sizeof(int32_t) * ((nl_nu[1] + 3) / 4 * 4 + 4)));
    k_pat_cols<<<counted(gb), 256, 0, st>>>(n, d_rowptr, d_colind, diagpos, lrow, urow, lcol, ucol);
    k_pat_pairs<false><<<counted(gb), 256, 0, st>>>(n, d_rowptr, d_colind, diagpos, lrow, urow, pair_cnt,
                                           nullptr, nullptr);
    TRY(cu(cudaGetLastError(), "k_pat_pairs count"));
    TRY(scan_i32(pair_cnt, pair_ptr, nnzb, scratch, err, st));
    int32_t npairs;
    TRY(cu(cudaMemcpyAsync(&npairs, pair_ptr + nnzb, 4, cudaMemcpyDeviceToHost, st), "read npairs"));
    TRY(cu(cudaMemcpyAsync(herr, err, sizeof herr, cudaMemcpyDeviceToHost, st), "read err"));
    TRY(cu(cudaStreamSynchronize(st), "sync"));
    if (herr[0] & (1u << 8)) {
        pattern_free(p);
        return fail(ABILU_EINVAL, "pattern_create: more than 2^31 product pairs");
    }
    int2 *pairs;
    TRY(alloc((void **)&pairs, sizeof(int2) * (npairs > 0 ? npairs : 1)));
    k_pat_pairs<true><<<counted(gb), 256, 0, st>>>(n, d_rowptr, d_colind, diagpos, lrow, urow, nullptr,
                                          pair_ptr, pairs);
    TRY(cu(cudaGetLastError(), "k_pat_pairs fill"));
    // work list of the build sweeps
    int32_t *wcnt = lcnt, *wptr;  // lcnt is free again: reuse it for the counts
    TRY(alloc((void **)&wptr, sizeof(int32_t) * (n + 1)));
    k_pat_work<false><<<counted(gb), 256, 0, st>>>(n, d_rowptr, d_colind, diagpos, lrow, urow,
                                                   pair_ptr, wcnt, nullptr, nullptr);
    TRY(cu(cudaGetLastError(), "k_pat_work count"));
    TRY(scan_i32(wcnt, wptr, n, scratch, err, st));
    int32_t nwork;
    TRY(cu(cudaMemcpyAsync(&nwork, wptr + n, 4, cudaMemcpyDeviceToHost, st), "read nwork"));
    TRY(cu(cudaStreamSynchronize(st), "sync"));
    int4 *work;
    TRY(alloc((void **)&work, sizeof(int4) * (nwork > 0 ? nwork : 1)));
    k_pat_work<true><<<counted(gb), 256, 0, st>>>(n, d_rowptr, d_colind, diagpos, lrow, urow,
                                                  pair_ptr, nullptr, wptr, work);
    TRY(cu(cudaGetLastError(), "k_pat_work fill"));
    {
        const int chunks = (nwork + WORK_CHUNK - 1) / WORK_CHUNK;
        if (chunks > 0) {
            k_pat_work_sort<<<counted((chunks + 127) / 128), 128, 0, st>>>(nwork, WORK_CHUNK, work);
            TRY(cu(cudaGetLastError(), "k_pat_work_sort"));
        }
    }
    int32_t *wpos;
    WorkItem *items;
    TRY(alloc((void **)&wpos, sizeof(int32_t) * nnzb));
    TRY(alloc((void **)&items, sizeof(WorkItem) * (nwork > 0 ? nwork : 1)));
    TRY(cu(cudaMemsetAsync(wpos, 0xFF, sizeof(int32_t) * nnzb, st), "memset wpos"));
    if (nwork > 0) {
        k_pat_work_items<<<counted((nwork + 255) / 256), 256, 0, st>>>(nwork, work, pair_ptr, pairs,
                                                                       wpos, items);
        TRY(cu(cudaGetLastError(), "k_pat_work_items"));
    }
    TRY(cu(cudaStreamSynchronize(st), "sync"));
#undef TRY
    p->v.n = n;
    p->v.nnzb = nnzb;
    p->v.nl = nl_nu[0];
    p->v.nu = nl_nu[1];
    p->v.npairs = npairs;
    p->v.rowptr = d_rowptr;
    p->v.colind = d_colind;
    p->v.diagpos = diagpos;
    p->v.lrow = lrow;
    p->v.urow = urow;
    p->v.lcol = lcol;
    p->v.ucol = ucol;
    p->v.pair_ptr = pair_ptr;
    p->v.pairs = pairs;
    p->v.nwork = nwork;
    p->v.work = items;
    p->v.wpos = wpos;
    p->max_row = (int)herr[2];
    *out = p;
    return ABILU_OK;
}

extern "C" abilu_status abilu_pattern_arrays(abilu_pattern p, int32_t *rowptr, int32_t *colind,
                                             abilu_stream stream) {
    if (!p) return fail(ABILU_EINVAL, "pattern_arrays: NULL pattern");
    cudaStream_t st = S(stream);
    if (rowptr)
        ABILU_CUDA(cudaMemcpyAsync(rowptr, p->v.rowptr, sizeof(int32_t) * ((size_t)p->v.n + 1),
                                   cudaMemcpyDeviceToDevice, st));
    if (colind)
        ABILU_CUDA(cudaMemcpyAsync(colind, p->v.colind, sizeof(int32_t) * (size_t)p->v.nnzb,
                                   cudaMemcpyDeviceToDevice, st));
    return ABILU_OK;
}

extern "C" abilu_status abilu_pattern_counts(abilu_pattern p, int64_t *out) {
    if (!p || !out) return fail(ABILU_EINVAL, "pattern_counts: NULL argument");
    out[0] = p->v.n;
    out[1] = p->v.nnzb;
    out[2] = p->v.nl;
    out[3] = p->v.nu;
    out[4] = p->v.npairs;
    out[5] = p->max_row;
    out[6] = p->v.nwork;
    return ABILU_OK;
}
