// C ABI entry points: factor handles and their device memory, build, apply,
// SpMV, export.  Pattern analysis lives in pattern.cu, FGMRES in fgmres.cu.
#include <string.h>

#include <atomic>

#include "common.cuh"

namespace abilu {

abilu_status build_dispatch(abilu_factors f, const double *A, int nsweeps, abilu_mode mode,
                            abilu_init init, cudaStream_t st);
abilu_status apply_dispatch(abilu_factors f, const double *r, const float *r32, double *z,
                            int nl, int nu, abilu_mode mode, cudaStream_t st, Skip skip);
abilu_status export_dispatch(abilu_factors f, double *X, double *Dinv, cudaStream_t st);
abilu_status spmv_launch(const PatternView &P, const double *A, double alpha, const double *x,
                         double beta, double *y, cudaStream_t st, Skip skip);
size_t solve_state_bytes();
size_t host_status_bytes();
int max_restart();

constexpr int MAXM_PARTIAL_STRIDE = 66;  // MAXM + 2 doubles per CTA

// (cached once; the caches of launch shapes are atomics: different handles
// may be driven from different host threads)
int red_ctas() {
    static std::atomic<int> cached{0};
    int v = cached.load(std::memory_order_relaxed);
    if (!v) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        v = 4 * (sms > 0 ? sms : 1);
        cached.store(v, std::memory_order_relaxed);
    }
    return v;
}

static inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

abilu_status ensure_krylov(abilu_factors f, int m) {
    if (f->krylov && f->krylov_m >= m) return ABILU_OK;
    if (f->krylov) cudaFree(f->krylov);
    f->krylov = nullptr;
    f->krylov_m = 0;
    const size_t nv = (size_t)f->p->v.n * BS;
    // V: m+1 vectors, Z: m vectors, w: 1 vector
    ABILU_CUDA(cudaMalloc(&f->krylov, sizeof(double) * nv * (2 * (size_t)m + 2)));
    f->krylov_m = m;
    return ABILU_OK;
}

}  // namespace abilu

using namespace abilu;

static void factors_free(abilu_factors f) {
    if (!f) return;
    for (void *e : f->ev)
        if (e) cudaEventDestroy(static_cast<cudaEvent_t>(e));
    for (void *e : f->tev)
        if (e) cudaEventDestroy(static_cast<cudaEvent_t>(e));
    if (f->krylov) cudaFree(f->krylov);
    if (f->mem) cudaFree(f->mem);
    if (f->host_status) cudaFreeHost(f->host_status);
    delete f;
}

extern "C" void abilu_factors_destroy(abilu_factors f) { factors_free(f); }

extern "C" abilu_status abilu_factors_create_scalar(abilu_pattern p, abilu_dtype dtype,
                                                    abilu_factors *out) {
    if (!out) return fail(ABILU_EINVAL, "factors_create_scalar: out is NULL");
    *out = nullptr;
    if (dtype != ABILU_F64) return fail(ABILU_EINVAL, "factors_create_scalar: FP64 factors only");
    abilu_status s = abilu_factors_create(p, dtype, out);
    if (s == ABILU_OK) (*out)->scalar = 1;
    return s;
}

extern "C" abilu_status abilu_factors_create(abilu_pattern p, abilu_dtype dtype, abilu_factors *out) {
    if (!p || !out) return fail(ABILU_EINVAL, "factors_create: NULL argument");
    *out = nullptr;
    size_t esz;
    switch (dtype) {
    case ABILU_F64: esz = 8; break;
    case ABILU_F32: esz = 4; break;
    case ABILU_BF16: esz = 2; break;
    default: return fail(ABILU_EINVAL, "factors_create: bad dtype %d", (int)dtype);
    }
    const PatternView &v = p->v;
    const size_t vt = dtype == ABILU_F64 ? 8 : 4;
    auto rnd = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t bl = rnd(esz * BB * (size_t)(v.nl > 0 ? v.nl : 1));
    const size_t bu = rnd(esz * BB * (size_t)(v.nu > 0 ? v.nu : 1));
    const size_t bd = rnd(esz * BB * (size_t)v.n);
    const size_t bv = rnd(vt * BS * (size_t)v.n);
    const size_t bc = rnd(sizeof(unsigned long long) * 8);   // counters, tickets, error word
    const size_t bs = rnd(solve_state_bytes());
    const size_t bp = rnd(sizeof(double) * MAXM_PARTIAL_STRIDE * (size_t)red_ctas());
    const bool narrow = dtype != ABILU_F64;
    const size_t ba = narrow ? rnd(sizeof(float) * BB * (size_t)v.nnzb) : 0;
    const size_t br = narrow ? rnd(sizeof(float) * BS * (size_t)v.n) : 0;
    const size_t bus = dtype == ABILU_F32 ? bu : 0;   // Dinv-scaled upper blocks
    const size_t bcd = rnd(sizeof(int) * ((size_t)(v.nwork + 31) / 32 + 1));
    const size_t total = 2 * bl + 2 * bu + 3 * bd + 4 * bv + bc + bs + bp + ba + br + bus + bcd;
    abilu_factors f = new abilu_factors_s();
    memset(f, 0, sizeof *f);
    f->p = p;
    f->dtype = dtype;
    f->esz = esz;
    cudaError_t e = cudaMalloc(&f->mem, total);
    if (e != cudaSuccess) { factors_free(f); return cuda_fail(e, "factors_create: cudaMalloc"); }
    char *m = reinterpret_cast<char *>(f->mem);
    f->L[0] = m; m += bl;
    f->L[1] = m; m += bl;
    f->U[0] = m; m += bu;
    f->U[1] = m; m += bu;
    f->D[0] = m; m += bd;
    f->D[1] = m; m += bd;
    f->Udiag = m; m += bd;
    f->y[0] = m; m += bv;
    f->y[1] = m; m += bv;
    f->x[0] = m; m += bv;
    f->x[1] = m; m += bv;
    f->ctr = reinterpret_cast<unsigned long long *>(m); m += bc;
    f->scal = reinterpret_cast<double *>(m); m += bs;
    f->partials = reinterpret_cast<double *>(m); m += bp;
    f->A32 = narrow ? m : nullptr; m += ba;
    f->r32 = narrow ? m : nullptr; m += br;
    f->Us = bus ? m : nullptr; m += bus;
    f->chunk_done = reinterpret_cast<int *>(m); m += bcd;
    e = cudaMemset(f->mem, 0, total);
    if (e == cudaSuccess) e = cudaHostAlloc(&f->host_status, host_status_bytes(), cudaHostAllocMapped);
    if (e != cudaSuccess) { factors_free(f); return cuda_fail(e, "factors_create"); }
    memset(f->host_status, 0, host_status_bytes());
    f->cur = 0;
    *out = f;
    return ABILU_OK;
}

extern "C" abilu_status abilu_build(abilu_factors f, const double *A, int nsweeps, abilu_mode mode,
                                    abilu_init init, abilu_stream stream) {
    if (!f || !A) return fail(ABILU_EINVAL, "build: NULL argument");
    if (!aligned16(A)) return fail(ABILU_EINVAL, "build: A_vals must be 16-byte aligned");
    if (nsweeps < 0) return fail(ABILU_EINVAL, "build: nsweeps < 0");
    if (mode != ABILU_SYNC && mode != ABILU_ASYNC) return fail(ABILU_EINVAL, "build: bad mode");
    if (init != ABILU_INIT_FROM_A && init != ABILU_INIT_FROM_PREVIOUS)
        return fail(ABILU_EINVAL, "build: bad init");
    return build_dispatch(f, A, nsweeps, mode, init, S(stream));
}

extern "C" abilu_status abilu_factors_timing(abilu_factors f, int enable) {
    if (!f) return fail(ABILU_EINVAL, "factors_timing: NULL factors");
    if (enable) {
        for (int k = 0; k < 2; k++)
            if (!f->tev[k]) ABILU_CUDA(cudaEventCreate(reinterpret_cast<cudaEvent_t *>(&f->tev[k])));
    }
    f->timing = enable != 0;
    f->timed = 0;
    return ABILU_OK;
}

extern "C" abilu_status abilu_factors_sweep_time(abilu_factors f, float *ms) {
    if (!f || !ms) return fail(ABILU_EINVAL, "factors_sweep_time: NULL argument");
    if (!f->timed) return fail(ABILU_EINVAL, "factors_sweep_time: no timed build since timing was enabled");
    cudaEvent_t e0 = static_cast<cudaEvent_t>(f->tev[0]), e1 = static_cast<cudaEvent_t>(f->tev[1]);
    ABILU_CUDA(cudaEventSynchronize(e1));
    ABILU_CUDA(cudaEventElapsedTime(ms, e0, e1));
    return ABILU_OK;
}

extern "C" abilu_status abilu_apply(abilu_factors f, const double *r, double *z, int nl, int nu,
                                    abilu_mode mode, abilu_stream stream) {
    if (!f || !r || !z) return fail(ABILU_EINVAL, "apply: NULL argument");
    if (r == z) return fail(ABILU_EINVAL, "apply: r and z must be distinct");
    if (!aligned16(r) || !aligned16(z)) return fail(ABILU_EINVAL, "apply: vectors must be 16-byte aligned");
    if (nl < 0 || nu < 0) return fail(ABILU_EINVAL, "apply: negative sweep count");
    if (mode != ABILU_SYNC && mode != ABILU_ASYNC) return fail(ABILU_EINVAL, "apply: bad mode");
    return apply_dispatch(f, r, nullptr, z, nl, nu, mode, S(stream), Skip{});
}

extern "C" abilu_status bsr_spmv(abilu_pattern p, const double *A, double alpha, const double *x,
                                 double beta, double *y, abilu_stream stream) {
    if (!p || !A || !x || !y) return fail(ABILU_EINVAL, "spmv: NULL argument");
    if (x == y) return fail(ABILU_EINVAL, "spmv: x and y must be distinct");
    if (!aligned16(A) || !aligned16(x) || !aligned16(y))
        return fail(ABILU_EINVAL, "spmv: pointers must be 16-byte aligned");
    return spmv_launch(p->v, A, alpha, x, beta, y, S(stream), Skip{});
}

extern "C" abilu_status abilu_factors_export(abilu_factors f, double *X, double *Dinv,
                                             abilu_stream stream) {
    if (!f) return fail(ABILU_EINVAL, "export: NULL factors");
    if ((X && !aligned16(X)) || (Dinv && !aligned16(Dinv)))
        return fail(ABILU_EINVAL, "export: pointers must be 16-byte aligned");
    if (!X && !Dinv) return ABILU_OK;
    return export_dispatch(f, X, Dinv, S(stream));
}

extern "C" abilu_status abilu_factors_status(abilu_factors f, int64_t *singular_blocks,
                                             abilu_stream stream) {
    if (!f || !singular_blocks) return fail(ABILU_EINVAL, "factors_status: NULL argument");
    unsigned long long cv[5] = {0, 0, 0, 0, 0};
    ABILU_CUDA(cudaMemcpyAsync(cv, f->ctr, sizeof cv, cudaMemcpyDeviceToHost, S(stream)));
    ABILU_CUDA(cudaStreamSynchronize(S(stream)));
    ABILU_CUDA(cudaMemsetAsync(f->ctr, 0, sizeof cv[0], S(stream)));
    *singular_blocks = (int64_t)cv[0];
    if (cv[4]) {  // a staged sweep's bounded wait ran out since the last check
        ABILU_CUDA(cudaMemsetAsync(f->ctr + 4, 0, sizeof cv[4], S(stream)));
        return fail(ABILU_ETIMEOUT, "factors_status: %llu pipeline waits timed out", cv[4]);
    }
    return ABILU_OK;
}

extern "C" abilu_status abilu_factors_set_spin_limit(abilu_factors f, int64_t limit) {
    if (!f) return fail(ABILU_EINVAL, "factors_set_spin_limit: NULL handle");
    if (limit < 0) return fail(ABILU_EINVAL, "factors_set_spin_limit: limit must be >= 0");
    f->spin_limit = (unsigned long long)limit;
    return ABILU_OK;
}

extern "C" abilu_status abilu_factors_set_build_chunk(abilu_factors f, int32_t blocks) {
    if (!f) return fail(ABILU_EINVAL, "factors_set_build_chunk: NULL handle");
    if (blocks != 0 && (blocks < 32 || blocks > 512 || blocks % 32 != 0))
        return fail(ABILU_EINVAL, "factors_set_build_chunk: blocks must be 0 or a multiple of 32 in 32..512");
    f->build_chunk = blocks;
    return ABILU_OK;
}

extern "C" abilu_status abilu_factors_inject_stall(abilu_factors f, int enable) {
    if (!f) return fail(ABILU_EINVAL, "factors_inject_stall: NULL handle");
    f->stall_flags = enable ? 1 : 0;
    return ABILU_OK;
}

namespace abilu {
__global__ void k_to_f32_int(const double *__restrict__ in, float *__restrict__ out, long long n) {
    const long long st = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += st)
        out[e] = to_f32_int(in[e]);
}
}  // namespace abilu

extern "C" abilu_status abilu_to_f32(const double *in, float *out, int64_t n, abilu_stream stream) {
    if (n < 0 || (n > 0 && (!in || !out))) return fail(ABILU_EINVAL, "to_f32: bad argument");
    if (n == 0) return ABILU_OK;
    const long long blocks = (n + 255) / 256;
    const int grid = (int)(blocks < red_ctas() ? blocks : red_ctas());
    k_to_f32_int<<<counted(grid), 256, 0, S(stream)>>>(in, out, n);
    ABILU_LAUNCH_CHECK("k_to_f32_int");
    return ABILU_OK;
}

namespace abilu {
// one thread per (block, row q): the row of 4 values, plus d on the diagonal
__global__ void k_add_block_diagonal(PatternView P, const double *__restrict__ Ain,
                                     double *Aout, const double *__restrict__ d) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long p = e >> 2;
    const int q = (int)(e & 3);
    if (p >= P.nnzb) return;
    double v[4];
    ld_row(Ain + (size_t)p * BB + q * BS, v);
    // p is a diagonal block iff p == diagpos[row of p]; rows are found from
    // the column: a diagonal block has colind[p] = i and diagpos[i] = p
    const int j = P.colind[p];
    if (P.diagpos[j] == p) v[q] += d[(size_t)j * BS + q];
    st_row(Aout + (size_t)p * BB + q * BS, v);
}
}  // namespace abilu

extern "C" abilu_status abilu_add_block_diagonal(abilu_pattern p, const double *A_in, double *A_out,
                                                 const double *d, abilu_stream stream) {
    if (!p || !A_in || !A_out || !d) return fail(ABILU_EINVAL, "add_block_diagonal: NULL argument");
    const long long threads = (long long)p->v.nnzb * 4;
    k_add_block_diagonal<<<counted((int)((threads + 255) / 256)), 256, 0, S(stream)>>>(p->v, A_in,
                                                                                      A_out, d);
    ABILU_LAUNCH_CHECK("k_add_block_diagonal");
    return ABILU_OK;
}
