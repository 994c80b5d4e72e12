// Internal definitions shared by the CUDA translation units of libabilu.
#pragma once

#include <cuda_runtime.h>
#include <utility>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/abilu.h"

namespace abilu {

constexpr int BS = 4;    // block size b = d + 2 (Sec. 2)
constexpr int BB = 16;   // entries per block

// thread-local error message, set by fail()
abilu_status fail(abilu_status s, const char *fmt, ...);
abilu_status cuda_fail(cudaError_t e, const char *what);

#define ABILU_CUDA(call)                                              \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return ::abilu::cuda_fail(e_, #call);  \
    } while (0)

#define ABILU_LAUNCH_CHECK(what)                                      \
    do {                                                              \
        cudaError_t e_ = cudaGetLastError();                          \
        if (e_ != cudaSuccess) return ::abilu::cuda_fail(e_, what);   \
    } while (0)

inline cudaStream_t S(abilu_stream s) { return reinterpret_cast<cudaStream_t>(s); }

// Host-side count of kernel launches made by the library (every launch site
// wraps its grid size in counted()); read through abilu_kernel_launches().
void note_launch();
void note_launches(long long delta);   // graph replays; captures taken back
unsigned long long launches();
template <typename G> inline G counted(G grid) { note_launch(); return grid; }

// Device view of an analysed pattern.  Positions: "p" indexes A's blocks,
// "lpos" indexes the compact strictly-lower array, "upos" the compact
// strictly-upper array.  Row i's L blocks are lpos lrow[i]..lrow[i+1]-1 (the
// first diagpos[i]-rowptr[i] blocks of row i in A's order), its U blocks are
// upos urow[i]..urow[i+1]-1 (the blocks after the diagonal).
struct PatternView {
    int32_t n, nnzb, nl, nu;
    int64_t npairs;
    const int32_t *rowptr, *colind, *diagpos;
    const int32_t *lrow, *urow, *lcol, *ucol;
    const int32_t *pair_ptr;   // [nnzb+1] product pairs of block p
    const int2 *pairs;         // (lpos of L_ik, upos of U_kj)
    // blocks a build sweep updates, in row-major order: every L and diagonal
    // block and the U blocks with product pairs (the others equal A always).
    // The FP32 copy of A that the sweeps read is stored in this order, so a
    // work item's A row is at its index w; wpos[p] = w (-1: constant block).
    int32_t nwork;
    const struct WorkItem *work;
    const int32_t *wpos;
};

enum : int { WORK_L = 0, WORK_D = 1, WORK_U = 2 };

// One work item of the build sweeps, 32 bytes: everything its loads depend
// on, so a sweep reads the record, its FP32 A row (at the item's index) and
// the rows the pairs name without a further lookup.  kind_np = kind | (number
// of product pairs << 2); pairs t0 .. t0+np-1 of the pair list, the first two
// repeated inline.
struct __align__(16) WorkItem {
    int32_t j, dst, kind_np, t0;
    int2 pr[2];
};
constexpr int WORK_CHUNK = 64;  // work blocks per CTA of the build kernels (<= 64)

}  // namespace abilu

struct abilu_pattern_s {
    abilu::PatternView v;
    int32_t max_row;
    int device;
    void *mem;                 // one allocation holding every array
};

struct abilu_factors_s {
    abilu_pattern p;
    abilu_dtype dtype;
    int scalar;                // 1: scalar ILU(0) (Chow-Patel) factors in the block layout
    size_t esz;                // bytes per stored scalar
    // factor storage; [cur] is the current iterate, [1-cur] the sync target
    void *L[2], *U[2], *D[2];
    void *Udiag;
    void *A32;                 // FP32 copy of A's non-constant blocks (FP32/BF16 factors)
    void *r32;                 // FP32 copy of the apply input (FP32/BF16 factors)
    int *chunk_done;           // per 32-block chunk: completed sweeps (ordered async builds)
    void *Us;                  // Dinv_i U_ij for every strictly upper block (FP32
                               // factors): the matrix of the upper sweeps, formed per build
    int cur;
    // apply work vectors (VT = double for F64, float otherwise)
    void *y[2], *x[2];
    // device counters: [0] singular blocks, [1] build tickets, [2] lower and
    // [3] upper apply tickets, [4] timed-out pipeline waits, [5..7] spare
    unsigned long long *ctr;
    // FGMRES workspace (grown on demand)
    double *krylov;            // V (m+1 vectors) then Z (m vectors)
    int krylov_m;
    double *scal;              // small device scalars (Hessenberg, Givens, ...)
    double *partials;          // per-CTA reduction partials
    void *host_status;         // pinned host mirror of the solve status
    void *ev[2];               // FGMRES look-ahead events (cudaEvent_t), made on first use
    void *tev[2];              // build timing events (cudaEvent_t), made by abilu_factors_timing
    int timing;                // nonzero: builds record tev[0], tev[1] around their sweep kernels
    int timed;                 // a build recorded tev since timing was enabled
    // polls of a bounded device-side wait before it gives up (0: the default,
    // PIPE_WAIT_LIMIT); set for the duration of an FGMRES solve from its options
    unsigned long long spin_limit;
    int stall_flags;           // failure injection: the next ordered async build's chunk
                               // flags start one sweep behind (abilu_factors_inject_stall)
    // per 64-row chunk (device, NULL: the build's init for every row): 1 = the
    // chunk's rows start from A, 0 = from the factors in place (the systems of
    // a server step: new ones from A, continuing ones warm-started)
    const int *chunk_init;
    int build_chunk;           // work blocks per ticket of the asynchronous block build (0: 128)
    void *mem;
};

// ---------------------------------------------------------------- device helpers
namespace abilu {

// Early exit of the row kernels.  `flag`: the whole launch returns when *flag
// is nonzero (an FGMRES cycle that has ended).  `chunk_sys`/`sys_done`: in a
// batch, the 64-row chunk c belongs to system chunk_sys[c], whose rows are
// skipped while sys_done[that system] is nonzero.  The flags are written only
// by earlier kernels of the stream, so they are read with ordinary (L1-cached)
// loads: a volatile load from every warp of a large grid queues on the one L2
// line that holds the flag.
constexpr int SKIP_CHUNK_ROWS = 64;
struct Skip {
    const int *flag;
    const int *chunk_sys;
    const int *sys_done;
};
// A right preconditioner z = M^{-1} v for fgmres_run, applied once per
// Arnoldi step on the solve's stream; its kernels return at once while
// skip.flag is set.  v32 (NULL: none) receives an FP32 copy of each
// normalised v from FGMRES (the input FP32/BF16 factors read).
// The Gram-Schmidt form of FGMRES's Arnoldi step (single-system and batch
// solves).  GS_SINGLE: one classical pass and one reduction, h_{j+1,j} =
// sqrt(||w||^2 - sum_k h_k^2).  That formula assumes an orthonormal basis, and
// a classical Gram-Schmidt basis loses orthogonality as the residual falls:
// in FP64 emulations of the solver (seven systems, 6-14 steps) the formula's
// relative error in h_{j+1,j} was about 1e-17 / (the relative residual
// estimate after the step), and at tolerances of 1e-8 a 96-cell system
// missed convergence inside a 30-step cycle.  Since the estimate stays above
// rtol within a cycle, the form is taken only for rtol >= 1e-7 (error below
// about 1e-10; the workloads' 1e-6 included).  GS_CLASSICAL: one classical
// pass with the explicit norm of the updated w (a second reduction and a
// scaling pass), for tighter tolerances.  GS_CGS2: two classical passes
// (opts->reorth).
enum : int { GS_SINGLE = 0, GS_CLASSICAL = 1, GS_CGS2 = 2 };
constexpr double GS_SINGLE_MIN_RTOL = 1e-7;
inline int gs_form_for(int reorth, double rtol) {
    return reorth ? GS_CGS2 : (rtol >= GS_SINGLE_MIN_RTOL ? GS_SINGLE : GS_CLASSICAL);
}

struct Precond {
    abilu_status (*fn)(void *ctx, const double *v, const float *v32, double *z, cudaStream_t st,
                       Skip skip);
    void *ctx;
    float *v32;
    // optional: a second destination of the FP32 copy (the application's
    // in-place iterate) and two ticket counters to zero, both done by the
    // FGMRES kernel that writes v32, so the application needs no start kernel
    float *y0;
    unsigned long long *tickets;
};

__device__ __forceinline__ bool skip_all(const Skip &s) {
    return s.flag && *s.flag;
}
__device__ __forceinline__ bool skip_chunk(const Skip &s, int chunk) {
    return s.chunk_sys && s.sys_done[s.chunk_sys[chunk]];
}

// FP64 -> FP32, round to nearest even, with integer instructions.  On this GPU
// the hardware conversion runs on the FP64 pipe (about 1/60 of the FP32 rate),
// so conversions at every FP64/FP32 boundary would bound the FP32 kernels.
// Results in the normal FP32 range are formed from the bits (23-bit mantissa
// from the top of the 52-bit one, rounded on the 29 dropped bits); zeros,
// subnormals, overflow, Inf and NaN take the hardware conversion.
__device__ __forceinline__ float to_f32(double d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const int e = (int)((hi >> 20) & 0x7FFu) - 1023 + 127;
    if (e < 1 || e > 253) return __double2float_rn(d);
    const unsigned m23 = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    const unsigned rem = lo & 0x1FFFFFFFu;
    unsigned f = (hi & 0x80000000u) | ((unsigned)e << 23) | m23;
    f += (rem > 0x10000000u) | ((rem == 0x10000000u) & (m23 & 1u));
    return __uint_as_float(f);
}

// to_f32 with every case in integer instructions, for kernels bound by the
// FP64 pipe (the Krylov normalisation): the hardware fallback above is issued
// there, predicated off, for every element and takes FP64-pipe cycles.
// Subnormal results shift the 53-bit significand right and round to nearest
// even (2^23 is the smallest normal); |d| < 2^-150 gives +-0; overflow Inf; NaN
// a quiet NaN with the top payload bits.  (Where the FP64 pipe is idle the
// shorter to_f32 is faster: fewer registers.)
__device__ __forceinline__ float to_f32_int(double d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned sign = hi & 0x80000000u;
    const int ed = (int)((hi >> 20) & 0x7FFu);
    const int e = ed - 1023 + 127;
    const unsigned m23 = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    const unsigned rem = lo & 0x1FFFFFFFu;
    if (e >= 1 && e <= 254) {
        unsigned f = sign | ((unsigned)e << 23) | m23;
        f += (rem > 0x10000000u) | ((rem == 0x10000000u) & (m23 & 1u));
        return __uint_as_float(f);
    }
    if (ed == 0x7FF) return __uint_as_float(sign | 0x7F800000u | ((m23 | rem) ? (0x400000u | m23) : 0u));
    if (e > 254) return __uint_as_float(sign | 0x7F800000u);
    if (e < -23) return __uint_as_float(sign);
    const unsigned long long M = (1ull << 52) | (b & 0xFFFFFFFFFFFFFull);
    const int sh = 926 - ed;  // 30 .. 53
    const unsigned long long half = 1ull << (sh - 1), drop = M & ((1ull << sh) - 1ull);
    unsigned long long q = M >> sh;
    q += (drop > half) | ((drop == half) & (q & 1ull));
    return __uint_as_float(sign | (unsigned)q);
}

// FP32 -> FP64 (exact) with integer instructions; zeros, subnormals, Inf and
// NaN take the hardware conversion.
__device__ __forceinline__ double to_f64(float x) {
    const unsigned u = __float_as_uint(x);
    const unsigned ex = (u >> 23) & 0xFFu;
    if (ex == 0u || ex == 0xFFu) return (double)x;
    const unsigned hi = (u & 0x80000000u) | ((ex + (1023u - 127u)) << 20) | ((u & 0x7FFFFFu) >> 3);
    const unsigned lo = (u & 0x7u) << 29;
    return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ void ld_row(const double *p, double v[4]) {
    double2 a = reinterpret_cast<const double2 *>(p)[0];
    double2 b = reinterpret_cast<const double2 *>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void ld_row(const float *p, double v[4]) {
    float4 a = *reinterpret_cast<const float4 *>(p);
    v[0] = to_f64(a.x); v[1] = to_f64(a.y); v[2] = to_f64(a.z); v[3] = to_f64(a.w);
}
__device__ __forceinline__ void ld_row(const __nv_bfloat16 *p, double v[4]) {
    uint2 u = *reinterpret_cast<const uint2 *>(p);
    float2 a = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&u.x));
    float2 b = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&u.y));
    v[0] = to_f64(a.x); v[1] = to_f64(a.y); v[2] = to_f64(b.x); v[3] = to_f64(b.y);
}
__device__ __forceinline__ void ld_row(const float *p, float v[4]) {
    float4 a = *reinterpret_cast<const float4 *>(p);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}
__device__ __forceinline__ void ld_row(const __nv_bfloat16 *p, float v[4]) {
    uint2 u = *reinterpret_cast<const uint2 *>(p);
    float2 a = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&u.x));
    float2 b = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&u.y));
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void ld_row(const double *p, float v[4]) {
    double w[4];
    ld_row(p, w);
    v[0] = to_f32(w[0]); v[1] = to_f32(w[1]); v[2] = to_f32(w[2]); v[3] = to_f32(w[3]);
}

// volatile (relaxed, uncached-in-L1) loads for data other threads may be
// writing concurrently: the in-place asynchronous sweeps.
__device__ __forceinline__ void ld_row_volatile(const double *p, double v[4]) {
    asm volatile("ld.volatile.global.v2.f64 {%0,%1}, [%2];" : "=d"(v[0]), "=d"(v[1]) : "l"(p));
    asm volatile("ld.volatile.global.v2.f64 {%0,%1}, [%2];" : "=d"(v[2]), "=d"(v[3]) : "l"(p + 2));
}
__device__ __forceinline__ void ld_row_volatile(const float *p, float v[4]) {
    asm volatile("ld.volatile.global.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]) : "l"(p));
}
__device__ __forceinline__ void ld_row_volatile(const float *p, double v[4]) {
    float w[4];
    ld_row_volatile(p, w);
    v[0] = to_f64(w[0]); v[1] = to_f64(w[1]); v[2] = to_f64(w[2]); v[3] = to_f64(w[3]);
}
__device__ __forceinline__ void ld_row_volatile(const __nv_bfloat16 *p, float v[4]) {
    unsigned a, b;
    asm volatile("ld.volatile.global.v2.u32 {%0,%1}, [%2];" : "=r"(a), "=r"(b) : "l"(p));
    float2 x = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&a));
    float2 y = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&b));
    v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
}
__device__ __forceinline__ void ld_row_volatile(const __nv_bfloat16 *p, double v[4]) {
    float w[4];
    ld_row_volatile(p, w);
    v[0] = to_f64(w[0]); v[1] = to_f64(w[1]); v[2] = to_f64(w[2]); v[3] = to_f64(w[3]);
}
__device__ __forceinline__ void ld_row_volatile(const double *p, float v[4]) {
    double w[4];
    ld_row_volatile(p, w);
    v[0] = to_f32(w[0]); v[1] = to_f32(w[1]); v[2] = to_f32(w[2]); v[3] = to_f32(w[3]);
}

template <bool VOL, typename T, typename C>
__device__ __forceinline__ void ld_row_sel(const T *p, C v[4]) {
    if constexpr (VOL) ld_row_volatile(p, v); else ld_row(p, v);
}

// stores: one 4-entry row of a block (or one cell's 4 unknowns) from registers
__device__ __forceinline__ void st_row(double *p, const double v[4]) {
    reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
}
__device__ __forceinline__ void st_row(float *p, const double v[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(to_f32(v[0]), to_f32(v[1]), to_f32(v[2]), to_f32(v[3]));
}
__device__ __forceinline__ void st_row(float *p, const float v[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st_row(__nv_bfloat16 *p, const double v[4]) {
    __nv_bfloat162 a = __floats2bfloat162_rn(to_f32(v[0]), to_f32(v[1]));
    __nv_bfloat162 b = __floats2bfloat162_rn(to_f32(v[2]), to_f32(v[3]));
    uint2 u;
    u.x = *reinterpret_cast<unsigned *>(&a);
    u.y = *reinterpret_cast<unsigned *>(&b);
    *reinterpret_cast<uint2 *>(p) = u;
}
__device__ __forceinline__ void st_row(double *p, const float v[4]) {
    double w[4] = {to_f64(v[0]), to_f64(v[1]), to_f64(v[2]), to_f64(v[3])};
    st_row(p, w);
}
__device__ __forceinline__ void st_row(__nv_bfloat16 *p, const float v[4]) {
    __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]);
    __nv_bfloat162 b = __floats2bfloat162_rn(v[2], v[3]);
    uint2 u;
    u.x = *reinterpret_cast<unsigned *>(&a);
    u.y = *reinterpret_cast<unsigned *>(&b);
    *reinterpret_cast<uint2 *>(p) = u;
}


// Programmatic dependent launch.  The kernels of the solve path are launched
// with programmatic stream serialization: a kernel's CTAs may be scheduled
// while the previous kernel of the stream drains its last wave, so launch
// latency and the tail overlap.  Every such kernel calls pdl_wait() before
// its first global access (griddepcontrol.wait returns once the previous
// grid has completed and its writes are visible; it is a no-op for a normal
// launch), then pdl_trigger() to let the next kernel be scheduled in turn.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*k)(KArgs...), int grid, int block, size_t smem, cudaStream_t st,
                              Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    note_launch();
    return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

// Quad helpers: the 4 threads of an aligned group of 4 lanes cooperate on one
// block row; thread q of the quad owns row q of every 4x4 block.
__device__ __forceinline__ unsigned quad_mask() {
    unsigned lane = threadIdx.x & 31u;
    return 0xFu << (lane & ~3u);
}
template <typename C>
__device__ __forceinline__ C qshfl(C v, int src_q) {
    unsigned lane = threadIdx.x & 31u;
    return __shfl_sync(quad_mask(), v, (int)(lane & ~3u) + src_q);
}

}  // namespace abilu
