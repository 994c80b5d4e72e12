// Shared-memory staging with the Tensor Memory Accelerator's bulk copies
// (cp.async.bulk, global -> shared, completion counted on an mbarrier) for
// the producer/consumer pipelines of the in-place sweeps.
//
// Rules kept by every caller: global source and shared destination 16-byte
// aligned, sizes multiples of 16 bytes, at most 2^20 - 1 bytes per barrier
// phase.  Every wait is bounded: after `limit` polls (the caller's spin
// limit, PIPE_WAIT_LIMIT by default) it counts a timeout in a device error
// word and returns false, and the caller leaves its loop, so no kernel can
// hang on a barrier.  A CTA that gives up still waits, again bounded, for the
// bulk copies it has issued before it retires (see mbar_drain), so no copy
// lands in shared memory that the CTA no longer owns.
#pragma once
#include <stdint.h>

namespace abilu {

constexpr unsigned long long PIPE_WAIT_LIMIT = 1ull << 24;

// the spin limit a kernel uses: the caller's, or the default when 0
__host__ __device__ __forceinline__ unsigned long long spin_limit_or_default(unsigned long long l) {
    return l ? l : PIPE_WAIT_LIMIT;
}

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

// makes initialised barriers visible to the async proxy (bulk copies)
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// arrive and add `bytes` to the transaction count the phase waits for
__device__ __forceinline__ void mbar_arrive_tx(uint64_t *bar, unsigned bytes) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
            smem_u32(bar)),
        "r"(bytes)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// wait for the phase with the given parity to complete; false = timed out
// after `limit` polls (counted in *err)
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity,
                                          unsigned long long *err, unsigned long long limit) {
    for (unsigned long long it = 0; it < limit; it++)
        if (mbar_try_wait(bar, parity)) return true;
    atomicAdd(err, 1ull);
    return false;
}

// Before a producer retires: wait for the last phase it armed on each of its
// `nstages` full barriers (armed[s] = phases armed on stage s so far), i.e.
// for every bulk copy it issued, since the phase before the last one was
// already consumed when the last one was armed.  Bounded like mbar_wait.
__device__ __forceinline__ void mbar_drain(uint64_t *full, const int *armed, int nstages,
                                           unsigned long long *err, unsigned long long limit) {
    for (int s = 0; s < nstages; s++)
        if (armed[s] > 0) mbar_wait(&full[s], (unsigned)(armed[s] - 1) & 1u, err, limit);
}

// bulk copy of `bytes` from global memory into shared memory; completion is
// counted on `bar` (which must expect the bytes)
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// orders this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (bulk copy) writes to the same memory
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

}  // namespace abilu
