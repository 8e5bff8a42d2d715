// Device helpers shared by the tcgen05 kernels: shared-memory matrix descriptors, mbarrier waits (all bounded),
// tcgen05 commits, TMEM loads and the fences between the generic proxy, the async proxy and the tensor cores.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "sse_internal.h"

namespace sse {

constexpr uint32_t kWaitIters = 1u << 22;  // bounded waits (well under a second of polling)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    // tcgen05 shared-memory matrix descriptor: K-major, no swizzle, base offset 0
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;  // stride between 16-B chunks along K
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;  // stride between 8-row groups along M/N
    d |= (uint64_t)1 << 46;                      // descriptor version
    return d;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(phase)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}


// power-of-two exponent e with 2^e <= m < 2^(e+1); 0 for m == 0
__device__ __forceinline__ int floor_log2(float m) {
    if (!(m > 0.f) || !isfinite(m)) return 0;
    int ex;
    frexpf(m, &ex);
    return ex - 1;
}


__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void named_bar(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// Bounded wait; after any wait of the CTA has given up, waits return at once (results are then
// discarded: the host reports SSE_ERR_TIMEOUT), so every role still runs its loops to the end.
__device__ __forceinline__ void wait_or_abort(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                              unsigned* status, uint32_t limit = kWaitIters) {
    if (*abort_flag) return;
    for (uint32_t it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return;
    *abort_flag = 1;
    atomicOr(status, DEV_TIMEOUT);
}

// Bounded wait that ignores the abort flag: at the end of the kernel, for the CTA's own TMA loads and MMAs still in
// flight, so that none of them writes shared memory or TMEM after the CTA has released it.
__device__ __forceinline__ void drain_wait(uint32_t bar, uint32_t parity, unsigned* status) {
    for (uint32_t it = 0; it < kWaitIters; ++it)
        if (mbar_try_wait(bar, parity)) return;
    atomicOr(status, DEV_TIMEOUT);
}

}  // namespace sse
