// Bulk asynchronous copies from global to shared memory (the TMA engine's untiled form, cp.async.bulk) with
// mbarrier completion, for sm_103a, in inline PTX.  A copy moves a contiguous run of bytes without passing
// through registers, so a few threads can keep many kilobytes in flight for a whole CTA.
//
// Rules the callers keep: both addresses 16-byte aligned and the size a multiple of 16 bytes; the expected
// byte count of a phase is registered (arrive.expect_tx) before any of its copies is issued; a buffer that
// generic loads have read is handed back to the copy engine only after those loads are ordered before the
// copy (a barrier among the reading threads, then a proxy fence by the issuing thread).
#pragma once

#include <stdint.h>

namespace scbb {

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// one-time initialisation of a barrier expecting `count` arrivals per phase; made visible to the copy
// engine by the release fence
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// one arrival that also adds `bytes` to the phase's expected transaction count
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// generic-proxy accesses of shared memory before this point are ordered before later async-proxy accesses
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// bytes from global src to shared dst; completion is counted on bar
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// true if the phase with the given parity has completed (does not wait)
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// true once the phase has completed; may suspend the thread for a short, hardware-defined time first
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Waits for the phase with the given parity, polling at most `limit` times (each poll may suspend the thread
// for a short, hardware-defined time); with a limit of 0 it gives up unless the phase had completed at the
// first, non-waiting test.  Returns false when it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit) {
    if (mbar_test(bar, parity)) return true;
    for (long long k = 0; k < limit; k++) {
        if (mbar_try(bar, parity)) return true;
        if ((k & 63) == 63) __nanosleep(128);
    }
    return false;
}

}  // namespace scbb
