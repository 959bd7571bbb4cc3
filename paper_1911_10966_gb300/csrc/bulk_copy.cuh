// Bulk global -> shared copies by the tensor memory accelerator (cp.async.bulk, sm_90 and later),
// completed on a shared-memory mbarrier, with a bounded wait.
//
// Use in a CTA: one thread initialises the barrier (mbar_init) before a __syncthreads(); one thread
// posts the byte count (mbar_expect_tx) and issues the copies (bulk_g2s: 16-byte aligned addresses, a
// multiple of 16 bytes); every thread that reads the data waits for phase 0 (mbar_wait_bounded).
// The wait gives up after kBulkWaitPolls polls of about 0.1 us each (about half a second): the
// caller then records an error code and returns instead of spinning forever.
#pragma once

#include <cstdint>

namespace esdc {

constexpr int kBulkWaitPolls = 1 << 22;
// device status bit recorded when a bounded wait for a bulk copy gave up (esdc_device_status)
constexpr int kStatusBulkWait = 1;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    // make the initialised barrier visible to the asynchronous (copy) proxy
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// arrive on the barrier and add `bytes` to the transaction count its phase waits for
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// bytes from global src to shared dst; completion counted on bar
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// true once the barrier's phase of the given parity has completed
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait for the phase of the given parity, polling at most kBulkWaitPolls times; false if it did not
// complete.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    for (int i = 0; i < kBulkWaitPolls; ++i) {
        if (mbar_test(bar, parity)) return true;
        __nanosleep(64);
    }
    return false;
}

}  // namespace esdc
