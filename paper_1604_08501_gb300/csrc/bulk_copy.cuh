// Bulk asynchronous copies (cp.async.bulk, the untiled TMA path) and
// mbarriers for staging element slabs in shared memory, in inline PTX for
// sm_100-class GPUs.
//
// Every wait is bounded: bulk_wait() gives up after a fixed number of polls
// and returns false, so a kernel never spins forever.  Rules of the untiled
// bulk copy: both addresses 16-byte aligned, size a multiple of 16 bytes.
#pragma once

#include <cstdint>

namespace numa {

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

// Make barrier initialisation and prior generic-proxy shared accesses visible
// to the async proxy (the bulk-copy engine).
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One arrival that also announces tx_bytes of incoming bulk-copy data.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t tx_bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(tx_bytes)
                 : "memory");
}

// Global -> shared bulk copy completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst_smem, const void *src_gmem, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}" : "=r"(done) : "r"(smem_addr(bar)), "r"(parity) : "memory");
    return done != 0;
}

// Wait for phase `parity` of `bar` to complete; false after max_polls polls.
// Each try_wait may suspend the thread for a hardware-chosen time, so the
// bound is far above any legitimate wait (microseconds) and far below a hang.
__device__ __forceinline__ bool bulk_wait(uint64_t *bar, uint32_t parity,
                                          uint32_t max_polls = 1u << 22) {
    for (uint32_t it = 0; it < max_polls; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

}  // namespace numa
