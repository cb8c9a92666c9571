// The bulk L2 prefetch (cp.async.bulk.prefetch.L2, the untiled TMA path) that
// the volume-term kernels issue for the element one wave ahead, and a bounded
// mbarrier wait, in inline PTX for sm_100-class GPUs.  Rule of the untiled
// bulk operations: address 16-byte aligned, size a multiple of 16 bytes.
//
// Every device wait is bounded: bulk_wait() gives up after a time limit (and
// a fixed number of polls) and returns false, so a kernel never spins forever.
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

// Bulk prefetch of [src, src + bytes) from global memory into L2 (no
// completion to wait for; src 16-byte aligned, bytes a multiple of 16).
__device__ __forceinline__ void prefetch_l2(const void *src_gmem, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src_gmem), "r"(bytes)
                 : "memory");
}

// One poll of phase `parity` of `bar`; the thread may be suspended for up to
// about hint_ns while the phase is incomplete.
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity, uint32_t hint_ns = 1000) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}" : "=r"(done) : "r"(smem_addr(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of `bar` to complete; false once limit_ns of
// global time have passed (or after 2^22 polls, a bound that holds even if
// the timer stood still).  Legitimate waits take microseconds; the default
// limit of one second is far above them and far below a hang.
__device__ __forceinline__ bool bulk_wait(uint64_t *bar, uint32_t parity,
                                          uint64_t limit_ns = 1000000000ull) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0; it < (1u << 22); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
    return false;
}

}  // namespace numa
