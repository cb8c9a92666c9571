// Failure-detection self-test of the bounded device wait.
//
// A device-side wait of the library (bulk_wait, on an mbarrier) gives up
// after a time limit; the kernel then sets the handle's status word, which
// numa_vol_status reports as NUMA_ETIMEOUT.  numa_vol_selftest_wait makes
// such a wait run out on purpose, without any fault: one thread waits on a
// barrier that nothing arrives at and no copy targets, so nothing is left in
// flight when it gives up.  The context stays usable.
#include <cuda_runtime.h>

#include <cstdint>

#include "bulk_copy.cuh"
#include "numa_internal.h"
#include "numa_vol.h"

namespace numa {

namespace {

__global__ void selftest_wait_kernel(int *err, uint64_t limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);   // one arrival expected, and none will come
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !bulk_wait(&bar, 0, limit_ns)) atomicOr(err, 1);
}

}  // namespace

}  // namespace numa

extern "C" int numa_vol_selftest_wait(numa_vol *h, uint32_t limit_us, void *stream) {
    if (!h || limit_us == 0 || limit_us > 1000000u) return NUMA_EINVAL;
    numa::selftest_wait_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(
        h->d_err, static_cast<uint64_t>(limit_us) * 1000ull);
    return cudaGetLastError() == cudaSuccess ? NUMA_OK : NUMA_ECUDA;
}
