// Mixed-precision element volume term at N = 7 (Nq = 8) with the D sums as
// TF32 split products on the tensor cores (numa_vol_set_sweep with
// NUMA_SWEEP_TENSOR_TF32 on a NUMA_MIXED handle).
//
// The operation of vol_mixed.cu (Sec. 2, Eq. (2); FP32 perturbation state, p'
// from Theta' without cancellation), with the three D sums of every field
// computed as in the batch's tensor-core tile (batch_tile_tc.cuh): the fluxes
// of an element as heads and tails in shared memory (canonical K-major
// layout, one row per line, conflict-free point accesses), two MMAs per block
// of 128 lines into tensor memory, the two accumulator halves added back into
// the flux slots, and the three sums of a point combined.
//
// A persistent grid of two 512-thread CTAs per SM, one element per CTA at a
// time, 128 TMEM columns per CTA (allocated once); thread 0 prefetches to L2
// the arrays of the element the CTA takes next.  Each element waits for its
// MMAs with the library's bounded wait; a wait that runs out sets bit 0 of the
// handle's status word (NUMA_ETIMEOUT from numa_vol_status) and the CTA stops.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "batch_tile_tc.cuh"
#include "bulk_copy.cuh"
#include "eos.cuh"
#include "numa_internal.h"
#include "tcgen05.cuh"

namespace numa {

namespace {

constexpr uint32_t kSingleTcCols = 128;

__global__ void __launch_bounds__(512, 2)
vol_rhs_mixed_tc_kernel(MixedGeometry geo, MixedParams P, const float *__restrict__ q,
                        float *__restrict__ rhs, int64_t M, int64_t e0, int64_t e_end, int *err) {
    using S = TcShape<8>;
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t s_tmem;
    const int l = threadIdx.x, w = l >> 5, lane = l & 31;
    if (w == 0) tc::tmem_alloc(&s_tmem, kSingleTcCols);
    if (l == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = s_tmem;
    tc_prepare_operands<8>(sm);
    tc::fence_proxy_async_smem();
    __syncthreads();

    int el, i, j, k;
    tc_thread_point<8>(l, el, i, j, k);
    const int p = i + 8 * j + 64 * k;
    int off[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) off[d] = d * 5 * S::BLK_BYTES + tc_point_offset<8>(d, el, i, j, k);
    const uint32_t lane_base = tmem + ((uint32_t)(32 * (w & 3)) << 16);
    unsigned char *Ah = sm;
    uint32_t phase = 0;
    bool ok = true;

    for (int64_t e = e0 + blockIdx.x; e < e_end; e += gridDim.x) {
        const int64_t node = e * 512 + p;
        if (l == 0 && e + gridDim.x < e_end) {
            // the arrays of this CTA's next element toward L2 (2 KB slabs)
            const int64_t nx = (e + gridDim.x) * 512;
            for (int b = 0; b < kFields; ++b) prefetch_l2(q + b * M + nx, 2048);
            for (int a = 0; a < 9; ++a) prefetch_l2(geo.g[a] + nx, 2048);
            prefetch_l2(geo.Jinv + nx, 2048);
            prefetch_l2(geo.rho_ref + nx, 2048);
            prefetch_l2(geo.theta_ref + nx, 2048);
        }
        // No barrier after the previous element's phase 3: it read, and this
        // phase 1 writes, only the thread's own point's slots of A (the
        // element's MMAs had completed before its readback).
        // ---- phase 1: p', fluxes, heads and tails into A -----------------
        const float rp = q[node];
        const float jinv = geo.Jinv[node];
        {
            const float U[3] = {q[M + node], q[2 * M + node], q[3 * M + node]};
            const float thp = q[4 * M + node];
            const float th0 = geo.theta_ref[node];
            const float rho = geo.rho_ref[node] + rp;
            const float Th = th0 + thp;
            const float pp = pressure_perturbation_f32(thp, th0, P);
            const float rinv = __frcp_rn(rho);   // correctly rounded, as 1.0f / rho
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const float g1 = geo.g[3 * d][node], g2 = geo.g[3 * d + 1][node],
                            g3 = geo.g[3 * d + 2][node];
                const float v = fmaf(g3, U[2], fmaf(g2, U[1], g1 * U[0]));
                const float u = v * rinv;
                const float F[kFields] = {v, fmaf(U[0], u, g1 * pp), fmaf(U[1], u, g2 * pp),
                                          fmaf(U[2], u, g3 * pp), Th * u};
#pragma unroll
                for (int b = 0; b < kFields; ++b) {
                    unsigned char *a = Ah + off[d] + b * S::BLK_BYTES;
                    *reinterpret_cast<float *>(a) = F[b];
                    *reinterpret_cast<float *>(a + S::REGION) = F[b] - tf32_head_dev(F[b]);
                }
            }
        }
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        // ---- phase 2: the split products on the tensor core --------------
        if (l == 0) {
            tc::fence_after_sync();
            constexpr uint32_t idesc = tc::idesc_tf32(128, S::NN);
            const uint32_t ah = smem_addr(sm), al = ah + S::REGION;
            const uint32_t b1 = ah + 2 * S::REGION, b2 = b1 + S::BBYTES;
#pragma unroll 1
            for (int m = 0; m < S::NBLK; ++m) {
                const uint32_t ao = m * 2048;
                tc::mma_tf32(tmem + m * S::NN, tc::smem_desc(ah + ao, S::LBO_A, 128),
                             tc::smem_desc(b1, S::LBO_B, 128), idesc, 0);
                tc::mma_tf32(tmem + m * S::NN, tc::smem_desc(al + ao, S::LBO_A, 128),
                             tc::smem_desc(b2, S::LBO_B, 128), idesc, 1);
            }
            tc::mma_commit(&bar);
        }
        ok = bulk_wait(&bar, phase);
        if (__syncthreads_or(!ok)) {
            ok = false;
            break;
        }
        phase ^= 1u;
        tc::fence_after_sync();
        // ---- readback: the two accumulator halves into the flux slots -----
#pragma unroll 1
        for (int m = w >> 2; m < S::NBLK; m += 4) {
            uint32_t hv[8], lv[8];
            tc::tmem_ld8(lane_base + m * S::NN, hv);
            tc::tmem_ld8(lane_base + m * S::NN + S::H, lv);
            tc::tmem_ld_wait8x2(hv, lv);
            tc_store_row<8>(Ah, m * 128 + 32 * (w & 3) + lane, 0, hv, lv);
        }
        tc::fence_before_sync();
        __syncthreads();
        // ---- phase 3: combine, scale, gravity, store ----------------------
#pragma unroll
        for (int b = 0; b < kFields; ++b) {
            const float R = *reinterpret_cast<const float *>(Ah + off[0] + b * S::BLK_BYTES) +
                            *reinterpret_cast<const float *>(Ah + off[1] + b * S::BLK_BYTES) +
                            *reinterpret_cast<const float *>(Ah + off[2] + b * S::BLK_BYTES);
            float v = -jinv * R;
            if (b == 3) v = fmaf(-rp, P.grav, v);
            rhs[b * M + node] = v;
        }
    }
    if (!ok) {
        if (l == 0) atomicOr(err, 1);
        bulk_wait(&bar, phase);   // the MMAs in flight, bounded again
    }
    tc::fence_before_sync();
    __syncthreads();
    if (w == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, kSingleTcCols);
    }
}

}  // namespace

cudaError_t prepare_vol_rhs_mixed_tc() {
    // once per device: this unit's D heads and tails, the shared-memory opt-in
    static std::mutex mu;
    static bool ready[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (ready[dev]) return cudaSuccess;
    e = upload_tc_tables();
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(vol_rhs_mixed_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 TcShape<8>::SMEM);
    if (e == cudaSuccess) ready[dev] = true;
    return e;
}

cudaError_t launch_vol_rhs_mixed_tc(ElemRange r, const MixedGeometry &geo, const MixedParams &P,
                                    const float *q, float *rhs, int num_sms, int *err,
                                    cudaStream_t s) {
    if (r.count <= 0) return cudaSuccess;
    const int64_t grid = std::min<int64_t>((int64_t)num_sms * 2, r.count);
    vol_rhs_mixed_tc_kernel<<<(unsigned)grid, 512, TcShape<8>::SMEM, s>>>(
        geo, P, q, rhs, r.M, r.e0, r.e0 + r.count, err);
    return cudaGetLastError();
}

}  // namespace numa
