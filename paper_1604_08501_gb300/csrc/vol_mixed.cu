// Mixed-precision element volume term (NUMA_MIXED), orders N = 1..7 (N = 8..15:
// vol_fp64_high.cu), with or without passive tracers.
//
// The operation of Sec. 2, Eq. (2) (sign and flux form of the paper's r/s
// subroutines, Sec. 3) on FP32 data:
//   state   (rho', U1, U2, U3, Theta'), the perturbations rho' = rho - rho_ref and
//           Theta' = Theta - Theta_ref, so no significant bits go to the large
//           hydrostatic part;
//   geometry and reference state in FP32 (rounded once at create time);
//   fluxes, sweeps and rhs in FP32.
// p' = p(Theta) - p(Theta_ref) = p_ref ((1 + x)^gamma - 1), x = Theta'/Theta_ref,
// is evaluated from Theta' directly (binomial series for |x| <= 1/64,
// expm1(gamma log1p(x)) beyond), so it has no cancellation and FP32 suffices:
// relative error ~1e-7.  p_ref/Theta_ref = K Theta_ref^(gamma - 1) with
// K = p0^(1 - gamma) R^gamma is recomputed per point instead of being stored,
// which keeps the traffic at the algorithmic 88 bytes per point
// (5 + 9 + 1 + 2 arrays read, 5 written, 4 bytes each).  The kernel is bound by
// HBM bandwidth, and the extra arithmetic is free.
//
// Structure as in vol_fp64.cu: fluxes by point into shared memory, even-odd D
// sweeps by line in place, combination by point; one CTA of Nq^3 threads per
// element, four CTAs of 512 threads per SM at Nq = 8 (32 registers, 35 KB of
// shared memory each).  Thread 0 of each CTA prefetches to L2
// (cp.async.bulk.prefetch.L2) the arrays of the element a quarter of a wave of
// resident CTAs ahead (one CTA per SM at Nq = 8), so that CTA's loads hit L2
// rather than DRAM.  Measured at N = 7 (GDOF/s): no prefetch 72.8, 1/8 of a
// wave 74.2, 1/4 74.7, 3/8 74.7, 1/2 74.2, 3/4 72.4, one wave 69.7, 3/2 55.0,
// two 48.3: a longer distance lets L2 evict the lines before their CTA
// starts.  At N = 7 the prefetch
// replaced a persistent kernel that staged each element's arrays in shared
// memory with cp.async.bulk on an mbarrier: the staging buffer limited that
// kernel to three CTAs per SM, and it ran at 0.271 against 0.254 ms here
// (0.242 ms with the line numbering of dir_slot at Nq = 8).
#include <cuda_runtime.h>

#include "bulk_copy.cuh"
#include "element_sweep.cuh"
#include "eos.cuh"
#include "numa_internal.h"

namespace numa {

namespace {

template <int NQ>
constexpr int mixed_min_ctas() {
    constexpr int n = 2048 / (NQ * NQ * NQ);
    return n < 1 ? 1 : (n > 32 ? 32 : n);
}

// Starts the 17 arrays element e reads toward L2, where an element's slab of
// one array is a whole number of 16-byte units (the bulk prefetch's rule).
template <int NQ>
__device__ __forceinline__ void prefetch_element(const MixedGeometry &geo, const float *q,
                                                 int64_t M, int nf, int64_t e) {
    constexpr uint32_t B = NQ * NQ * NQ * sizeof(float);
    if constexpr (B % 16 == 0) {
        const int64_t off = e * (NQ * NQ * NQ);
        for (int b = 0; b < nf; ++b) prefetch_l2(q + b * M + off, B);
#pragma unroll
        for (int a = 0; a < 9; ++a) prefetch_l2(geo.g[a] + off, B);
        prefetch_l2(geo.Jinv + off, B);
        prefetch_l2(geo.rho_ref + off, B);
        prefetch_l2(geo.theta_ref + off, B);
    }
}

// TRACERS: nf = 5 + tracers fields at run time (tracers Q in FP32 as they are,
// flux Q u_d, no source).  Without tracers nf is 5.
template <int NQ, bool TRACERS>
__global__ void __launch_bounds__(NQ * NQ * NQ, mixed_min_ctas<NQ>())
vol_rhs_mixed_kernel(MixedGeometry geo, MixedParams P, const float *__restrict__ q,
                     float *__restrict__ rhs, int64_t M, int64_t e0, int nf_run, int64_t e_end,
                     int64_t ahead) {
    constexpr int N3 = NQ * NQ * NQ;
    constexpr int NL = NQ * NQ;
    constexpr int EW = block_words<NQ, float>();   // one (direction, field) block
    const int nf = TRACERS ? nf_run : kFields;
    extern __shared__ float sFm[];            // [direction*nf + field][slot]

    const int l = threadIdx.x;
    const int i = l % NQ, j = (l / NQ) % NQ, k = l / (NQ * NQ);
    const int64_t node = (e0 + blockIdx.x) * N3 + l;
    if (l == 0 && e0 + blockIdx.x + ahead < e_end)
        prefetch_element<NQ>(geo, q, M, nf, e0 + blockIdx.x + ahead);

    // ---- phase 1: p', fluxes ----------------------------------------
    const float rp = q[node];
    const float U[3] = {q[M + node], q[2 * M + node], q[3 * M + node]};
    const float thp = q[4 * M + node];
    const float th0 = geo.theta_ref[node];
    const float rho = geo.rho_ref[node] + rp;
    const float Th = th0 + thp;
    const float pp = pressure_perturbation_f32(thp, th0, P);
    const float rinv = __frcp_rn(rho);   // correctly rounded, as 1.0f / rho
    // J^-1 with the other loads (loaded after phase 2 instead: 68.6 against
    // 69.5 GDOF/s at N = 7)
    const float Jinv = geo.Jinv[node];
    float Q[kMaxFields - kFields];
    if constexpr (TRACERS) {
#pragma unroll
        for (int t = 0; t < kMaxFields - kFields; ++t)
            Q[t] = kFields + t < nf ? q[(kFields + t) * M + node] : 0.f;
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float g1 = geo.g[3 * d][node], g2 = geo.g[3 * d + 1][node],
                    g3 = geo.g[3 * d + 2][node];
        const float v = fmaf(g3, U[2], fmaf(g2, U[1], g1 * U[0]));
        const float u = v * rinv;
        float *F = sFm + d * nf * EW + dir_slot<NQ, float>(d, i, j, k);
        F[0 * EW] = v;
        F[1 * EW] = fmaf(U[0], u, g1 * pp);
        F[2 * EW] = fmaf(U[1], u, g2 * pp);
        F[3 * EW] = fmaf(U[2], u, g3 * pp);
        F[4 * EW] = Th * u;
        if constexpr (TRACERS) {
#pragma unroll
            for (int t = 0; t < kMaxFields - kFields; ++t)
                if (kFields + t < nf) F[(kFields + t) * EW] = Q[t] * u;
        }
    }
    __syncthreads();

    // ---- phase 2: even-odd sweeps, one line per task, in place --------
    for (int item = l; item < 3 * nf * NL; item += N3)
        sweep_line<NQ>(sFm + (item / NL) * EW, item % NL, P);
    __syncthreads();

    // ---- phase 3: combine, scale, gravity, store ----------------------
#pragma unroll
    for (int b = 0; b < (TRACERS ? kMaxFields : kFields); ++b) {
        if (TRACERS && b >= nf) break;
        const float R = sFm[(0 * nf + b) * EW + dir_slot<NQ, float>(0, i, j, k)] +
                        sFm[(1 * nf + b) * EW + dir_slot<NQ, float>(1, i, j, k)] +
                        sFm[(2 * nf + b) * EW + dir_slot<NQ, float>(2, i, j, k)];
        float v = -Jinv * R;
        if (b == 3) v = fmaf(-rp, P.grav, v);
        rhs[b * M + node] = v;
    }
}

template <int NQ, bool TRACERS>
cudaError_t launch_kernel(ElemRange r, int nf, const MixedGeometry &geo, const MixedParams &P,
                          const float *q, float *rhs, int num_sms, cudaStream_t s) {
    constexpr int N3 = NQ * NQ * NQ;
    const size_t smem = sizeof(float) * nf * 3 * block_words<NQ, float>();
    cudaError_t e = cudaFuncSetAttribute(vol_rhs_mixed_kernel<NQ, TRACERS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, vol_rhs_mixed_kernel<NQ, TRACERS>,
                                                      N3, smem);
    if (e != cudaSuccess) return e;
    const int64_t wave = (int64_t)num_sms * (per_sm > 0 ? per_sm : 1);
    const int64_t ahead = wave / 4 > 0 ? wave / 4 : 1;   // a quarter of a wave
    vol_rhs_mixed_kernel<NQ, TRACERS><<<(unsigned)r.count, N3, smem, s>>>(
        geo, P, q, rhs, r.M, r.e0, nf, r.e0 + r.count, ahead);
    return cudaGetLastError();
}

template <int NQ>
cudaError_t launch_nq(ElemRange r, int nf, const MixedGeometry &geo, const MixedParams &P,
                      const float *q, float *rhs, int num_sms, cudaStream_t s) {
    if (nf == kFields) return launch_kernel<NQ, false>(r, nf, geo, P, q, rhs, num_sms, s);
    return launch_kernel<NQ, true>(r, nf, geo, P, q, rhs, num_sms, s);
}

__global__ void to_f32_kernel(const double *__restrict__ src, float *__restrict__ dst, int64_t M) {
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < M;
         m += (int64_t)gridDim.x * blockDim.x)
        dst[m] = __double2float_rn(src[m]);
}

}  // namespace

cudaError_t launch_to_f32(const double *src, float *dst, int64_t M, cudaStream_t s) {
    if (M == 0) return cudaSuccess;
    to_f32_kernel<<<1216, 256, 0, s>>>(src, dst, M);
    return cudaGetLastError();
}

cudaError_t launch_vol_rhs_mixed(int N, int nf, ElemRange r, const MixedGeometry &geo,
                                 const MixedParams &P, const float *q, float *rhs, int num_sms,
                                 cudaStream_t s) {
    if (r.count <= 0) return cudaSuccess;
    if (nf < kFields || nf > kMaxFields) return cudaErrorInvalidValue;
    switch (N) {
        case 1: return launch_nq<2>(r, nf, geo, P, q, rhs, num_sms, s);
        case 2: return launch_nq<3>(r, nf, geo, P, q, rhs, num_sms, s);
        case 3: return launch_nq<4>(r, nf, geo, P, q, rhs, num_sms, s);
        case 4: return launch_nq<5>(r, nf, geo, P, q, rhs, num_sms, s);
        case 5: return launch_nq<6>(r, nf, geo, P, q, rhs, num_sms, s);
        case 6: return launch_nq<7>(r, nf, geo, P, q, rhs, num_sms, s);
        case 7: return launch_nq<8>(r, nf, geo, P, q, rhs, num_sms, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace numa
