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
// sweeps by line in place, combination by point.  Two kernels:
//  * vol_rhs_mixed_kernel<Nq>: one CTA of Nq^3 threads per element, direct loads.
//  * vol_rhs_mixed_bulk_kernel (Nq = 8): persistent CTAs, 3 per SM.  The element
//    slab (17 arrays x 2 KB, contiguous per array and element) is staged in
//    shared memory by bulk asynchronous copies (cp.async.bulk) completing on an
//    mbarrier.  One stage per CTA: once phase 1 has read an element's slab, the
//    stage is refilled with the CTA's next element, whose copies stay in flight
//    during the sweeps and stores.  (Two stages per CTA fit only two CTAs per
//    SM; three CTAs with one stage each keep more warps resident, +2 %.)  Waits
//    are bounded: on a timeout the kernel sets bit 0 of *err, drains its copies
//    (again bounded) and returns.
#include <cuda_runtime.h>

#include "bulk_copy.cuh"
#include "element_sweep.cuh"
#include "eos.cuh"
#include "numa_internal.h"

namespace numa {

namespace {

template <int NQ>
constexpr int mixed_min_ctas() {
    constexpr int n = 1536 / (NQ * NQ * NQ);
    return n < 1 ? 1 : (n > 32 ? 32 : n);
}

// TRACERS: nf = 5 + tracers fields at run time (tracers Q in FP32 as they are,
// flux Q u_d, no source).  Without tracers nf is 5.
template <int NQ, bool TRACERS>
__global__ void __launch_bounds__(NQ * NQ * NQ, mixed_min_ctas<NQ>())
vol_rhs_mixed_kernel(MixedGeometry geo, MixedParams P, const float *__restrict__ q,
                     float *__restrict__ rhs, int64_t M, int64_t e0, int nf_run) {
    constexpr int N3 = NQ * NQ * NQ;
    constexpr int NL = NQ * NQ;
    constexpr int EW = block_words<NQ, float>();   // one (direction, field) block
    const int nf = TRACERS ? nf_run : kFields;
    extern __shared__ float sFm[];            // [direction*nf + field][slot]

    const int l = threadIdx.x;
    const int i = l % NQ, j = (l / NQ) % NQ, k = l / (NQ * NQ);
    const int64_t node = (e0 + blockIdx.x) * N3 + l;

    // ---- phase 1: p', fluxes ----------------------------------------
    const float rp = q[node];
    const float U[3] = {q[M + node], q[2 * M + node], q[3 * M + node]};
    const float thp = q[4 * M + node];
    const float th0 = geo.theta_ref[node];
    const float rho = geo.rho_ref[node] + rp;
    const float Th = th0 + thp;
    const float pp = pressure_perturbation_f32(thp, th0, P);
    const float rinv = __frcp_rn(rho);   // correctly rounded, as 1.0f / rho
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
    const float Jinv = geo.Jinv[node];
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

// ---------------------------------------------------------------------------
// Nq = 8, persistent, bulk-copy staged.
// ---------------------------------------------------------------------------
constexpr int kSlabArrays = 17;                       // 5 state + 9 metric + Jinv + 2 reference
constexpr int kPts = 512;
constexpr uint32_t kSlabBytes = kPts * sizeof(float);  // one array of one element
// Stages per CTA and CTAs per SM: one stage (34 KB) and 34.6 KB of fluxes (lines
// of 9 slots) make 69 KB per CTA, so three CTAs of 512 threads share an SM.
constexpr int kBulkStages = 1;
constexpr int kBulkCtasPerSm = kBulkStages == 1 ? 3 : 2;
constexpr int kBlk = block_words<8, float>();            // one (direction, field) block
constexpr size_t kBulkSmem = sizeof(float) * (kBulkStages * kSlabArrays * kPts + 3 * kFields * kBlk);

__device__ __forceinline__ void issue_slab(int64_t e, int64_t M, const float *q,
                                           const MixedGeometry &geo, float *st, uint64_t *bar) {
    mbar_arrive_expect_tx(bar, kSlabArrays * kSlabBytes);
    const int64_t off = e * kPts;
#pragma unroll
    for (int a = 0; a < kFields; ++a) bulk_g2s(st + a * kPts, q + a * M + off, kSlabBytes, bar);
#pragma unroll
    for (int a = 0; a < 9; ++a) bulk_g2s(st + (kFields + a) * kPts, geo.g[a] + off, kSlabBytes, bar);
    bulk_g2s(st + 14 * kPts, geo.Jinv + off, kSlabBytes, bar);
    bulk_g2s(st + 15 * kPts, geo.rho_ref + off, kSlabBytes, bar);
    bulk_g2s(st + 16 * kPts, geo.theta_ref + off, kSlabBytes, bar);
}

__global__ void __launch_bounds__(kPts, kBulkCtasPerSm)
vol_rhs_mixed_bulk_kernel(MixedGeometry geo, MixedParams P, const float *__restrict__ q,
                          float *__restrict__ rhs, int64_t M, int64_t e0, int64_t e_end,
                          int *err) {
    constexpr int NQ = 8;
    constexpr int S = kBulkStages;
    extern __shared__ __align__(128) float smem_f[];
    __shared__ __align__(8) uint64_t bar[S];
    float *sF = smem_f + S * kSlabArrays * kPts;

    const int l = threadIdx.x;
    const int i = l & 7, j = (l >> 3) & 7, k = l >> 6;
    if (l == 0) {
#pragma unroll
        for (int b = 0; b < S; ++b) mbar_init(&bar[b], 1);
        fence_mbar_init();
    }
    __syncthreads();

    // Per stage b: bit b of `parity` is the phase to wait for; bit b of
    // `pending` (thread 0 only) marks copies in flight.
    uint32_t parity = 0u, pending = 0u;
    const int64_t G = gridDim.x;
    int64_t e = e0 + blockIdx.x;
    // S elements in flight from the start: this CTA's first S into stages 0..S-1.
    if (l == 0) {
#pragma unroll
        for (int b = 0; b < S; ++b)
            if (e + b * G < e_end) {
                issue_slab(e + b * G, M, q, geo, smem_f + b * kSlabArrays * kPts, &bar[b]);
                pending |= 1u << b;
            }
    }
    int buf = 0;
    bool failed = false;
    for (; e < e_end; e += G) {
        const bool ok = bulk_wait(&bar[buf], (parity >> buf) & 1u);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        parity ^= 1u << buf;
        pending &= ~(1u << buf);
        float *const st = smem_f + buf * kSlabArrays * kPts;

        // ---- phase 1: p', fluxes ------------------------------------
        const float rp = st[0 * kPts + l];
        const float U[3] = {st[1 * kPts + l], st[2 * kPts + l], st[3 * kPts + l]};
        const float thp = st[4 * kPts + l];
        const float th0 = st[16 * kPts + l];
        const float rho = st[15 * kPts + l] + rp;
        const float Th = th0 + thp;
        const float pp = pressure_perturbation_f32(thp, th0, P);
        const float rinv = __frcp_rn(rho);   // correctly rounded, as 1.0f / rho
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float g1 = st[(kFields + 3 * d) * kPts + l];
            const float g2 = st[(kFields + 3 * d + 1) * kPts + l];
            const float g3 = st[(kFields + 3 * d + 2) * kPts + l];
            const float v = fmaf(g3, U[2], fmaf(g2, U[1], g1 * U[0]));
            const float u = v * rinv;
            float *F = sF + d * kFields * kBlk + dir_slot<NQ, float>(d, i, j, k);
            F[0 * kBlk] = v;
            F[1 * kBlk] = fmaf(U[0], u, g1 * pp);
            F[2 * kBlk] = fmaf(U[1], u, g2 * pp);
            F[3 * kBlk] = fmaf(U[2], u, g3 * pp);
            F[4 * kBlk] = Th * u;
        }
        const float Jinv = st[14 * kPts + l];
        __syncthreads();
        // This stage is dead now (phase 1 read all of it, and phase 3 uses
        // registers): refill it with the element S ahead, so that its copies
        // are in flight during the sweeps and stores.
        if (l == 0 && e + S * G < e_end) {
            fence_proxy_async();   // order the generic reads above before the async writes
            issue_slab(e + S * G, M, q, geo, st, &bar[buf]);
            pending |= 1u << buf;
        }

        // ---- phase 2: even-odd sweeps ---------------------------------
        for (int item = l; item < 3 * kFields * 64; item += kPts)
            sweep_line<NQ>(sF + (item >> 6) * kBlk, item & 63, P);
        __syncthreads();

        // ---- phase 3: combine, scale, gravity, store ------------------
        const int64_t node = e * kPts + l;
#pragma unroll
        for (int b = 0; b < kFields; ++b) {
            const float R = sF[(0 * kFields + b) * kBlk + dir_slot<NQ, float>(0, i, j, k)] +
                            sF[(1 * kFields + b) * kBlk + dir_slot<NQ, float>(1, i, j, k)] +
                            sF[(2 * kFields + b) * kBlk + dir_slot<NQ, float>(2, i, j, k)];
            float v = -Jinv * R;
            if (b == 3) v = fmaf(-rp, P.grav, v);
            rhs[b * M + node] = v;
        }
        // No barrier here: the barrier after the next wait orders this phase 3's
        // reads of sF before the next phase 1 writes it.
        buf = buf + 1 == S ? 0 : buf + 1;
    }
    if (failed && l == 0) {
        atomicOr(err, 1);
        // Drain the copies still in flight into this CTA's shared memory.
#pragma unroll
        for (int b = 0; b < S; ++b)
            if ((pending >> b) & 1u) bulk_wait(&bar[b], (parity >> b) & 1u);
    }
}

template <int NQ, bool TRACERS>
cudaError_t launch_kernel(ElemRange r, int nf, const MixedGeometry &geo, const MixedParams &P,
                          const float *q, float *rhs, cudaStream_t s) {
    constexpr int N3 = NQ * NQ * NQ;
    const size_t smem = sizeof(float) * nf * 3 * block_words<NQ, float>();
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(vol_rhs_mixed_kernel<NQ, TRACERS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    vol_rhs_mixed_kernel<NQ, TRACERS><<<(unsigned)r.count, N3, smem, s>>>(geo, P, q, rhs, r.M, r.e0,
                                                                          nf);
    return cudaGetLastError();
}

template <int NQ>
cudaError_t launch_nq(ElemRange r, int nf, const MixedGeometry &geo, const MixedParams &P,
                      const float *q, float *rhs, cudaStream_t s) {
    if (nf == kFields) return launch_kernel<NQ, false>(r, nf, geo, P, q, rhs, s);
    return launch_kernel<NQ, true>(r, nf, geo, P, q, rhs, s);
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
                                 const MixedParams &P, const float *q, float *rhs, int *err,
                                 int num_sms, cudaStream_t s) {
    if (r.count <= 0) return cudaSuccess;
    if (nf < kFields || nf > kMaxFields) return cudaErrorInvalidValue;
    if (N == 7 && nf == kFields) {   // the staged kernel holds the five fields' slabs
        cudaError_t e = cudaFuncSetAttribute(vol_rhs_mixed_bulk_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kBulkSmem);
        if (e != cudaSuccess) return e;
        const int64_t per = kBulkCtasPerSm * (int64_t)num_sms;
        const int64_t ctas = r.count < per ? r.count : per;
        vol_rhs_mixed_bulk_kernel<<<(unsigned)ctas, kPts, kBulkSmem, s>>>(
            geo, P, q, rhs, r.M, r.e0, r.e0 + r.count, err);
        return cudaGetLastError();
    }
    switch (N) {
        case 1: return launch_nq<2>(r, nf, geo, P, q, rhs, s);
        case 2: return launch_nq<3>(r, nf, geo, P, q, rhs, s);
        case 3: return launch_nq<4>(r, nf, geo, P, q, rhs, s);
        case 4: return launch_nq<5>(r, nf, geo, P, q, rhs, s);
        case 5: return launch_nq<6>(r, nf, geo, P, q, rhs, s);
        case 6: return launch_nq<7>(r, nf, geo, P, q, rhs, s);
        case 7: return launch_nq<8>(r, nf, geo, P, q, rhs, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace numa
