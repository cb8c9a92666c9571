// Element volume term for orders N = 8..15 (Nq = 9..16), native FP64 and
// mixed precision.
//
// The operation of vol_fp64.cu (Sec. 2, Eq. (2); sign and flux form of the
// paper's r/s subroutines, Sec. 3), for the high orders of the paper's Nq
// study (Sec. 5, Nq up to 16).  An element of Nq = 16 has 4096 points: more
// than a CTA has threads, and its fifteen FP64 flux arrays (491 KB) exceed
// shared memory.  So:
//  * one CTA of 3 Nq^2 threads per element: three per (i, j) column, each
//    looping over a third of its k-planes, as the paper's kernels own (i, j)
//    lanes and loop over k;
//  * a first pass forms the contravariant velocities u_d and p' of all points
//    into shared memory (4 Nq^3 values);
//  * then one pass per field b: its three flux arrays F_d[b] into shared
//    memory (3 Nq^2 lines of 16 slots), the three D sweeps in place (one line
//    per thread, even-odd split), and rhs_b of the thread's points straight
//    to HBM.
// Shared memory: (4 Nq^3 + 48 Nq^2) values, 224 KB at Nq = 16 in FP64 (every
// operation FP64; bound by the FP64 pipe like the low orders) and 112 KB in
// the mixed mode (FP32 perturbation state and arithmetic, as vol_mixed.cu).
#include <cuda_runtime.h>

#include "element_sweep.cuh"
#include "eos.cuh"
#include "numa_internal.h"

namespace numa {

namespace {

// T: double (NUMA_FP64) or float (NUMA_MIXED: FP32 perturbation state
// (rho', U, Theta', tracers), FP32 geometry, p' from Theta' without
// cancellation).
template <int NQ, typename T>
constexpr size_t high_smem_bytes() {
    return sizeof(T) * (4 * NQ * NQ * NQ + 3 * NQ * NQ * 16);
}

// Threads: three per (i, j) column, each owning a slab of KS = ceil(Nq/3)
// k-planes in the point phases and one line in the sweep phase
// (3 directions x Nq^2 lines = 3 Nq^2 threads).
template <int NQ>
constexpr int high_threads() {
    return 3 * NQ * NQ;
}

// CTAs per SM the register budget is sized for: two where two CTAs' shared
// memory fits an SM and still leaves 64 registers per thread, else one.
template <int NQ, typename T>
constexpr int high_min_ctas() {
    return (2 * (high_smem_bytes<NQ, T>() + 1024) <= 228 * 1024 && 2 * high_threads<NQ>() <= 1024)
               ? 2
               : 1;
}

template <typename T> struct HighTypes;
template <> struct HighTypes<double> { using Geo = DeviceGeometry; using Params = HighParams; };
template <> struct HighTypes<float> { using Geo = MixedGeometry; using Params = HighParams32; };

template <int NQ, typename T>
__global__ void __launch_bounds__(3 * NQ * NQ, (high_min_ctas<NQ, T>()))
vol_rhs_high_kernel(typename HighTypes<T>::Geo geo, typename HighTypes<T>::Params P,
                    const T *__restrict__ q, T *__restrict__ rhs, int64_t M, int64_t e0, int nf) {
    constexpr bool MIXED = sizeof(T) == 4;
    constexpr int NL = NQ * NQ;      // columns; lines per direction
    constexpr int N3 = NQ * NL;
    constexpr int FB = NL * 16;      // one direction's flux block (padded lines)
    constexpr int KS = (NQ + 2) / 3; // k-planes per slab
    // k-loop unrolling: full in FP32 (registers to spare, more loads in
    // flight), two planes in FP64 (register budget)
    constexpr int KU = MIXED ? KS : 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sU = reinterpret_cast<T *>(smem_raw);   // u_d of every point: [d][k][j][i]
    T *sP = sU + 3 * N3;                       // p' of every point: [k][j][i]
    T *sF = sU + 4 * N3;                       // fluxes of one field: [d][line][slot]

    const int t = threadIdx.x;
    const int c = t % NL, slab = t / NL;
    const int i = c % NQ, j = c / NQ;
    const int kb = slab * KS;                          // first k-plane of the slab
    const int64_t node0 = (e0 + blockIdx.x) * N3 + c;  // point (i, j, 0); + k NL

    // ---- pass 0: u_d, p', and the density fluxes F_d[rho] = g_d . U ------
#pragma unroll(KU)
    for (int kk = 0; kk < KS; ++kk) {
        const int k = kb + kk;
        if (k < NQ) {
            const int64_t node = node0 + k * NL;
            const T U1 = q[M + node], U2 = q[2 * M + node], U3 = q[3 * M + node];
            T rinv;
            if constexpr (MIXED) {
                const float th0 = geo.theta_ref[node];
                sP[k * NL + c] = pressure_perturbation_f32(q[4 * M + node], th0, P);
                rinv = __frcp_rn(geo.rho_ref[node] + q[node]);
            } else {
                sP[k * NL + c] = pressure_perturbation(q[4 * M + node], geo.theta_ref[node],
                                                       geo.w[node], geo.A[node], P);
                rinv = __drcp_rn(q[node]);
            }
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const T v = fma(geo.g[3 * d + 2][node], U3,
                                fma(geo.g[3 * d + 1][node], U2, geo.g[3 * d][node] * U1));
                sU[d * N3 + k * NL + c] = v * rinv;
                sF[d * FB + dir_slot<NQ, T>(d, i, j, k)] = v;
            }
        }
    }

#pragma unroll 1
    for (int b = 0; b < nf; ++b) {   // 5 fields, then the tracers
        if (b > 0) {
            __syncthreads();   // the previous field's combination has read sF
#pragma unroll(KU)
            for (int kk = 0; kk < KS; ++kk) {
                const int k = kb + kk;
                if (k < NQ) {
                    const int64_t node = node0 + k * NL;
                    T qb = q[b * M + node];
                    if (MIXED && b == 4) qb += geo.theta_ref[node];   // Theta = Theta_ref + Theta'
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        const T u = sU[d * N3 + k * NL + c];
                        // F_d[U_a] = U_a u_d + g_{ad} p';  F_d[Theta] = Theta u_d,
                        // and likewise Q u_d for a tracer
                        const T F =
                            b < 4 ? fma(qb, u, geo.g[3 * d + (b - 1)][node] * sP[k * NL + c]) : qb * u;
                        sF[d * FB + dir_slot<NQ, T>(d, i, j, k)] = F;
                    }
                }
            }
        }
        __syncthreads();
        // ---- sweeps: thread t sweeps line c of direction `slab` ------------
        sweep_line<NQ>(sF + slab * FB, c, P);
        __syncthreads();
        // ---- rhs_b of the slab: -Jinv (S_r + S_s + S_t), gravity on U3 ------
#pragma unroll(KU)
        for (int kk = 0; kk < KS; ++kk) {
            const int k = kb + kk;
            if (k < NQ) {
                const int64_t node = node0 + k * NL;
                const T R = sF[dir_slot<NQ, T>(0, i, j, k)] + sF[FB + dir_slot<NQ, T>(1, i, j, k)] +
                            sF[2 * FB + dir_slot<NQ, T>(2, i, j, k)];
                T v = -geo.Jinv[node] * R;
                if (b == 3) {
                    if constexpr (MIXED)
                        v = fma(-q[node], P.grav, v);   // rho' is the stored state
                    else
                        v = fma(-(q[node] - geo.rho_ref[node]), P.eos.grav, v);
                }
                rhs[b * M + node] = v;
            }
        }
    }
}

template <int NQ, typename T, typename Geo, typename Params>
cudaError_t launch_high(ElemRange r, int nf, const Geo &geo, const Params &P, const T *q, T *rhs,
                        cudaStream_t s) {
    constexpr size_t smem = high_smem_bytes<NQ, T>();
    cudaError_t e = cudaFuncSetAttribute(vol_rhs_high_kernel<NQ, T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    vol_rhs_high_kernel<NQ, T><<<(unsigned)r.count, high_threads<NQ>(), smem, s>>>(geo, P, q, rhs,
                                                                                r.M, r.e0, nf);
    return cudaGetLastError();
}

template <typename T, typename Geo, typename Params>
cudaError_t launch_high_order(int N, int nf, ElemRange r, const Geo &geo, const Params &P,
                              const T *q, T *rhs, cudaStream_t s) {
    if (r.count <= 0) return cudaSuccess;
    if (nf < kFields || nf > kMaxFields) return cudaErrorInvalidValue;
    switch (N) {
        case 8: return launch_high<9>(r, nf, geo, P, q, rhs, s);
        case 9: return launch_high<10>(r, nf, geo, P, q, rhs, s);
        case 10: return launch_high<11>(r, nf, geo, P, q, rhs, s);
        case 11: return launch_high<12>(r, nf, geo, P, q, rhs, s);
        case 12: return launch_high<13>(r, nf, geo, P, q, rhs, s);
        case 13: return launch_high<14>(r, nf, geo, P, q, rhs, s);
        case 14: return launch_high<15>(r, nf, geo, P, q, rhs, s);
        case 15: return launch_high<16>(r, nf, geo, P, q, rhs, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_vol_rhs_fp64_high(int N, int nf, ElemRange r, const DeviceGeometry &geo,
                                     const HighParams &P, const double *q, double *rhs,
                                     cudaStream_t s) {
    return launch_high_order<double>(N, nf, r, geo, P, q, rhs, s);
}

cudaError_t launch_vol_rhs_mixed_high(int N, int nf, ElemRange r, const MixedGeometry &geo,
                                      const HighParams32 &P, const float *q, float *rhs,
                                      cudaStream_t s) {
    return launch_high_order<float>(N, nf, r, geo, P, q, rhs, s);
}

}  // namespace numa
