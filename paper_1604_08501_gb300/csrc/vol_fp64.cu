// FP64 element volume term on sm_103a.
//
// Computes, per element and point, the pressure perturbation from the Theta
// equation of state, the contravariant fluxes of the five fields in the three
// reference directions, the three D sweeps, the Jinv scaling and the gravity
// source (Sec. 2, Eq. (2); sign and flux form of the paper's r/s subroutines,
// Sec. 3).
//
// Kernel structure: one CTA per element, one thread per point.  Each thread
// computes the fifteen fluxes of its own point once (the paper's "precompute
// fluxes" step, Sec. 3 opt. level 5) into shared memory.  After a barrier it
// applies the three D sweeps from shared memory, keeps the sum in registers
// and applies Jinv once at write-back (opt. levels 7 and 8).  State and
// geometry are read once from HBM, and rhs is written once.
#include <cuda_runtime.h>

#include "numa_internal.h"

namespace numa {

namespace {

// p0 (R Theta / p0)^gamma, the equation of state of Sec. 2.  Each step is
// rounded explicitly, so the create-time evaluation of p(Theta_ref) and the
// per-call evaluation of p(Theta) agree bit for bit for equal arguments.
__device__ __forceinline__ double eos_pressure(double Th, const EosConstants &c) {
    return __dmul_rn(c.p0, pow(__ddiv_rn(__dmul_rn(c.R, Th), c.p0), c.gamma));
}

__global__ void pref_kernel(double *p, int64_t M, EosConstants c) {
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < M;
         m += (int64_t)gridDim.x * blockDim.x)
        p[m] = eos_pressure(p[m], c);
}

template <int NQ>
__global__ void __launch_bounds__(NQ * NQ * NQ)
vol_rhs_fp64_kernel(DeviceGeometry geo, EosConstants c, const double *__restrict__ q,
                    double *__restrict__ rhs, int64_t M) {
    constexpr int N3 = NQ * NQ * NQ;
    __shared__ double sD[NQ * NQ];
    extern __shared__ double sF[];  // [direction][field][point], 15 * N3

    const int l = threadIdx.x;
    const int64_t node = (int64_t)blockIdx.x * N3 + l;
    for (int t = l; t < NQ * NQ; t += N3) sD[t] = geo.D[t];

    const double rho = q[node];
    const double U1 = q[M + node], U2 = q[2 * M + node], U3 = q[3 * M + node];
    const double Th = q[4 * M + node];
    const double pp = eos_pressure(Th, c) - geo.p_ref[node];

#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double g1 = geo.g[3 * d][node], g2 = geo.g[3 * d + 1][node],
                     g3 = geo.g[3 * d + 2][node];
        const double u = (g1 * U1 + g2 * U2 + g3 * U3) / rho;
        double *F = sF + d * kFields * N3 + l;
        F[0 * N3] = rho * u;
        F[1 * N3] = U1 * u + g1 * pp;
        F[2 * N3] = U2 * u + g2 * pp;
        F[3 * N3] = U3 * u + g3 * pp;
        F[4 * N3] = Th * u;
    }
    __syncthreads();

    const int i = l % NQ, j = (l / NQ) % NQ, k = l / (NQ * NQ);
    const double Jinv = geo.Jinv[node];
    const double drho = rho - geo.rho_ref[node];
#pragma unroll
    for (int b = 0; b < kFields; ++b) {
        const double *Fr = sF + (0 * kFields + b) * N3;
        const double *Fs = sF + (1 * kFields + b) * N3;
        const double *Ft = sF + (2 * kFields + b) * N3;
        double s = 0.0;
#pragma unroll
        for (int n = 0; n < NQ; ++n) s += sD[i * NQ + n] * Fr[(k * NQ + j) * NQ + n];
#pragma unroll
        for (int n = 0; n < NQ; ++n) s += sD[j * NQ + n] * Fs[(k * NQ + n) * NQ + i];
#pragma unroll
        for (int n = 0; n < NQ; ++n) s += sD[k * NQ + n] * Ft[(n * NQ + j) * NQ + i];
        double v = -Jinv * s;
        if (b == 3) v -= drho * c.grav;
        rhs[b * M + node] = v;
    }
}

template <int NQ>
cudaError_t launch_nq(int64_t Ne, const DeviceGeometry &geo, EosConstants c, const double *q,
                      double *rhs, cudaStream_t s) {
    constexpr int N3 = NQ * NQ * NQ;
    const size_t smem = sizeof(double) * kFields * 3 * N3;
    // The opt-in above 48 KB is per device; setting it on every launch keeps
    // multi-device processes correct and costs about a microsecond.
    cudaError_t e = cudaFuncSetAttribute(vol_rhs_fp64_kernel<NQ>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t M = Ne * N3;
    vol_rhs_fp64_kernel<NQ><<<(unsigned)Ne, N3, smem, s>>>(geo, c, q, rhs, M);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_pref_fp64(const double *rhotheta_ref, double *p_ref, int64_t M,
                             EosConstants c, cudaStream_t s) {
    if (M == 0) return cudaSuccess;
    if (rhotheta_ref != p_ref) {
        cudaError_t e = cudaMemcpyAsync(p_ref, rhotheta_ref, sizeof(double) * M,
                                        cudaMemcpyDefault, s);
        if (e != cudaSuccess) return e;
    }
    pref_kernel<<<1216, 256, 0, s>>>(p_ref, M, c);
    return cudaGetLastError();
}

cudaError_t launch_vol_rhs_fp64(int N, int64_t Ne, const DeviceGeometry &geo, EosConstants c,
                                const double *q, double *rhs, cudaStream_t s) {
    if (Ne == 0) return cudaSuccess;
    switch (N) {
        case 1: return launch_nq<2>(Ne, geo, c, q, rhs, s);
        case 2: return launch_nq<3>(Ne, geo, c, q, rhs, s);
        case 3: return launch_nq<4>(Ne, geo, c, q, rhs, s);
        case 4: return launch_nq<5>(Ne, geo, c, q, rhs, s);
        case 5: return launch_nq<6>(Ne, geo, c, q, rhs, s);
        case 6: return launch_nq<7>(Ne, geo, c, q, rhs, s);
        case 7: return launch_nq<8>(Ne, geo, c, q, rhs, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace numa
