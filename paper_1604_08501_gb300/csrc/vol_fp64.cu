// Native FP64 element volume term on sm_103a, orders N = 1..7 (N = 8..15:
// vol_fp64_high.cu), with or without passive tracers.
//
// Computes, per element and point, the pressure perturbation from the Theta
// equation of state, the contravariant fluxes of the five fields in the three
// reference directions, the three D sweeps, the Jinv scaling and the gravity
// source (Sec. 2, Eq. (2); sign and flux form of the paper's r/s subroutines,
// Sec. 3).  Every floating-point operation is an FP64 operation.
//
// On GB300 the FP64 pipe (about 0.53 T DFMA/s) binds this kernel, so the
// design minimises FP64 instructions per point:
//  * p' = p(Theta) - p(Theta_ref) is evaluated as p_ref ((1+x)^gamma - 1) by
//    its binomial series in x = (Theta - Theta_ref)/Theta_ref (12 FP64
//    operations for |x| <= 1/64, and no cancellation); eos.cuh has the wider
//    forms.
//  * 1/rho is formed once; u_d = (g_d . U) * (1/rho).
//  * The fluxes are computed once per point into shared memory (the paper's
//    flux precompute, Sec. 3, opt. level 5).
//  * Each line of each (direction, field) is swept by one thread with the
//    even-odd split of the GLL D (D[N-i][N-n] = -D[i][n]): E_m = F_m + F_{N-m},
//    O_m = F_m - F_{N-m}, and S_i = a_i + b_i, S_{N-i} = b_i - a_i with
//    a_i = sum_m De[i][m] E_m (+ D[i][c] F_c for odd Nq), b_i = sum_m Do[i][m] O_m.
//    That is half the multiplies of the direct sweep.
//  * Jinv is applied once to the sum of the three sweeps (opt. level 8).
//
// One CTA of Nq^3 threads per element, in three phases: fluxes by point,
// sweeps by line (in place), combination by point.
#include <cuda_runtime.h>

#include "element_sweep.cuh"
#include "eos.cuh"
#include "numa_internal.h"

namespace numa {

namespace {

// Resident CTAs per SM the register budget is sized for: 1024 threads per SM,
// at most 32 CTAs.
template <int NQ>
constexpr int min_ctas() {
    constexpr int n = 1024 / (NQ * NQ * NQ);
    return n < 1 ? 1 : (n > 32 ? 32 : n);
}

// TRACERS: nf = 5 + tracers fields (up to 8) at run time; the tracers follow
// Theta with flux Q u_d and no source.  Without tracers nf is 5.
template <int NQ, bool TRACERS>
__global__ void __launch_bounds__(NQ * NQ * NQ, min_ctas<NQ>())
vol_rhs_fp64_kernel(DeviceGeometry geo, NativeParams P, const double *__restrict__ q,
                    double *__restrict__ rhs, int64_t M, int64_t e0, int nf_run) {
    constexpr int N3 = NQ * NQ * NQ;
    constexpr int NL = NQ * NQ;               // lines per (direction, field)
    const int nf = TRACERS ? nf_run : kFields;
    extern __shared__ double sF[];            // [direction*nf + field][slot]

    const int l = threadIdx.x;
    const int i = l % NQ, j = (l / NQ) % NQ, k = l / (NQ * NQ);
    const int64_t node = (e0 + blockIdx.x) * N3 + l;

    // ---- phase 1: p', fluxes ----------------------------------------
    const double rho = q[node];
    const double U[3] = {q[M + node], q[2 * M + node], q[3 * M + node]};
    const double Th = q[4 * M + node];
    const double pp = pressure_perturbation(Th, geo.theta_ref[node], geo.w[node], geo.A[node], P);
    const double rinv = __drcp_rn(rho);
    double Q[kMaxFields - kFields];
    if constexpr (TRACERS) {
#pragma unroll
        for (int t = 0; t < kMaxFields - kFields; ++t)
            Q[t] = kFields + t < nf ? q[(kFields + t) * M + node] : 0.0;
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double g1 = geo.g[3 * d][node], g2 = geo.g[3 * d + 1][node],
                     g3 = geo.g[3 * d + 2][node];
        const double v = fma(g3, U[2], fma(g2, U[1], g1 * U[0]));
        const double u = v * rinv;
        const int s = dir_slot<NQ, double>(d, i, j, k);
        double *F = sF + d * nf * N3 + s;
        F[0 * N3] = v;
        F[1 * N3] = fma(U[0], u, g1 * pp);
        F[2 * N3] = fma(U[1], u, g2 * pp);
        F[3 * N3] = fma(U[2], u, g3 * pp);
        F[4 * N3] = Th * u;
        if constexpr (TRACERS) {
#pragma unroll
            for (int t = 0; t < kMaxFields - kFields; ++t)
                if (kFields + t < nf) F[(kFields + t) * N3] = Q[t] * u;
        }
    }
    __syncthreads();

    // ---- phase 2: even-odd sweeps, one line per task, in place --------
    for (int item = l; item < 3 * nf * NL; item += N3)
        sweep_line<NQ>(sF + (item / NL) * N3, item % NL, P);
    __syncthreads();

    // ---- phase 3: combine, scale, gravity, store ----------------------
    const double Jinv = geo.Jinv[node];
    const double drho = rho - geo.rho_ref[node];
#pragma unroll
    for (int b = 0; b < (TRACERS ? kMaxFields : kFields); ++b) {
        if (TRACERS && b >= nf) break;
        const double R = sF[(0 * nf + b) * N3 + dir_slot<NQ, double>(0, i, j, k)] +
                         sF[(1 * nf + b) * N3 + dir_slot<NQ, double>(1, i, j, k)] +
                         sF[(2 * nf + b) * N3 + dir_slot<NQ, double>(2, i, j, k)];
        double v = -Jinv * R;
        if (b == 3) v = fma(-drho, P.eos.grav, v);
        rhs[b * M + node] = v;
    }
}

template <int NQ, bool TRACERS>
cudaError_t launch_kernel(ElemRange r, int nf, const DeviceGeometry &geo, const NativeParams &P,
                          const double *q, double *rhs, cudaStream_t s) {
    constexpr int N3 = NQ * NQ * NQ;
    const size_t smem = sizeof(double) * nf * 3 * N3;
    // The opt-in above 48 KB is per device; setting it on every launch keeps
    // multi-device processes correct and costs about a microsecond.
    cudaError_t e = cudaFuncSetAttribute(vol_rhs_fp64_kernel<NQ, TRACERS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    vol_rhs_fp64_kernel<NQ, TRACERS><<<(unsigned)r.count, N3, smem, s>>>(geo, P, q, rhs, r.M, r.e0,
                                                                         nf);
    return cudaGetLastError();
}

template <int NQ>
cudaError_t launch_nq(ElemRange r, int nf, const DeviceGeometry &geo, const NativeParams &P,
                      const double *q, double *rhs, cudaStream_t s) {
    if (nf == kFields) return launch_kernel<NQ, false>(r, nf, geo, P, q, rhs, s);
    return launch_kernel<NQ, true>(r, nf, geo, P, q, rhs, s);
}

// w = 1/Theta_ref and A = p(Theta_ref)/Theta_ref, in place of a copy of Theta_ref.
__global__ void reference_eos_kernel(const double *__restrict__ theta_ref, double *__restrict__ w,
                                     double *__restrict__ A, int64_t M, EosConstants c) {
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < M;
         m += (int64_t)gridDim.x * blockDim.x) {
        const double th = theta_ref[m];
        w[m] = 1.0 / th;
        A[m] = eos_pressure(th, c) / th;
    }
}

}  // namespace

cudaError_t launch_reference_eos(const double *theta_ref, double *w, double *A, int64_t M,
                                 EosConstants c, cudaStream_t s) {
    if (M == 0) return cudaSuccess;
    reference_eos_kernel<<<1216, 256, 0, s>>>(theta_ref, w, A, M, c);
    return cudaGetLastError();
}

cudaError_t launch_vol_rhs_fp64(int N, int nf, ElemRange r, const DeviceGeometry &geo,
                                const NativeParams &P, const double *q, double *rhs,
                                cudaStream_t s) {
    if (r.count <= 0) return cudaSuccess;
    if (nf < kFields || nf > kMaxFields) return cudaErrorInvalidValue;
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
