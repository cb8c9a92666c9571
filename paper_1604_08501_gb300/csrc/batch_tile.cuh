// Per-tile device code of the batched low-storage Runge-Kutta integrator:
// one CTA of 512 threads takes `count` elements of one instance through all
// 5 * nsteps stages (see batch_lsrk.cu for the scheme and the design).
#pragma once

#include <type_traits>

#include "element_sweep.cuh"
#include "eos.cuh"
#include "numa_internal.h"

namespace numa {

namespace {

constexpr int kThreads = 512;

template <int NQ, bool MIXED>
__device__ void run_tile(const BatchInstance &I, int64_t e0, int64_t count, const LsrkCoef &co,
                         int nsteps, double dt, void *smem) {
    using T = typename std::conditional<MIXED, float, double>::type;
    constexpr int N3 = NQ * NQ * NQ;
    constexpr int NL = NQ * NQ;
    constexpr int EPP = kThreads / N3;          // elements per pass
    T *sF = static_cast<T *>(smem);             // [(d*5 + b)*EPP + el][slot]
    const int l = threadIdx.x;
    const int el = l / N3, p = l % N3;
    const int i = p % NQ, j = (p / NQ) % NQ, k = p / NL;
    const int64_t M = I.M;
    T *qv = static_cast<T *>(I.q);
    const T dtt = static_cast<T>(dt);

    for (int64_t base = e0; base < e0 + count; base += EPP) {
        const int npass = (int)((e0 + count - base) < EPP ? (e0 + count - base) : EPP);
        const bool active = el < npass;
        const int64_t node = (base + (active ? el : 0)) * N3 + p;
        T q[kFields], dq[kFields];
#pragma unroll
        for (int b = 0; b < kFields; ++b) {
            q[b] = active ? qv[b * M + node] : T(0);
            dq[b] = T(0);
        }
        if (!active) q[0] = MIXED ? T(0) : T(1);   // idle threads hold a harmless state

        for (int step = 0; step < nsteps; ++step) {
#pragma unroll 1
            for (int st = 0; st < 5; ++st) {
                __syncthreads();   // previous phase-3 reads of sF are done
                // ---- phase 1: p', fluxes ------------------------------
                if (active) {
                    T rho, Th, pp, g[9];
                    if constexpr (MIXED) {
#pragma unroll
                        for (int s2 = 0; s2 < 9; ++s2) g[s2] = __ldg(I.mgeo.g[s2] + node);
                        const T t0 = __ldg(I.mgeo.theta_ref + node);
                        rho = __ldg(I.mgeo.rho_ref + node) + q[0];
                        Th = t0 + q[4];
                        pp = pressure_perturbation_f32(q[4], t0, I.mp);
                    } else {
#pragma unroll
                        for (int s2 = 0; s2 < 9; ++s2) g[s2] = __ldg(I.geo.g[s2] + node);
                        rho = q[0];
                        Th = q[4];
                        pp = pressure_perturbation(Th, __ldg(I.geo.theta_ref + node),
                                                   __ldg(I.geo.w + node), __ldg(I.geo.A + node), I.np);
                    }
                    const T rinv = T(1) / rho;
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        const T g1 = g[3 * d], g2 = g[3 * d + 1], g3 = g[3 * d + 2];
                        const T v = fma(g3, q[3], fma(g2, q[2], g1 * q[1]));
                        const T u = v * rinv;
                        T *F = sF + (d * kFields * EPP + el) * N3 + dir_slot<NQ, T>(d, i, j, k);
                        F[0 * EPP * N3] = v;
                        F[1 * EPP * N3] = fma(q[1], u, g1 * pp);
                        F[2 * EPP * N3] = fma(q[2], u, g2 * pp);
                        F[3 * EPP * N3] = fma(q[3], u, g3 * pp);
                        F[4 * EPP * N3] = Th * u;
                    }
                }
                __syncthreads();
                // ---- phase 2: sweeps ------------------------------------
                for (int t = l; t < 3 * kFields * npass * NL; t += kThreads) {
                    const int bd = t / (npass * NL), rem = t % (npass * NL);
                    if constexpr (MIXED)
                        sweep_line<NQ>(sF + (bd * EPP + rem / NL) * N3, rem % NL, I.mp);
                    else
                        sweep_line<NQ>(sF + (bd * EPP + rem / NL) * N3, rem % NL, I.np);
                }
                __syncthreads();
                // ---- phase 3: rhs, stage update ------------------------
                if (active) {
                    const T a = static_cast<T>(co.A[st]), bcoef = static_cast<T>(co.B[st]);
                    const T jinv = MIXED ? T(__ldg(I.mgeo.Jinv + node)) : T(__ldg(I.geo.Jinv + node));
                    // rho - rho_ref of this stage's state, taken before q is updated below
                    const T drho = MIXED ? q[0] : q[0] - T(__ldg(I.geo.rho_ref + node));
#pragma unroll
                    for (int b = 0; b < kFields; ++b) {
                        const T *base_b = sF + el * N3;
                        const T R = base_b[(0 * kFields + b) * EPP * N3 + dir_slot<NQ, T>(0, i, j, k)] +
                                    base_b[(1 * kFields + b) * EPP * N3 + dir_slot<NQ, T>(1, i, j, k)] +
                                    base_b[(2 * kFields + b) * EPP * N3 + dir_slot<NQ, T>(2, i, j, k)];
                        T rhs = -jinv * R;
                        if (b == 3)
                            rhs = fma(-drho, static_cast<T>(MIXED ? I.mp.grav : I.np.eos.grav), rhs);
                        dq[b] = fma(a, dq[b], dtt * rhs);
                        q[b] = fma(bcoef, dq[b], q[b]);
                    }
                }
            }
        }
        if (active) {
#pragma unroll
            for (int b = 0; b < kFields; ++b) qv[b * M + node] = q[b];
        }
    }
}

}  // namespace

}  // namespace numa
