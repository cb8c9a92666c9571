// Per-tile device code of the batched low-storage Runge-Kutta integrator:
// one CTA of 512 threads takes `count` elements of one instance through all
// 5 * nsteps stages (see batch_lsrk.cu for the scheme and the design).
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "element_sweep.cuh"
#include "eos.cuh"
#include "numa_internal.h"

namespace numa {

namespace {

constexpr int kThreads = 512;

// Shared memory of one CTA and CTAs per SM.  FP64: the fluxes (15 values per
// thread); q and dq stay in registers and one CTA holds an SM (the FP64 pipe
// binds).  Mixed: the fluxes, q and dq (10 values) and the point's geometry
// (g and Jinv, 10 values) in shared memory, so that the kernel fits 64
// registers and two CTAs share an SM, twice the warps to hide latency.
// Flux words of one pass: 3 x NF blocks of EPP elements; the largest over the
// orders sizes the flux region (4-byte values at Nq = 8: lines of 9 slots).
// NF = 5, or 8 in the tiles' tracer forms (TR), whose tracers' q and dq also
// live in shared memory in FP64 (3 + 3 values per thread after the fluxes).
template <typename T, int NQ, int NF = kFields>
__host__ __device__ constexpr int pass_flux_words() {
    return 3 * NF * (kThreads / (NQ * NQ * NQ)) * block_words<NQ, T>();
}
template <typename T, int NF = kFields>
__host__ __device__ constexpr int tile_flux_words() {
    constexpr int w[] = {pass_flux_words<T, 2, NF>(), pass_flux_words<T, 3, NF>(),
                         pass_flux_words<T, 4, NF>(), pass_flux_words<T, 5, NF>(),
                         pass_flux_words<T, 6, NF>(), pass_flux_words<T, 7, NF>(),
                         pass_flux_words<T, 8, NF>()};
    int m = 0;
    for (int x : w) m = x > m ? x : m;
    return m;
}
constexpr int kMixedFluxWords = tile_flux_words<float>();
constexpr int kMixedSmemWords = kMixedFluxWords + (2 * 5 + 10) * kThreads;
template <bool MIXED, bool TR = false>
constexpr size_t tile_smem_bytes() {
    constexpr int NF = TR ? kMaxFields : kFields;
    return MIXED ? sizeof(float) * (tile_flux_words<float, NF>() + (2 * NF + 10) * kThreads)
                 : sizeof(double) * (tile_flux_words<double, NF>() +
                                     (TR ? 2 * (kMaxFields - kFields) * kThreads : 0));
}
template <bool MIXED>
constexpr int tile_ctas_per_sm() {
    return MIXED ? 2 : 1;
}

// Sweep tables per Nq (index Nq; 2..8 used).  They depend only on the order:
// every handle's D is the library's GLL D.  In constant memory, every
// coefficient of a sweep is a constant-bank operand of its FMA, as in the
// single-evaluation kernels, where the tables are kernel parameters.
template <typename T>
struct SweepTables {
    T De[16], Do[16], Dc[4], Dcr[4];
};
__constant__ SweepTables<double> c_sweep64[9];
__constant__ SweepTables<float> c_sweep32[9];

// Fills this translation unit's tables on the current device (synchronous).
inline cudaError_t upload_sweep_tables() {
    SweepTables<double> t64[9] = {};
    SweepTables<float> t32[9] = {};
    for (int N = 1; N <= 7; ++N) {
        double D[64];
        gll_diff_matrix(N, D);
        SweepTables<double> &a = t64[N + 1];
        sweep_tables(N, D, a.De, a.Do, a.Dc, a.Dcr);
        SweepTables<float> &b = t32[N + 1];
        for (int t = 0; t < 16; ++t) {
            b.De[t] = static_cast<float>(a.De[t]);
            b.Do[t] = static_cast<float>(a.Do[t]);
        }
        for (int t = 0; t < 4; ++t) {
            b.Dc[t] = static_cast<float>(a.Dc[t]);
            b.Dcr[t] = static_cast<float>(a.Dcr[t]);
        }
    }
    cudaError_t e = cudaMemcpyToSymbol(c_sweep64, t64, sizeof(t64));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_sweep32, t32, sizeof(t32));
    return e;
}

// Stage coefficients of the scheme in the tile's arithmetic type: A[s] at
// [s], B[s] at [5 + s].  The kernels keep them in shared memory.
template <bool MIXED>
using tile_t = typename std::conditional<MIXED, float, double>::type;

template <bool MIXED>
__device__ __forceinline__ void load_stage_coefficients(const LsrkCoef &co, tile_t<MIXED> *sco) {
    if (threadIdx.x == 0) {   // constant indices: the parameter is read in place
#pragma unroll
        for (int s = 0; s < 5; ++s) {
            sco[s] = static_cast<tile_t<MIXED>>(co.A[s]);
            sco[5 + s] = static_cast<tile_t<MIXED>>(co.B[s]);
        }
    }
}

// TR: the tracer form (instances of 5..8 fields, I.nf): flux blocks laid out
// for 8 fields, the tracers' q and dq in shared memory in both precisions.
template <int NQ, bool MIXED, bool TR = false>
__device__ void run_tile(const BatchInstance &I, int64_t e0, int64_t count,
                         const tile_t<MIXED> *sco, int nsteps, double dt, void *smem) {
    using T = tile_t<MIXED>;
    constexpr int N3 = NQ * NQ * NQ;
    constexpr int NL = NQ * NQ;
    constexpr int NF = TR ? kMaxFields : kFields;   // flux blocks per direction
    constexpr int NTR = kMaxFields - kFields;       // tracers at most
    constexpr int EPP = kThreads / N3;          // elements per pass
    constexpr int EW = block_words<NQ, T>();    // one element's (direction, field) block
    constexpr int BLK = EPP * EW;               // one (direction, field) block of sF
    constexpr int TASKS = 3 * NF * EPP * NL;    // lines per stage (TR: some blocks unused)
    const int nf = TR ? I.nf : kFields;
    T *sF = static_cast<T *>(smem);             // [(d*NF + b)*EPP + el][slot]
    const int l = threadIdx.x;
    const int el = l / N3, p = l % N3;
    const int i = p % NQ, j = (p / NQ) % NQ, k = p / NL;
    // this thread's flux slot of field b in direction d: f[d] + b * BLK
    int f[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) f[d] = d * NF * BLK + el * EW + dir_slot<NQ, T>(d, i, j, k);
    const int64_t M = I.M;
    T *qv = static_cast<T *>(I.q);
    const T dtt = static_cast<T>(dt);
    T grav;
    if constexpr (MIXED)
        grav = I.mp.grav;
    else
        grav = I.np.eos.grav;

    for (int64_t base = e0; base < e0 + count; base += EPP) {
        const int npass = (int)((e0 + count - base) < EPP ? (e0 + count - base) : EPP);
        const bool active = el < npass;
        const int64_t node = (base + (active ? el : 0)) * N3 + p;
        // q and the scheme's dq of this thread's point (registers in FP64,
        // shared memory in the mixed mode), and the mixed mode's per-point
        // constants, kept for all stages
        T qr[kFields], dqr[kFields];
        T *sQ = sF + tile_flux_words<T, NF>() + l;   // [b * kThreads], mixed: every field
        T *sD = sQ + NF * kThreads;                  // FP64 (TR): the tracers
        T *sG = sD + NF * kThreads;                  // g (9), Jinv; mixed only
        // the tracers' q and dq (TR): shared memory in both precisions
        auto QT = [&](int t) -> T & {
            if constexpr (MIXED) return sQ[(kFields + t) * kThreads];
            else return sF[tile_flux_words<T, NF>() + t * kThreads + l];
        };
        auto DQT = [&](int t) -> T & {
            if constexpr (MIXED) return sD[(kFields + t) * kThreads];
            else return sF[tile_flux_words<T, NF>() + (NTR + t) * kThreads + l];
        };
        auto Q = [&](int b) -> T & {
            if constexpr (MIXED) return sQ[b * kThreads]; else return qr[b];
        };
        auto DQ = [&](int b) -> T & {
            if constexpr (MIXED) return sD[b * kThreads]; else return dqr[b];
        };
#pragma unroll
        for (int b = 0; b < kFields; ++b) {
            Q(b) = active ? qv[b * M + node] : T(0);
            DQ(b) = T(0);
        }
        if (!active) Q(0) = MIXED ? T(0) : T(1);   // idle threads hold a harmless state
        if constexpr (TR) {
#pragma unroll
            for (int t = 0; t < NTR; ++t) {
                QT(t) = active && kFields + t < nf ? qv[(kFields + t) * M + node] : T(0);
                DQT(t) = T(0);
            }
        }
        float th0 = 0.f, rho0 = 0.f;
        EosRef32 er{0.f, 0.f};
        if constexpr (MIXED) {
            if (active) {
                th0 = __ldg(I.mgeo.theta_ref + node);
                rho0 = __ldg(I.mgeo.rho_ref + node);
                if (th0 > 0.f) er = eos_reference_f32(th0, I.mp);
#pragma unroll
                for (int s2 = 0; s2 < 9; ++s2) sG[s2 * kThreads] = __ldg(I.mgeo.g[s2] + node);
                sG[9 * kThreads] = __ldg(I.mgeo.Jinv + node);
            }
        }

        for (int step = 0; step < nsteps; ++step) {
#pragma unroll 1
            for (int st = 0; st < 5; ++st) {
                // Phase 3 reads and phase 1 writes only the thread's own
                // point's flux slots (and its own state words), so within a
                // pass the next stage's phase 1 needs no barrier after phase 3.
                // The first stage of a pass takes one: the previous pass or
                // work item (possibly another order) gave its slots to other
                // threads.
                if (step == 0 && st == 0) __syncthreads();
                // ---- phase 1: p', fluxes ------------------------------
                if (active) {
                    T q[kFields];
#pragma unroll
                    for (int b = 0; b < kFields; ++b) q[b] = Q(b);
                    T rho, Th, pp, g[9];
                    if constexpr (MIXED) {
#pragma unroll
                        for (int s2 = 0; s2 < 9; ++s2) g[s2] = sG[s2 * kThreads];
                        rho = rho0 + q[0];
                        Th = th0 + q[4];
                        pp = pressure_perturbation_f32(q[4], th0, er, I.mp);
                    } else {
#pragma unroll
                        for (int s2 = 0; s2 < 9; ++s2) g[s2] = __ldg(I.geo.g[s2] + node);
                        rho = q[0];
                        Th = q[4];
                        pp = pressure_perturbation(Th, __ldg(I.geo.theta_ref + node),
                                                   __ldg(I.geo.w + node), __ldg(I.geo.A + node), I.np);
                    }
                    T rinv;
                    if constexpr (MIXED)
                        rinv = __frcp_rn(rho);   // the correctly rounded 1/rho, as 1.0f / rho
                    else
                        rinv = __drcp_rn(rho);   // the correctly rounded 1/rho, as 1.0 / rho
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        const T g1 = g[3 * d], g2 = g[3 * d + 1], g3 = g[3 * d + 2];
                        const T v = fma(g3, q[3], fma(g2, q[2], g1 * q[1]));
                        const T u = v * rinv;
                        T *F = sF + f[d];
                        F[0 * BLK] = v;
                        F[1 * BLK] = fma(q[1], u, g1 * pp);
                        F[2 * BLK] = fma(q[2], u, g2 * pp);
                        F[3 * BLK] = fma(q[3], u, g3 * pp);
                        F[4 * BLK] = Th * u;
                        if constexpr (TR) {
#pragma unroll
                            for (int t = 0; t < NTR; ++t)
                                if (kFields + t < nf) F[(kFields + t) * BLK] = QT(t) * u;   // Q u_d
                        }
                    }
                }
                __syncthreads();
                // ---- phase 2: sweeps, one line per task ------------------
#pragma unroll 1
                for (int t = l; t < TASKS; t += kThreads) {
                    const int bd = t / (EPP * NL), rem = t % (EPP * NL);
                    const int e = rem / NL, line = rem % NL;
                    if (e < npass && (!TR || bd % NF < nf)) {
                        if constexpr (MIXED)
                            sweep_line<NQ>(sF + bd * BLK + e * EW, line, c_sweep32[NQ]);
                        else
                            sweep_line<NQ>(sF + bd * BLK + e * EW, line, c_sweep64[NQ]);
                    }
                }
                // FP64: J^-1 and rho_ref loaded before the barrier, so that
                // their latency passes while the last sweeps finish
                T jinv_g = T(0), rho_ref_g = T(0);
                if constexpr (!MIXED) {
                    if (active) {
                        jinv_g = __ldg(I.geo.Jinv + node);
                        rho_ref_g = __ldg(I.geo.rho_ref + node);
                    }
                }
                __syncthreads();
                // ---- phase 3: rhs, stage update ------------------------
                if (active) {
                    const T a = sco[st], bcoef = sco[5 + st];
                    T jinv, drho;   // drho: rho - rho_ref of this stage's state, before the update
                    if constexpr (MIXED) {
                        jinv = sG[9 * kThreads];
                        drho = Q(0);
                    } else {
                        jinv = jinv_g;
                        drho = Q(0) - rho_ref_g;
                    }
#pragma unroll
                    for (int b = 0; b < kFields; ++b) {
                        const T R = sF[f[0] + b * BLK] + sF[f[1] + b * BLK] + sF[f[2] + b * BLK];
                        T rhs = -jinv * R;
                        if (b == 3) rhs = fma(-drho, grav, rhs);
                        const T d = fma(a, DQ(b), dtt * rhs);
                        DQ(b) = d;
                        Q(b) = fma(bcoef, d, Q(b));
                    }
                    if constexpr (TR) {
#pragma unroll
                        for (int t = 0; t < NTR; ++t) {
                            if (kFields + t >= nf) break;
                            const int b = kFields + t;
                            const T R = sF[f[0] + b * BLK] + sF[f[1] + b * BLK] + sF[f[2] + b * BLK];
                            const T d = fma(a, DQT(t), dtt * (-jinv * R));
                            DQT(t) = d;
                            QT(t) = fma(bcoef, d, QT(t));
                        }
                    }
                }
            }
        }
        if (active) {
#pragma unroll
            for (int b = 0; b < kFields; ++b) qv[b * M + node] = Q(b);
            if constexpr (TR) {
#pragma unroll
                for (int t = 0; t < NTR; ++t)
                    if (kFields + t < nf) qv[(kFields + t) * M + node] = QT(t);
            }
        }
    }
}

}  // namespace

}  // namespace numa
