// Batched explicit time integration of dq/dt = v(q), v the element volume term
// (Sec. 2, Eq. (2)), for many independent instances of mixed order and size in
// one persistent launch.
//
// Scheme: the five-stage fourth-order 2N-storage Runge-Kutta method of
// Carpenter and Kennedy (NASA TM-109112, 1994): per stage s,
//   dq <- A_s dq + dt v(q),  q <- q + B_s dq,   dq = 0 at the start.
// The paper frames the volume term as the rate function of such an explicit
// solver (Sec. 2); the scheme is the benchmark's choice.
//
// The volume term couples only the points of one element.  So a CTA can take
// a tile of elements through all 5 * nsteps stages with q and dq of its
// points in registers: q is read from and written to HBM once, and there is
// no grid-wide synchronisation.  The tile's geometry (56 KB in FP64 for one
// Nq = 8 element) is re-read every stage; after the first stage it comes from
// L2.  Each stage
// runs the same three phases as the single-evaluation kernels: fluxes by point
// into shared memory, even-odd D sweeps by line in place, combination by point.
//
// Work items (instance, element range) are claimed dynamically through an
// atomic counter.  Orders are mixed within one launch: a CTA of 512 threads
// holds 512 / Nq^3 elements per pass.  Tile sizes (elements per item) come
// from the batch's autotuner.
#include <cuda_runtime.h>

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

template <bool MIXED>
__global__ void __launch_bounds__(kThreads, 1)
batch_lsrk_kernel(const BatchInstance *__restrict__ inst, const BatchItem *__restrict__ items,
                  int num_items, int *counter, LsrkCoef co, int nsteps, double dt) {
    extern __shared__ __align__(16) double smem_d[];
    __shared__ BatchInstance sI;
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= num_items) break;
        const BatchItem item = items[it];
        {
            // instance description into shared memory, word by word
            const int *src = reinterpret_cast<const int *>(inst + item.instance);
            int *dst = reinterpret_cast<int *>(&sI);
            for (int w = threadIdx.x; w < (int)(sizeof(BatchInstance) / sizeof(int)); w += kThreads)
                dst[w] = src[w];
        }
        __syncthreads();
        switch (item.nq) {
            case 2: run_tile<2, MIXED>(sI, item.e0, item.count, co, nsteps, dt, smem_d); break;
            case 3: run_tile<3, MIXED>(sI, item.e0, item.count, co, nsteps, dt, smem_d); break;
            case 4: run_tile<4, MIXED>(sI, item.e0, item.count, co, nsteps, dt, smem_d); break;
            case 5: run_tile<5, MIXED>(sI, item.e0, item.count, co, nsteps, dt, smem_d); break;
            case 6: run_tile<6, MIXED>(sI, item.e0, item.count, co, nsteps, dt, smem_d); break;
            case 7: run_tile<7, MIXED>(sI, item.e0, item.count, co, nsteps, dt, smem_d); break;
            case 8: run_tile<8, MIXED>(sI, item.e0, item.count, co, nsteps, dt, smem_d); break;
            default: break;
        }
        __syncthreads();   // sI and s_item are rewritten by the next claim
    }
}

}  // namespace

cudaError_t prepare_batch_lsrk() {
    return cudaFuncSetAttribute(batch_lsrk_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(double) * 3 * kFields * kThreads));
}

cudaError_t launch_batch_lsrk(bool mixed, const BatchInstance *inst, const BatchItem *items,
                              int num_items, int *counter, const LsrkCoef &co, int nsteps,
                              double dt, int grid, cudaStream_t s) {
    if (num_items <= 0 || nsteps <= 0) return cudaSuccess;
    if (mixed)
        batch_lsrk_kernel<true><<<grid, kThreads, sizeof(float) * 3 * kFields * kThreads, s>>>(
            inst, items, num_items, counter, co, nsteps, dt);
    else
        batch_lsrk_kernel<false><<<grid, kThreads, sizeof(double) * 3 * kFields * kThreads, s>>>(
            inst, items, num_items, counter, co, nsteps, dt);
    return cudaGetLastError();
}

}  // namespace numa
