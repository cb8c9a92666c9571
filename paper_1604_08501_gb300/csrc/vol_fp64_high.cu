// Element volume term for orders N = 8..15 (Nq = 9..16), native FP64 and
// mixed precision.
//
// The operation of vol_fp64.cu (Sec. 2, Eq. (2); sign and flux form of the
// paper's r/s subroutines, Sec. 3), for the high orders of the paper's Nq
// study (Sec. 4, Table 2, Nq up to 16).  An element of Nq = 16 has 4096 points: more
// than a CTA has threads, and its fifteen FP64 flux arrays (491 KB) exceed
// shared memory.  So:
//  * one CTA per element with three threads per (i, j) column (four in FP32
//    at Nq >= 15), each looping over its share of the k-planes, as the
//    paper's kernels own (i, j) lanes and loop over k;
//  * one pass per group of fields (one field in FP64; as many as shared
//    memory holds in FP32): their flux arrays into shared memory (3 Nq^2
//    lines per field: 16 slots in FP64, an odd number >= Nq in FP32), the D
//    sweeps in place (even-odd split, lines dealt out to the threads), and the
//    rhs of the thread's points straight to HBM;
//  * FP64: the first pass also keeps the contravariant velocities u_d and p'
//    of all points in shared memory (4 Nq^3 values), from which each later
//    pass forms its field's fluxes;
//  * FP32: the first pass forms the fluxes of every field; those beyond the
//    first group wait in tensor memory (tcgen05.st, one TMEM lane per thread)
//    until their pass copies them into shared memory (tcgen05.ld), so no later
//    pass reads the state or the metrics again, and without u_d and p' the
//    groups are large (five fields: four per group at Nq = 12, 13 and 16, one
//    pass at the other orders; a separate form for tracers); after its first
//    pass each CTA prefetches the element of the next wave to L2.
// Shared memory at Nq = 16: 224 KB in FP64 (every operation FP64; bound by the
// FP64 pipe like the low orders), 204 KB in the mixed mode (FP32 perturbation
// state and arithmetic as vol_mixed.cu).
#include <cuda_runtime.h>

#include <type_traits>

#include "bulk_copy.cuh"
#include "element_sweep.cuh"
#include "eos.cuh"
#include "numa_internal.h"
#include "tcgen05.cuh"

namespace numa {

namespace {

// T: double (NUMA_FP64) or float (NUMA_MIXED: FP32 perturbation state
// (rho', U, Theta', tracers), FP32 geometry, p' from Theta' without
// cancellation).

// Threads: TPC per (i, j) column, each owning a slab of KS = ceil(Nq/TPC)
// k-planes in the point phases; the sweep phase deals the 3 Nq^2 lines of
// each field of a group out to the threads.  TPC = 3 (one line per thread and
// field); 4 for the FP32 instances at Nq >= 15, which fill the 1024 threads of
// the one CTA their shared memory allows per SM.
template <int NQ, typename T>
__host__ __device__ constexpr int high_tpc() {
    if (sizeof(T) == 4 && NQ >= 15 && 4 * NQ * NQ <= 1024) return 4;
    return 3;
}

// FP32: rounded up to whole warps, since tensor-memory accesses are
// warp-wide; the extra threads own no points and sweep no lines.
template <int NQ, typename T>
__host__ __device__ constexpr int high_threads() {
    return sizeof(T) == 4 ? (high_tpc<NQ, T>() * NQ * NQ + 31) / 32 * 32
                          : high_tpc<NQ, T>() * NQ * NQ;
}

// Flux slot of point (i, j, k) in direction d.  A warp of the point phases is
// 32 consecutive (i, j) columns at one k.  For FP32 at Nq = 16 (lines of 17
// slots) r line k + 16 j and s line 2 i + (k & 1) + 32 (k >> 1) put the warp on
// 32 distinct banks in every direction, where the natural numbering of
// dir_slot takes two wavefronts in r and s; the sweeps only need a bijection
// of lines.  At Nq = 12 the s numbering 2 i + (k & 1) + 24 (k >> 1) cut the
// counted wavefronts by a third but measured no faster (the kernel is bound by
// global-load latency), so the other orders keep dir_slot's numbering.
template <int NQ, typename T>
__device__ __forceinline__ int high_slot(int d, int i, int j, int k) {
    if constexpr (NQ == 16 && sizeof(T) == 4) {
        if (d == 0) return slot<NQ, T>(k + 16 * j, i);
        if (d == 1) return slot<NQ, T>(2 * i + (k & 1) + 32 * (k >> 1), j);
        return slot<NQ, T>(16 * j + i, k);
    } else {
        return dir_slot<NQ, T>(d, i, j, k);
    }
}

// The FP32 instance comes in two forms per order, chosen at launch by the
// handle's field count: NF = 5 (five fields) and NF = 8 (six to eight:
// tracers).  FP64 has one form, NF = 8.
//
// Fields per pass.  FP64: one (the flux arrays of one field already take
// 98 KB at Nq = 16).  FP32: as many as a shared-memory budget holds, but at
// least as many as leave the other NF - G fields room in the tensor memory of
// the CTAs of one SM (256 columns each with two CTAs per SM, 512 with one).
// The budget is 226 KB with one CTA per SM; with two, 113 KB (all of it) for
// NF = 8 but 100 KB for NF = 5, whose parked fields must also fit the
// registers of pass 0 (high_hold).  At Nq = 12, five fields: one 110 KB group
// measured 27.9 GDOF/s against 31.7 for four fields (88 KB) with the fifth
// parked, the larger shared-memory carveout leaving the L1 too little room
// for the loads in flight; eight fields: 25.4 against 19.8 for groups of
// four and four (the second group's four parked fields waiting on global
// loads: long-scoreboard stalls 4.2 against 7.4 per issue).
// Parked fluxes a thread may hold in registers over its k-planes before it
// stores them (pass 0 below): one field's at Nq = 12, 13 and 16.  Two fields'
// (24 values) at Nq = 16 with three fields per group measured slower (26.2
// against 27.7 GDOF/s for four fields per group and one held).
template <int NQ, typename T>
__host__ __device__ constexpr int high_hold() {
    return 16;
}

template <int NQ, typename T, int NF>
__host__ __device__ constexpr int high_tmem_need(int g) {
    const int ks = (NQ + high_tpc<NQ, T>() - 1) / high_tpc<NQ, T>();
    const int need = (high_threads<NQ, T>() / 32 + 3) / 4 * ks * 3 * (NF - g);
    int c = 32;
    while (c < need) c *= 2;
    return need <= 0 ? 0 : c;
}

template <int NQ, typename T, int NF>
__host__ __device__ constexpr int high_group() {
    if constexpr (sizeof(T) == 8) {
        return 1;
    } else {
        constexpr bool two = 2 * high_threads<NQ, T>() <= 1024;
        constexpr size_t per = sizeof(T) * 3 * NQ * NQ * line_stride<NQ, T>();   // one field's fluxes
        constexpr size_t budget = (two ? (NF > kFields ? 113 : 100) : 226) * 1024;
        int g = (int)(budget / per);
        g = g < 1 ? 1 : (g > NF ? NF : g);
        while (g < NF && high_tmem_need<NQ, T, NF>(g) > (two ? 256 : 512)) ++g;
        if (NF == kFields) {   // no more parked fields than registers hold (pass 0)
            const int ks = (NQ + high_tpc<NQ, T>() - 1) / high_tpc<NQ, T>();
            const int lo = NF - high_hold<NQ, T>() / (3 * ks);
            g = g < lo ? lo : g;
        }
        return g;
    }
}

template <int NQ, typename T, int NF>
__host__ __device__ constexpr size_t high_smem_bytes() {
    return sizeof(T) * ((sizeof(T) == 8 ? 4 * NQ * NQ * NQ : 0) +
                        high_group<NQ, T, NF>() * 3 * NQ * NQ * line_stride<NQ, T>());
}

// CTAs per SM the register budget is sized for: two where two CTAs' shared
// memory fits an SM and still leaves 64 registers per thread, else one.
template <int NQ, typename T, int NF>
__host__ __device__ constexpr int high_min_ctas() {
    return (2 * (high_smem_bytes<NQ, T, NF>() + 1024) <= 228 * 1024 &&
            2 * high_threads<NQ, T>() <= 1024)
               ? 2
               : 1;
}

// Tensor memory of the FP32 instance: per warp, the fluxes of the fields
// beyond the first group for its threads' points, 3 (NF - G) per point
// (column (f KS + kk) 3 + d for parked field f, k-plane kk of the slab,
// direction d); the warps of one lane quarter (warp % 4) side by side.  The
// allocation (a power of two >= 32 columns) is sized for NF fields and made
// only when the launch has fields beyond the first group.
template <int NQ, typename T, int NF>
__host__ __device__ constexpr int high_park_cols() {
    constexpr int KS = (NQ + high_tpc<NQ, T>() - 1) / high_tpc<NQ, T>();
    return sizeof(T) == 4 ? KS * 3 * (NF - high_group<NQ, T, NF>()) : 0;
}

template <int NQ, typename T, int NF>
__host__ __device__ constexpr int high_tmem_cols() {
    return sizeof(T) == 4 ? high_tmem_need<NQ, T, NF>(high_group<NQ, T, NF>()) : 0;
}

template <typename T> struct HighTypes;
template <> struct HighTypes<double> { using Geo = DeviceGeometry; using Params = HighParams; };
template <> struct HighTypes<float> { using Geo = MixedGeometry; using Params = HighParams32; };

template <int NQ, typename T, int NF>
__global__ void __launch_bounds__((high_threads<NQ, T>()), (high_min_ctas<NQ, T, NF>()))
vol_rhs_high_kernel(typename HighTypes<T>::Geo geo, typename HighTypes<T>::Params P,
                    const T *__restrict__ q, T *__restrict__ rhs, int64_t M, int64_t e0, int nf,
                    int64_t e_end, int64_t ahead) {
    constexpr bool MIXED = sizeof(T) == 4;
    constexpr int NL = NQ * NQ;      // columns; lines per direction
    constexpr int N3 = NQ * NL;
    constexpr int FB = NL * line_stride<NQ, T>();   // one direction's flux block (padded lines)
    constexpr int TPC = high_tpc<NQ, T>();
    constexpr int NT = high_threads<NQ, T>();
    constexpr int KS = (NQ + TPC - 1) / TPC; // k-planes per slab
    constexpr int G = high_group<NQ, T, NF>();
    constexpr int PC = high_park_cols<NQ, T, NF>();     // TMEM columns per warp
    constexpr int TC = high_tmem_cols<NQ, T, NF>();
    constexpr int PL = PC > 0 ? NF - G : 1;   // fields a point can park
    static_assert(TC <= 512 / high_min_ctas<NQ, T, NF>(), "tensor memory of the CTAs of one SM");
    // k-loop unrolling: full in FP32 (registers to spare, more loads in
    // flight), two planes in FP64 (register budget)
    constexpr int KU = MIXED ? KS : 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint32_t s_tmem;
    T *sU = reinterpret_cast<T *>(smem_raw);   // FP64: u_d of every point: [d][k][j][i]
    T *sP = sU + 3 * N3;                       // FP64: p' of every point: [k][j][i]
    T *sF = MIXED ? sU : sU + 4 * N3;          // fluxes of a group: [field][d][line][slot]

    const int t = threadIdx.x;
    const int c = t % NL, slab = t / NL;   // slab == TPC: a padding thread
    const int i = c % NQ, j = c / NQ;
    const int kb = slab * KS;                          // first k-plane of the slab
    const int64_t node0 = (e0 + blockIdx.x) * N3 + c;  // point (i, j, 0); + k NL

    // FP32: the arrays of the element `ahead` CTAs later (the next wave of
    // resident CTAs) toward L2, where its first pass then finds them.  Only
    // where an element's array is whole 16-byte units (even Nq).
    auto prefetch_next = [&]() {
        if constexpr (MIXED && (N3 * sizeof(T)) % 16 == 0) {
            const int64_t ea = e0 + blockIdx.x + ahead;
            if (t == 0 && ahead > 0 && ea < e_end) {
                const int64_t off = ea * N3;
                constexpr uint32_t B = N3 * sizeof(T);
                for (int b = 0; b < nf; ++b) prefetch_l2(q + b * M + off, B);
#pragma unroll
                for (int a = 0; a < 9; ++a) prefetch_l2(geo.g[a] + off, B);
                prefetch_l2(geo.Jinv + off, B);
                prefetch_l2(geo.rho_ref + off, B);
                prefetch_l2(geo.theta_ref + off, B);
            }
        }
    };
    // Issued after the first pass, when the CTA's own loads are done: at the
    // start it competed with them (Nq = 16, one CTA per SM: 24.7 GDOF/s
    // against 26.8 without a prefetch and 30.7 after the first pass; Nq = 12:
    // 30.3 against 27.4 and 31.7).

    // FP32 with fields beyond the first group: their fluxes wait in TMEM
    const bool park = PC > 0 && nf > G;   // uniform over the CTA
    uint32_t tpark = 0;                   // this thread's lane, its warp's first column
    if constexpr (PC > 0) {
        if (t < 32) {
            if (park) tc::tmem_alloc(&s_tmem, TC);
            else tc::tmem_relinquish();   // lets a second CTA onto the SM
        }
        if (park) {
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
            const int w = t >> 5;
            tpark = s_tmem + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)((w >> 2) * PC);
        }
    }

    // Flux of field b in direction d at a point: F_d[rho] = g_d . U,
    // F_d[U_a] = U_a u_d + g_{ad} p', F_d[Theta] = Theta u_d, tracers Q u_d.
    // ---- pass 0: the fluxes of the first group (FP64: and u_d, p'; FP32:
    // and the fluxes of LP more fields, parked in TMEM).  Where they fit
    // (high_hold) the parked fluxes of all the slab's planes stay in
    // registers until after the planes, so that the compiler can still issue
    // every plane's loads at once: a TMEM store between two planes keeps the
    // later plane's loads behind it (measured: 22.7 against 25.7 GDOF/s at
    // Nq = 16 with one parked field).  Otherwise they are stored plane by
    // plane.
    auto pass0 = [&](auto lp) {
        constexpr int LP = decltype(lp)::value;
        constexpr bool HOLD = LP > 0 && 3 * LP * KS <= high_hold<NQ, T>();
        T hold[HOLD ? 3 * LP * KS : 1];
#pragma unroll(KU)
        for (int kk = 0; kk < KS; ++kk) {
            const int k = kb + kk;
            T pk[3 * (LP > 0 ? LP : 1)];   // this point's parked fluxes
#pragma unroll
            for (int x = 0; x < 3 * (LP > 0 ? LP : 1); ++x) pk[x] = T(0);
            if (k < NQ) {
                const int64_t node = node0 + k * NL;
                const T U[3] = {q[M + node], q[2 * M + node], q[3 * M + node]};
                T rinv, pp, Th;
                if constexpr (MIXED) {
                    const float th0 = geo.theta_ref[node];
                    pp = pressure_perturbation_f32(q[4 * M + node], th0, P);
                    rinv = __frcp_rn(geo.rho_ref[node] + q[node]);
                    Th = th0 + q[4 * M + node];
                } else {
                    pp = pressure_perturbation(q[4 * M + node], geo.theta_ref[node], geo.w[node],
                                               geo.A[node], P);
                    rinv = __drcp_rn(q[node]);
                    Th = q[4 * M + node];
                    sP[k * NL + c] = pp;
                }
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const T g[3] = {geo.g[3 * d][node], geo.g[3 * d + 1][node],
                                    geo.g[3 * d + 2][node]};
                    const T v = fma(g[2], U[2], fma(g[1], U[1], g[0] * U[0]));
                    const T u = v * rinv;
                    if constexpr (!MIXED) sU[d * N3 + k * NL + c] = u;
                    const int sl = high_slot<NQ, T>(d, i, j, k);
#pragma unroll
                    for (int b = 0; b < G + LP; ++b) {
                        if (b >= nf) break;
                        T F;
                        if (b == 0) F = v;
                        else if (b < 4) F = fma(U[b - 1], u, g[b - 1] * pp);
                        else if (b == 4) F = Th * u;
                        else F = q[b * M + node] * u;
                        if (b < G) sF[(b * 3 + d) * FB + sl] = F;
                        else pk[(b - G) * 3 + d] = F;
                    }
                }
            }
            if constexpr (HOLD) {
#pragma unroll
                for (int x = 0; x < 3 * LP; ++x) hold[(x / 3) * 3 * KS + 3 * kk + x % 3] = pk[x];
            } else if constexpr (LP > 0) {   // every lane: the stores are warp-wide
#pragma unroll
                for (int f = 0; f < LP; ++f) {
                    if (G + f >= nf) break;
#pragma unroll
                    for (int d = 0; d < 3; ++d)
                        tc::tmem_st1(tpark + (f * KS + kk) * 3 + d, __float_as_uint(pk[f * 3 + d]));
                }
            }
        }
        if constexpr (HOLD) {
#pragma unroll
            for (int x = 0; x < 3 * LP * KS; ++x) {
                if (G + x / (3 * KS) >= nf) break;
                tc::tmem_st1(tpark + x, __float_as_uint(hold[x]));
            }
        }
        if constexpr (LP > 0) tc::tmem_st_wait();
    };
    if constexpr (PC > 0) {
        if (!park) pass0(std::integral_constant<int, 0>{});
        else if (nf == G + 1) pass0(std::integral_constant<int, 1>{});
        else if (nf == G + 2) pass0(std::integral_constant<int, PL < 2 ? PL : 2>{});
        else pass0(std::integral_constant<int, PL>{});
    } else {
        pass0(std::integral_constant<int, 0>{});
    }

#pragma unroll 1
    for (int b0 = 0; b0 < nf; b0 += G) {   // groups of G fields: 5 fields, then the tracers
        const int gn = nf - b0 < G ? nf - b0 : G;
        if (b0 > 0) {
            // No barrier after the previous group's combination: it read, and
            // this group's fluxes are written to, only the thread's own
            // points' slots (a bijection per direction).
            if constexpr (MIXED) {
                // the group's parked fluxes from TMEM into the flux arrays
                if constexpr (PC > 0) {
#pragma unroll(KU)
                    for (int kk = 0; kk < KS; ++kk) {
                        const int k = kb + kk;
                        uint32_t v[3 * G];
#pragma unroll
                        for (int gl = 0; gl < G; ++gl) {
                            if (gl >= gn) break;
#pragma unroll
                            for (int d = 0; d < 3; ++d)
                                v[gl * 3 + d] = tc::tmem_ld1(tpark + ((b0 - G + gl) * KS + kk) * 3 + d);
                        }
                        tc::tmem_ld_wait_all();
                        if (k < NQ) {
#pragma unroll
                            for (int gl = 0; gl < G; ++gl) {
                                if (gl >= gn) break;
#pragma unroll
                                for (int d = 0; d < 3; ++d)
                                    sF[(gl * 3 + d) * FB + high_slot<NQ, T>(d, i, j, k)] =
                                        __uint_as_float(tc::after_wait(v[gl * 3 + d]));
                            }
                        }
                    }
                }
            } else {
#pragma unroll(KU)
                for (int kk = 0; kk < KS; ++kk) {
                    const int k = kb + kk;
                    if (k < NQ) {
                        const int64_t node = node0 + k * NL;
#pragma unroll
                        for (int gl = 0; gl < G; ++gl) {
                            if (gl >= gn) break;
                            const int b = b0 + gl;
                            const T qb = q[b * M + node];
#pragma unroll
                            for (int d = 0; d < 3; ++d) {
                                const T u = sU[d * N3 + k * NL + c];
                                T F = qb * u;
                                if (b < 4) {
                                    // g_{b,d} by selection: a run-time index into the
                                    // parameter's pointer array would copy it to local memory
                                    const T *gp = b == 1 ? geo.g[3 * d]
                                                         : (b == 2 ? geo.g[3 * d + 1] : geo.g[3 * d + 2]);
                                    F = fma(qb, u, gp[node] * sP[k * NL + c]);
                                }
                                sF[(gl * 3 + d) * FB + high_slot<NQ, T>(d, i, j, k)] = F;
                            }
                        }
                    }
                }
            }
        }
        __syncthreads();
        if (b0 == 0) prefetch_next();
        // ---- sweeps: line c of direction `slab`, for each field of the group
        // (TPC = 3), or the group's 3 Nq^2 lines per field dealt out in turn
        if constexpr (TPC == 3) {
            if (slab < 3) {
#pragma unroll 1
                for (int gl = 0; gl < gn; ++gl) sweep_line<NQ>(sF + (gl * 3 + slab) * FB, c, P);
            }
        } else {
#pragma unroll 1
            for (int item = t; item < gn * 3 * NL; item += NT)
                sweep_line<NQ>(sF + (item / NL) * FB, item % NL, P);
        }
        // FP32: J^-1 and rho' of the thread's points, loaded before the
        // barrier so that their latency passes while the CTA's last sweeps
        // finish (Nq = 12 / 16: 34.9 / 33.8 GDOF/s against 31.8 / 30.7 loaded
        // after it; in FP64 it cost 3.6 % at Nq = 16, and FP64 loads after it)
        T jv[KS], rv[KS];
        if constexpr (MIXED) {
            const bool grav = b0 <= 3 && 3 < b0 + gn;   // U3 in this group
#pragma unroll
            for (int kk = 0; kk < KS; ++kk) {
                jv[kk] = rv[kk] = T(0);
                const int k = kb + kk;
                if (k < NQ) {
                    const int64_t node = node0 + k * NL;
                    jv[kk] = geo.Jinv[node];
                    if (grav) rv[kk] = q[node];   // rho' is the stored state
                }
            }
        }
        __syncthreads();
        // ---- rhs of the group's fields: -Jinv (S_r + S_s + S_t), gravity on U3
#pragma unroll(KU)
        for (int kk = 0; kk < KS; ++kk) {
            const int k = kb + kk;
            if (k < NQ) {
                const int64_t node = node0 + k * NL;
                const T jinv = MIXED ? jv[kk] : geo.Jinv[node];
                const int s0 = high_slot<NQ, T>(0, i, j, k), s1 = high_slot<NQ, T>(1, i, j, k),
                          s2 = high_slot<NQ, T>(2, i, j, k);
#pragma unroll
                for (int gl = 0; gl < G; ++gl) {
                    if (gl >= gn) break;
                    const int b = b0 + gl;
                    const T *F = sF + gl * 3 * FB;
                    T v = -jinv * (F[s0] + F[FB + s1] + F[2 * FB + s2]);
                    if (b == 3) {
                        if constexpr (MIXED)
                            v = fma(-rv[kk], P.grav, v);
                        else
                            v = fma(-(q[node] - geo.rho_ref[node]), P.eos.grav, v);
                    }
                    rhs[b * M + node] = v;
                }
            }
        }
    }
    if constexpr (PC > 0) {
        if (park) {   // every TMEM load has completed (waited above)
            tc::fence_before_sync();
            __syncthreads();
            if (t < 32) {
                tc::fence_after_sync();
                tc::tmem_dealloc(s_tmem, TC);
            }
        }
    }
}

template <int NQ, typename T, int NF, typename Geo, typename Params>
cudaError_t launch_high_form(ElemRange r, int nf, const Geo &geo, const Params &P, const T *q,
                             T *rhs, int num_sms, cudaStream_t s) {
    constexpr size_t smem = high_smem_bytes<NQ, T, NF>();
    cudaError_t e = cudaFuncSetAttribute(vol_rhs_high_kernel<NQ, T, NF>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int64_t ahead = 0;   // FP64: no prefetch (bound by the FP64 pipe)
    if (sizeof(T) == 4 && num_sms > 0) {
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, vol_rhs_high_kernel<NQ, T, NF>,
                                                          high_threads<NQ, T>(), smem);
        if (e != cudaSuccess) return e;
        ahead = (int64_t)num_sms * (per_sm > 0 ? per_sm : 1);
    }
    vol_rhs_high_kernel<NQ, T, NF><<<(unsigned)r.count, high_threads<NQ, T>(), smem, s>>>(
        geo, P, q, rhs, r.M, r.e0, nf, r.e0 + r.count, ahead);
    return cudaGetLastError();
}

// FP32: the five-field form for five fields where its group differs from
// the eight-field form's, else the eight-field form (at Nq = 16 both have
// groups of four, and the five-field form measured 29.1 against 30.7 GDOF/s);
// FP64: the one form.
template <int NQ, typename T, typename Geo, typename Params>
cudaError_t launch_high(ElemRange r, int nf, const Geo &geo, const Params &P, const T *q, T *rhs,
                        int num_sms, cudaStream_t s) {
    if constexpr (sizeof(T) == 4 && high_group<NQ, T, kFields>() != high_group<NQ, T, kMaxFields>()) {
        if (nf == kFields)
            return launch_high_form<NQ, T, kFields>(r, nf, geo, P, q, rhs, num_sms, s);
    }
    return launch_high_form<NQ, T, kMaxFields>(r, nf, geo, P, q, rhs, num_sms, s);
}

template <typename T, typename Geo, typename Params>
cudaError_t launch_high_order(int N, int nf, ElemRange r, const Geo &geo, const Params &P,
                              const T *q, T *rhs, int num_sms, cudaStream_t s) {
    if (r.count <= 0) return cudaSuccess;
    if (nf < kFields || nf > kMaxFields) return cudaErrorInvalidValue;
    switch (N) {
        case 8: return launch_high<9>(r, nf, geo, P, q, rhs, num_sms, s);
        case 9: return launch_high<10>(r, nf, geo, P, q, rhs, num_sms, s);
        case 10: return launch_high<11>(r, nf, geo, P, q, rhs, num_sms, s);
        case 11: return launch_high<12>(r, nf, geo, P, q, rhs, num_sms, s);
        case 12: return launch_high<13>(r, nf, geo, P, q, rhs, num_sms, s);
        case 13: return launch_high<14>(r, nf, geo, P, q, rhs, num_sms, s);
        case 14: return launch_high<15>(r, nf, geo, P, q, rhs, num_sms, s);
        case 15: return launch_high<16>(r, nf, geo, P, q, rhs, num_sms, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_vol_rhs_fp64_high(int N, int nf, ElemRange r, const DeviceGeometry &geo,
                                     const HighParams &P, const double *q, double *rhs,
                                     cudaStream_t s) {
    return launch_high_order<double>(N, nf, r, geo, P, q, rhs, 0, s);
}

cudaError_t launch_vol_rhs_mixed_high(int N, int nf, ElemRange r, const MixedGeometry &geo,
                                      const HighParams32 &P, const float *q, float *rhs,
                                      int num_sms, cudaStream_t s) {
    return launch_high_order<float>(N, nf, r, geo, P, q, rhs, num_sms, s);
}

}  // namespace numa
