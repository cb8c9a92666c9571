// FP64-accurate element volume term for N = 1..7 (Nq = 2..8) in double-float
// arithmetic on the FP32 pipes.
//
// Same operation as vol_fp64.cu (Sec. 2, Eq. (2); flux form and sign of the
// paper's r/s subroutines, Sec. 3), evaluated with about 48 significant bits
// instead of 53.  Every quantity is carried as a double-float.  Geometry and
// the reference state are stored pre-split as (h, l) float pairs by the
// handle.  The state is split with integer operations, and each rhs value
// costs one FP64 add.  Accuracy against an FP64 evaluation is about 1e-14,
// normwise.
//
// One CTA (Nq^3 threads) per element, in three phases:
//  1. Thread per point: the pressure perturbation p' (series in
//     x = Theta'/Theta_ref, below), 1/rho, and the fifteen contravariant
//     fluxes of the point.  Each flux goes into a per-(direction, field) buffer
//     in shared memory, laid out line by line (the paper's per-k-slice flux
//     precompute, Sec. 3, opt. level 5, extended to whole elements).
//  2. Thread per line (5 fields x 3 directions x Nq^2 lines): the D sweep of one
//     line by the even-odd split of the GLL differentiation matrix.  D is
//     centro-antisymmetric (D[N-i][N-n] = -D[i][n]), so with E_m = F_m + F_{N-m}
//     and O_m = F_m - F_{N-m}, the pair S_i, S_{N-i} (i < Nq/2) comes from
//     a_i = sum_m De[i][m] E_m (+ D[i][c] F_c for odd Nq) and
//     b_i = sum_m Do[i][m] O_m as S_i = a_i + b_i, S_{N-i} = b_i - a_i, and for
//     odd Nq the centre row S_c = sum_m D[c][m] O_m.  That is half the products
//     of the direct sweep.  Each result overwrites its flux in place.
//  3. Thread per point: sum of the three sweeps, times -Jinv, the gravity
//     source, one rounding to FP64 and one store per field.
//
// Shared layout: at Nq = 8, slot(line, n) = 8*line + (n ^ h(line)), with
// h(line) = (line & 6) | ((line >> 3) & 1): 8-byte accesses are then free of
// bank conflicts in all three access patterns (phase-1 writes by points,
// phase-2 line reads and writes, phase-3 reads by points).  Other orders
// keep lines of Nq slots.
//
// Theta - Theta_ref and rho - rho_ref are formed in FP64 (one exact
// subtraction each) before splitting.  In double-float the 2^-48 error of each
// operand would be amplified by Theta/Theta' ~ 1e3.
//
// Elements whose state holds a non-finite value or a magnitude >= 2^41, or
// rho <= 0, or whose double-float result overflows, are evaluated in native
// FP64 from the same stored geometry.  So are single points whose |x| exceeds
// 1/64: they take their p' from the FP64 pow.  State values below 2^-74 enter
// as zero.
#include <cuda_runtime.h>

#include "bulk_copy.cuh"
#include "df64.cuh"
#include "numa_internal.h"

namespace numa {

namespace {

template <int NQ>
struct DfShape {
    static constexpr int N3 = NQ * NQ * NQ;
    static constexpr int NL = NQ * NQ;                 // lines per (direction, field)
    static constexpr int kItems = kFields * 3 * NL;    // (direction, field, line) sweep tasks
};

// Resident CTAs per SM the register budget is sized for: two 512-thread CTAs
// at Nq = 8 (64 registers); about 640 threads per SM at the other orders
// (about 100 registers: the double-float sweeps of one line need more than
// 64 without spilling), at most 32 CTAs.
template <int NQ>
constexpr int df_min_ctas() {
    constexpr int n = NQ == 8 ? 2 : 640 / (NQ * NQ * NQ);
    return n < 1 ? 1 : (n > 32 ? 32 : n);
}

__device__ __forceinline__ df ld_df(const float2 *p, int64_t i) {
    float2 v = __ldg(p + i);
    return df{v.x, v.y};
}

__device__ __forceinline__ int swz_h(int line) { return (line & 6) | ((line >> 3) & 1); }

template <int NQ>
__device__ __forceinline__ int slot(int line, int n) {
    if constexpr (NQ == 8)
        return line * 8 + (n ^ swz_h(line));
    else
        return line * NQ + n;
}

// Line and position of point (i, j, k) for reference direction d.
template <int NQ>
__device__ __forceinline__ int dir_slot(int d, int i, int j, int k) {
    if (d == 0) return slot<NQ>(NQ * k + j, i);
    if (d == 1) return slot<NQ>(NQ * k + i, j);
    return slot<NQ>(NQ * j + i, k);
}

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// 1/a in df: one Newton step from the hardware reciprocal of a.h (7 flops).
__device__ __forceinline__ df df_rcp(df a) {
    const float r0 = rcp_approx(a.h);
    float p, pe;
    two_prod(a.h, r0, p, pe);
    const float t = __fsub_rn(1.0f, p);              // exact: p is within 2 ulps of 1
    const float e = __fmaf_rn(-a.l, r0, __fsub_rn(t, pe));
    return df{r0, __fmul_rn(r0, e)};
}

// p(Theta) - p(Theta_ref) = p_ref ((1 + x)^gamma - 1), x = Theta'/Theta_ref,
// written as A Theta' g(x) with A = p_ref / Theta_ref and
// g(x) = sum_k c_k x^(k-1), c_k = binom(gamma, k).  For |x| <= 1/64 the
// truncation after c_9 is below 2e-18 relative.  c_1..c_3 are carried in df,
// c_4..c_9 in FP32, where their share of g is below 1e-6.
__device__ __forceinline__ df eos_series(df thp, df x, df A, const DfParams &P) {
    float t = P.ct[5];
#pragma unroll
    for (int k = 4; k >= 0; --k) t = __fmaf_rn(t, x.h, P.ct[k]);   // c4 + x(c5 + ...)
    df T3;
    {
        float p, e;
        two_prod(x.h, t, p, e);
        T3 = df_add(P.c3, df{p, e});
    }
    df T2 = df_add(P.c2, df_mul(x, T3));
    df g = df_add(P.c1, df_mul(x, T2));
    return df_mul(df_mul(A, thp), df_norm(g));
}

// FP64 equation of state, for points outside the series range (out of line).
__device__ __noinline__ double eos_pressure_fp64(double Th, const DfParams &P) {
    return __dmul_rn(P.p0, pow(__ddiv_rn(__dmul_rn(P.R, Th), P.p0), P.gamma));
}

// Native FP64 evaluation of one element from df-stored geometry (rare path).
template <int NQ, bool TR>
__device__ void element_fp64(const DfGeometry &geo, const DfParams &P, const double *__restrict__ q,
                             double *__restrict__ rhs, int64_t M, int64_t e, int nf, double *sF) {
    constexpr int N3 = DfShape<NQ>::N3;
    const int NF = TR ? nf : kFields;   // flux blocks per direction
    const int l = threadIdx.x;
    const int64_t node = e * N3 + l;
    __syncthreads();  // sF aliases the df buffers of the caller
    const double rho = q[node];
    const double U1 = q[M + node], U2 = q[2 * M + node], U3 = q[3 * M + node];
    const double Th = q[4 * M + node];
    const double pp = eos_pressure_fp64(Th, P) - eos_pressure_fp64(geo.theta_ref[node], P);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double g1 = df_to_double(ld_df(geo.g[3 * d], node));
        const double g2 = df_to_double(ld_df(geo.g[3 * d + 1], node));
        const double g3 = df_to_double(ld_df(geo.g[3 * d + 2], node));
        const double u = (g1 * U1 + g2 * U2 + g3 * U3) / rho;
        double *F = sF + d * NF * N3 + l;
        F[0 * N3] = rho * u;
        F[1 * N3] = U1 * u + g1 * pp;
        F[2 * N3] = U2 * u + g2 * pp;
        F[3 * N3] = U3 * u + g3 * pp;
        F[4 * N3] = Th * u;
        if constexpr (TR) {
            for (int b = kFields; b < nf; ++b) F[b * N3] = q[b * M + node] * u;   // tracers Q u_d
        }
    }
    __syncthreads();
    const int i = l % NQ, j = (l / NQ) % NQ, k = l / (NQ * NQ);
    const double Jinv = df_to_double(ld_df(geo.Jinv, node));
    const double drho = rho - geo.rho_ref[node];
#pragma unroll 1
    for (int b = 0; b < NF; ++b) {
        const double *Fr = sF + (0 * NF + b) * N3;
        const double *Fs = sF + (1 * NF + b) * N3;
        const double *Ft = sF + (2 * NF + b) * N3;
        double s = 0.0;
#pragma unroll
        for (int n = 0; n < NQ; ++n) s += P.D[i * NQ + n] * Fr[(k * NQ + j) * NQ + n];
#pragma unroll
        for (int n = 0; n < NQ; ++n) s += P.D[j * NQ + n] * Fs[(k * NQ + n) * NQ + i];
#pragma unroll
        for (int n = 0; n < NQ; ++n) s += P.D[k * NQ + n] * Ft[(n * NQ + j) * NQ + i];
        double v = -Jinv * s;
        if (b == 3) v -= drho * P.grav;
        rhs[b * M + node] = v;
    }
}

// Starts the arrays of element e toward L2 (Nq^3 points of 8 bytes per array),
// where an element's slab of one array is a whole number of 16-byte units
// (the bulk prefetch's rule; even Nq).
template <int NQ>
__device__ __forceinline__ void prefetch_element(const DfGeometry &geo, const double *q,
                                                 int64_t M, int nf, int64_t e) {
    constexpr int N3 = DfShape<NQ>::N3;
    constexpr uint32_t B = N3 * 8;
    if constexpr (B % 16 == 0) {
        const int64_t off = e * N3;
        for (int b = 0; b < nf; ++b) prefetch_l2(q + b * M + off, B);
#pragma unroll
        for (int a = 0; a < 9; ++a) prefetch_l2(geo.g[a] + off, B);
        prefetch_l2(geo.Jinv + off, B);
        prefetch_l2(geo.rho_ref + off, B);
        prefetch_l2(geo.theta_ref + off, B);
        prefetch_l2(geo.w + off, B);
        prefetch_l2(geo.A + off, B);
    }
}

// ahead: half the CTAs resident on the GPU at once.  The element that many
// launch slots later starts soon on some SM, so its arrays are prefetched to
// L2 now and its loads then hit L2 rather than DRAM (one wave ahead: 1.30 ->
// 1.22 ms at N = 7, 32768 elements; half a wave 14.06 against 13.91 GDOF/s
// for one wave and 13.98 for a quarter; two waves ahead was slower than
// none, the prefetched data displacing the running wave's).
// TR: the 8-field form (nf = 5 + tracers, 6..8): the tracers' state is split
// like the other fields and their fluxes are Q u_d; nf blocks per direction.
template <int NQ, bool TR>
__global__ void __launch_bounds__(NQ * NQ * NQ, df_min_ctas<NQ>())
vol_rhs_df64_kernel(DfGeometry geo, DfParams P, const double *__restrict__ q,
                    double *__restrict__ rhs, int64_t M, int64_t e0, int64_t e_end,
                    int64_t ahead, int nf) {
    constexpr int N3 = DfShape<NQ>::N3;
    constexpr int NL = DfShape<NQ>::NL;
    constexpr int HALF = NQ / 2;
    constexpr bool ODD = (NQ & 1) != 0;
    constexpr int C = NQ / 2;
    constexpr int NT = kMaxFields - kFields;   // tracers at most
    const int NF = TR ? nf : kFields;          // flux blocks per direction
    extern __shared__ float2 sbuf[];  // [direction*NF + field][slot], 3 NF Nq^3 float2
    const int l = threadIdx.x;
    const int i = l % NQ, j = (l / NQ) % NQ, k = l / (NQ * NQ);
    const int64_t e = e0 + blockIdx.x;
    const int64_t node = e * N3 + l;
    if (l == 0 && e + ahead < e_end) prefetch_element<NQ>(geo, q, M, NF, e + ahead);

    // ---- phase 1: state, p', fluxes -----------------------------------
    bool big = false, tiny = false;
    df Q[kFields];
    double qd[kFields];
#pragma unroll
    for (int b = 0; b < kFields; ++b) qd[b] = q[b * M + node];
#pragma unroll
    for (int b = 0; b < kFields; ++b) Q[b] = df_split(qd[b], big, tiny);
    df QT[TR ? NT : 1];   // the tracers
    if constexpr (TR) {
#pragma unroll
        for (int t = 0; t < NT; ++t)
            QT[t] = kFields + t < nf ? df_split(q[(kFields + t) * M + node], big, tiny)
                                     : df{0.0f, 0.0f};
    }
    // Exact FP64 differences (Sterbenz: the operands are within a factor 2 in
    // the fast path) before splitting, so the perturbations keep full accuracy.
    const double th0 = geo.theta_ref[node];
    const double thp_d = qd[4] - th0;
    const double drho_d = qd[0] - geo.rho_ref[node];
    const df thp = df_split(thp_d, big, tiny);
    const df drho = df_split(drho_d, big, tiny);
    const bool bad = big || !(qd[0] > 0.0);
    if (__syncthreads_or(bad)) {
        element_fp64<NQ, TR>(geo, P, q, rhs, M, e, nf, reinterpret_cast<double *>(sbuf));
        return;
    }

    const df rinv = df_rcp(Q[0]);
    // J^-1 here rather than after the sweeps: its load overlaps phase 1
    // (13.90 against 13.74 GDOF/s at N = 7)
    const df jinv = ld_df(geo.Jinv, node);
    df pp;
    {
        const df x = df_mul(thp, ld_df(geo.w, node));
        if (fabsf(x.h) <= 0.015625f) {
            pp = eos_series(thp, x, ld_df(geo.A, node), P);
        } else {
            bool b2 = false, t2 = false;
            pp = df_split(eos_pressure_fp64(qd[4], P) - eos_pressure_fp64(th0, P), b2, t2);
        }
    }

#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const df g1 = ld_df(geo.g[3 * d], node);
        const df g2 = ld_df(geo.g[3 * d + 1], node);
        const df g3 = ld_df(geo.g[3 * d + 2], node);
        dot2 acc = dot2_first(g1, Q[1]);
        dot2_add(acc, g2, Q[2]);
        dot2_add(acc, g3, Q[3]);
        const df v = dot2_value(acc);
        const df u = df_mul(df_norm(v), rinv);
        df F[kFields];
        F[0] = v;
        {
            dot2 a = dot2_first(Q[1], u);
            dot2_add(a, g1, pp);
            F[1] = dot2_value(a);
            dot2 b = dot2_first(Q[2], u);
            dot2_add(b, g2, pp);
            F[2] = dot2_value(b);
            dot2 c = dot2_first(Q[3], u);
            dot2_add(c, g3, pp);
            F[3] = dot2_value(c);
        }
        F[4] = df_mul(Q[4], u);
        const int s = dir_slot<NQ>(d, i, j, k);
#pragma unroll
        for (int b = 0; b < kFields; ++b) sbuf[(d * NF + b) * N3 + s] = make_float2(F[b].h, F[b].l);
        if constexpr (TR) {
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                if (kFields + t >= nf) break;
                const df Ft = df_mul(QT[t], u);
                sbuf[(d * NF + kFields + t) * N3 + s] = make_float2(Ft.h, Ft.l);
            }
        }
    }
    __syncthreads();

    // ---- phase 2: even-odd D sweeps, one line per task -----------------
    for (int item = l; item < (TR ? 3 * NF * NL : DfShape<NQ>::kItems); item += N3) {
        float2 *buf = sbuf + (item / NL) * N3;
        const int line = item % NL;
        df F[NQ];
#pragma unroll
        for (int n = 0; n < NQ; ++n) {
            const float2 v = buf[slot<NQ>(line, n)];
            F[n] = df{v.x, v.y};
        }
        df E[HALF], O[HALF];
#pragma unroll
        for (int m = 0; m < HALF; ++m) {
            E[m] = df_add(F[m], F[NQ - 1 - m]);
            O[m] = df_sub(F[m], F[NQ - 1 - m]);
        }
#pragma unroll
        for (int r = 0; r < HALF; ++r) {
            dot2 a = dot2_first(P.De[r][0], E[0]);
            dot2 b = dot2_first(P.Do[r][0], O[0]);
#pragma unroll
            for (int m = 1; m < HALF; ++m) {
                dot2_add(a, P.De[r][m], E[m]);
                dot2_add(b, P.Do[r][m], O[m]);
            }
            if constexpr (ODD) dot2_add(a, P.Dc[r], F[C]);
            const df A = dot2_value(a), B = dot2_value(b);
            const df Si = df_add(B, A);
            const df Sm = df_sub(B, A);
            buf[slot<NQ>(line, r)] = make_float2(Si.h, Si.l);
            buf[slot<NQ>(line, NQ - 1 - r)] = make_float2(Sm.h, Sm.l);
        }
        if constexpr (ODD) {
            dot2 c = dot2_first(P.Dcr[0], O[0]);
#pragma unroll
            for (int m = 1; m < HALF; ++m) dot2_add(c, P.Dcr[m], O[m]);
            const df Sc = df_norm(dot2_value(c));
            buf[slot<NQ>(line, C)] = make_float2(Sc.h, Sc.l);
        }
    }
    __syncthreads();

    // ---- phase 3: combine, scale, gravity, store -----------------------
    double out[kFields];
    bool finite = true;
    auto field = [&](int b) -> double {
        const float2 r = sbuf[(0 * NF + b) * N3 + dir_slot<NQ>(0, i, j, k)];
        const float2 s = sbuf[(1 * NF + b) * N3 + dir_slot<NQ>(1, i, j, k)];
        const float2 t = sbuf[(2 * NF + b) * N3 + dir_slot<NQ>(2, i, j, k)];
        df R = df_add(df_add(df{r.x, r.y}, df{s.x, s.y}), df{t.x, t.y});
        df v = df_mul(df_norm(R), jinv);
        if (b == 3) v = df_add(v, df_mul(drho, P.grav_df));
        v = df_norm(v);
        finite = finite && isfinite(v.h) && isfinite(v.l);
        return -df_to_double(v);
    };
#pragma unroll
    for (int b = 0; b < kFields; ++b) out[b] = field(b);
    if constexpr (TR) {
        // the tracers stored at once (the FP64 evaluation below rewrites
        // every field of an element that overflowed)
#pragma unroll 1
        for (int b = kFields; b < nf; ++b) rhs[b * M + node] = field(b);
    }
    // An overflow anywhere in the element (float range) sends it to FP64.
    if (__syncthreads_or(!finite)) {
        element_fp64<NQ, TR>(geo, P, q, rhs, M, e, nf, reinterpret_cast<double *>(sbuf));
        return;
    }
#pragma unroll
    for (int b = 0; b < kFields; ++b) rhs[b * M + node] = out[b];
}

// Largest magnitude of an array (bit patterns of nonnegative doubles order
// like their values).
__global__ void abs_max_kernel(const double *__restrict__ src, int64_t M,
                               unsigned long long *amax) {
    unsigned long long best = 0ull;
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < M;
         m += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(src[m]));
        best = b > best ? b : best;
    }
    atomicMax(amax, best);
}

// FP64 -> df conversion of the handle's per-point arrays with the splitting the
// kernel applies to the state.  Magnitudes below thresh (rounding noise far
// below the array's largest entry) become zero; what remains outside the
// fast-path range is flagged.
__global__ void to_df_kernel(const double *__restrict__ src, float2 *__restrict__ dst, int64_t M,
                             double thresh, int *bad) {
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < M;
         m += (int64_t)gridDim.x * blockDim.x) {
        bool big = false, tiny = false;
        const double x = fabs(src[m]) < thresh ? 0.0 : src[m];
        const df v = df_split(x, big, tiny);
        dst[m] = make_float2(v.h, v.l);
        if (big || tiny) atomicOr(bad, 1);   // a significant value would be lost
    }
}

}  // namespace

cudaError_t launch_abs_max(const double *src, int64_t M, unsigned long long *amax_bits,
                           cudaStream_t s) {
    if (M == 0) return cudaSuccess;
    abs_max_kernel<<<1216, 256, 0, s>>>(src, M, amax_bits);
    return cudaGetLastError();
}

cudaError_t launch_to_df(const double *src, float2 *dst, int64_t M, double thresh, int *bad,
                         cudaStream_t s) {
    if (M == 0) return cudaSuccess;
    to_df_kernel<<<1216, 256, 0, s>>>(src, dst, M, thresh, bad);
    return cudaGetLastError();
}

namespace {

template <int NQ, bool TR>
cudaError_t launch_df_form(ElemRange r, int nf, const DfGeometry &geo, const DfParams &P,
                           const double *q, double *rhs, int num_sms, cudaStream_t s) {
    constexpr int N3 = NQ * NQ * NQ;
    const size_t smem = sizeof(float2) * (TR ? nf : kFields) * 3 * N3;
    cudaError_t e = cudaFuncSetAttribute(vol_rhs_df64_kernel<NQ, TR>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, vol_rhs_df64_kernel<NQ, TR>, N3, smem);
    if (e != cudaSuccess) return e;
    const int64_t wave = (int64_t)num_sms * (per_sm > 0 ? per_sm : 1);
    const int64_t ahead = wave / 2 > 0 ? wave / 2 : 1;
    vol_rhs_df64_kernel<NQ, TR><<<(unsigned)r.count, N3, smem, s>>>(geo, P, q, rhs, r.M, r.e0,
                                                                    r.e0 + r.count, ahead, nf);
    return cudaGetLastError();
}

template <int NQ>
cudaError_t launch_df(ElemRange r, int nf, const DfGeometry &geo, const DfParams &P,
                      const double *q, double *rhs, int num_sms, cudaStream_t s) {
    if (nf > kFields) return launch_df_form<NQ, true>(r, nf, geo, P, q, rhs, num_sms, s);
    return launch_df_form<NQ, false>(r, nf, geo, P, q, rhs, num_sms, s);
}

}  // namespace

cudaError_t launch_vol_rhs_df64(int N, int nf, ElemRange r, const DfGeometry &geo,
                                const DfParams &P, const double *q, double *rhs, int num_sms,
                                cudaStream_t s) {
    if (r.count <= 0) return cudaSuccess;
    if (nf < kFields || nf > kMaxFields) return cudaErrorInvalidValue;
    switch (N) {
        case 1: return launch_df<2>(r, nf, geo, P, q, rhs, num_sms, s);
        case 2: return launch_df<3>(r, nf, geo, P, q, rhs, num_sms, s);
        case 3: return launch_df<4>(r, nf, geo, P, q, rhs, num_sms, s);
        case 4: return launch_df<5>(r, nf, geo, P, q, rhs, num_sms, s);
        case 5: return launch_df<6>(r, nf, geo, P, q, rhs, num_sms, s);
        case 6: return launch_df<7>(r, nf, geo, P, q, rhs, num_sms, s);
        case 7: return launch_df<8>(r, nf, geo, P, q, rhs, num_sms, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace numa
