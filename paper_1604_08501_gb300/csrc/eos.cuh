// Pressure perturbation p' = p(Theta) - p(Theta_ref) for the native FP64 and
// the mixed-precision kernels (equation of state of Sec. 2:
// p = p0 (R Theta / p0)^gamma, gamma = cp / (cp - R)).
//
// Both evaluate p' = p_ref ((1 + x)^gamma - 1) with x = Theta'/Theta_ref,
// written A Theta' g(x) with A = p_ref / Theta_ref and
// g(x) = sum_k binom(gamma, k) x^(k-1).  That is the same quantity as the
// difference of two pressures, without its cancellation.
//
// FP64 has three forms, each accurate to a few ulps over its whole range:
// the series to 9 terms for |x| <= 1/64 and to 15 terms for |x| <= 1/8
// (truncation below 2^-55 relative for gamma near 1.4), and
// p_ref expm1(gamma log1p(x)) for any x > -1.  A warp takes the widest form
// any of its lanes needs, so that a warp never runs several of them one after
// the other: states advanced over many stages drift past 1/64, and on fine
// meshes past 1/8.  Where Theta_ref = 0 (w and A not finite) or x <= -1 the
// definition, two evaluations of the equation of state, is used.
// FP32 likewise: 5 terms for |x| <= 1/64, 16 terms for |x| <= 1/2 (truncation
// below 2^-26), expm1f(gamma log1pf(x)) beyond, chosen per warp.
#pragma once

#include "kernel_params.h"

namespace numa {

// p0 (R Theta / p0)^gamma, the equation of state of Sec. 2.  Not inlined:
// the rhs kernel calls it only where the series does not apply, and keeping
// pow out of line keeps its registers out of the kernel's budget.
static __device__ __noinline__ double eos_pressure(double Th, const EosConstants &c) {
    return __dmul_rn(c.p0, pow(__ddiv_rn(__dmul_rn(c.R, Th), c.p0), c.gamma));
}

// p' of one point; the form is chosen per warp (see above).  Every active
// lane of the warp must call it together.
// Params: NativeParams or HighParams (the series coefficients c and eos).
template <typename Params>
static __device__ __forceinline__ double pressure_perturbation(double Th, double th0, double w, double A,
                                                        const Params &P) {
    const double thp = Th - th0;              // Theta'
    const double x = thp * w;                 // Theta' / Theta_ref
    const double ax = fabs(x);
    const unsigned lanes = __activemask();
    if (__all_sync(lanes, ax <= 0.015625)) {
        double g = P.c[8];
#pragma unroll
        for (int k = 7; k >= 0; --k) g = fma(g, x, P.c[k]);   // sum_k c_{k+1} x^k
        return (A * thp) * g;
    }
    if (__all_sync(lanes, ax <= 0.125)) {
        double g = P.c[14];
#pragma unroll
        for (int k = 13; k >= 0; --k) g = fma(g, x, P.c[k]);
        return (A * thp) * g;
    }
    // x > -1 and finite (a NaN fails the comparison, an infinite x fails < 2^1000)
    if (__all_sync(lanes, x > -1.0 && ax < 1e300))
        return (A * th0) * expm1(P.eos.gamma * log1p(x));
    return eos_pressure(Th, P.eos) - eos_pressure(th0, P.eos);
}

// FP32 form from the perturbation Theta' itself (mixed precision): the series
// (5 or 16 terms) or expm1f(gamma log1pf(x)), chosen per warp as in FP64, all
// free of cancellation.
// A = K Theta_ref^(gamma - 1) with K = p0^(1 - gamma) R^gamma is recomputed
// from Theta_ref instead of being read from memory.  eos_reference_f32 forms
// the per-point factors (w = 1/Theta_ref and A), which a caller that keeps a
// point for many evaluations computes once.
struct EosRef32 {
    float w, A;
};

template <typename Params>
static __device__ __forceinline__ EosRef32 eos_reference_f32(float th0, const Params &P) {
    return EosRef32{__frcp_rn(th0), P.K * exp2f(P.gm1 * log2f(th0))};   // A = p(Theta_ref)/Theta_ref
}

// Params: MixedParams or HighParams32 (c, K, gm1, gamma).
template <typename Params>
static __device__ __forceinline__ float pressure_perturbation_f32(float thp, float th0, EosRef32 r,
                                                           const Params &P) {
    const unsigned lanes = __activemask();
    if (__all_sync(lanes, th0 > 0.0f)) {
        const float x = thp * r.w;
        const float ax = fabsf(x);
        if (__all_sync(lanes, ax <= 0.015625f)) {
            float g = P.c[4];
#pragma unroll
            for (int k = 3; k >= 0; --k) g = fmaf(g, x, P.c[k]);   // sum_k c_{k+1} x^k
            return (r.A * thp) * g;
        }
        if (__all_sync(lanes, ax <= 0.5f)) {
            float g = P.c[15];
#pragma unroll
            for (int k = 14; k >= 0; --k) g = fmaf(g, x, P.c[k]);
            return (r.A * thp) * g;
        }
        if (__all_sync(lanes, x > -1.0f)) return (r.A * th0) * expm1f(P.gamma * log1pf(x));
    }
    // Theta_ref = 0 (the paper's full-pressure form): p' = p(Theta'); and,
    // per lane, whatever the warp's common forms do not cover.
    if (th0 > 0.0f) return (r.A * th0) * expm1f(P.gamma * log1pf(thp * r.w));
    return P.K * powf(thp, P.gamma);
}

template <typename Params>
static __device__ __forceinline__ float pressure_perturbation_f32(float thp, float th0,
                                                           const Params &P) {
    if (th0 > 0.0f) return pressure_perturbation_f32(thp, th0, eos_reference_f32(th0, P), P);
    return P.K * powf(thp, P.gamma);
}

}  // namespace numa
