// Double-float ("df") arithmetic on the FP32 pipes: a value is the unevaluated
// sum h + l of two floats, about 48 significant bits.  On GB300 the FP32 FMA
// pipe issues 68 times as many operations per clock as the FP64 pipe, so an
// FP64-accurate evaluation of the volume term runs faster in df than in
// native doubles.
//
// The error-free transformations used here are the classical ones:
//   two_sum  (Knuth 1969):   s + e == a + b exactly, 6 flops, any ordering.
//   two_prod (FMA form):     p + e == a * b exactly, 2 flops.
// Every FP32 operation below is an explicit round-to-nearest intrinsic
// (__fadd_rn, __fmul_rn, __fmaf_rn), so the compiler neither contracts nor
// reorders them.  The transformations stay exact only in that form.
//
// "Unnormalised" results keep |l| a few ulps of h rather than <= ulp(h)/2;
// they feed further df operations, where l enters only as a correction.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "kernel_params.h"

namespace numa {

__device__ __forceinline__ df df_make(float h, float l) { return df{h, l}; }

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// |a| >= |b| (or a == 0): s + e == a + b exactly, 3 flops.
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

__device__ __forceinline__ df df_norm(df a) {
    df r;
    fast_two_sum(a.h, a.l, r.h, r.l);
    return r;
}

// a + b, unnormalised (7 flops).
__device__ __forceinline__ df df_add(df a, df b) {
    df r;
    float e;
    two_sum(a.h, b.h, r.h, e);
    r.l = __fadd_rn(e, __fadd_rn(a.l, b.l));
    return r;
}

__device__ __forceinline__ df df_neg(df a) { return df{-a.h, -a.l}; }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

// a * b, unnormalised (4 flops).
__device__ __forceinline__ df df_mul(df a, df b) {
    df r;
    float e;
    two_prod(a.h, b.h, r.h, e);
    e = __fmaf_rn(a.h, b.l, e);
    r.l = __fmaf_rn(a.l, b.h, e);
    return r;
}

// a * f for a float f, unnormalised (3 flops).
__device__ __forceinline__ df df_mulf(df a, float f) {
    df r;
    float e;
    two_prod(a.h, f, r.h, e);
    r.l = __fmaf_rn(a.l, f, e);
    return r;
}

// Compensated dot product accumulator (the Dot2 scheme of Ogita, Rump and
// Oishi, 2005, extended to df operands): s collects the exact high products
// through two_sum, c collects every error term and the cross products.
struct dot2 {
    float s, c;
};

__device__ __forceinline__ dot2 dot2_first(df a, df b) {
    dot2 r;
    float e;
    two_prod(a.h, b.h, r.s, e);
    e = __fmaf_rn(a.h, b.l, e);
    r.c = __fmaf_rn(a.l, b.h, e);
    return r;
}

__device__ __forceinline__ void dot2_add(dot2 &acc, df a, df b) {
    float p, e, s, err;
    two_prod(a.h, b.h, p, e);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    two_sum(acc.s, p, s, err);
    acc.s = s;
    acc.c = __fadd_rn(acc.c, __fadd_rn(err, e));
}

__device__ __forceinline__ df dot2_value(dot2 a) { return df{a.s, a.c}; }

// ---------------------------------------------------------------------------
// FP64 <-> df by integer operations.  GB300 runs FP64<->FP32 conversions at
// the FP64 rate, so the bits are moved by shifts and masks instead.
// ---------------------------------------------------------------------------

// Split range: finite magnitudes below 2^41 (exponent field <= 1063).  Values
// below 2^-74 (exponent field < 949) flush to zero, an absolute error under
// 5.3e-23: the low part of a smaller value would not be a normal float.
constexpr int kDfMinExp = 949;
constexpr int kDfMaxExp = 1023 + 40;

// Split a double into h (its first 24 significant bits, truncated) and l (the
// remaining 29 bits, rounded to 24): |x - (h + l)| <= 2^-48 |x|.  Sets big if
// x is not finite or |x| >= 2^41, tiny if x is nonzero and flushed to zero.
__device__ __forceinline__ df df_split(double x, bool &big, bool &tiny) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    const uint32_t sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7FFu);
    const bool zero = (b << 1) == 0ull;
    big = big || e > kDfMaxExp;
    tiny = tiny || (!zero && e < kDfMinExp);
    if (e < kDfMinExp || e > kDfMaxExp) return df{0.0f, 0.0f};
    const uint32_t mtop = ((hi & 0xFFFFFu) << 3) | (lo >> 29);          // 23 bits
    const float h = __uint_as_float(sign | ((uint32_t)(e - 896) << 23) | mtop);
    const uint32_t rest = lo & 0x1FFFFFFFu;                              // 29 bits
    // rest * 2^(e - 1075): scale built as a float with exponent e - 1075.
    const float scale = __uint_as_float((uint32_t)(e - 1075 + 127) << 23);
    const float l = __uint_as_float(__float_as_uint(__fmul_rn(__uint2float_rn(rest), scale)) | sign);
    return df{h, l};
}

// A float widened to a double exactly (zero and normal floats).
__device__ __forceinline__ double f32_to_f64_bits(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xFFu;
    if (e == 0u) return 0.0;
    const uint32_t hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7FFFFFu) >> 3);
    const uint32_t lo = u << 29;
    return __hiloint2double((int)hi, (int)lo);
}

// h + l rounded to double: two exact widenings and one FP64 add.
__device__ __forceinline__ double df_to_double(df a) {
    return f32_to_f64_bits(a.h) + f32_to_f64_bits(a.l);
}

}  // namespace numa
