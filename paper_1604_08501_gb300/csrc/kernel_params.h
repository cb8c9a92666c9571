// Parameters and per-point array descriptors that the volume-term kernels take
// by value: what a kernel's device code depends on besides its own source.
// (The launchers, the batch and engine structures and the handle are in
// numa_internal.h.)
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace numa {

constexpr int kFields = 5;      // rho, U1, U2, U3, Theta
constexpr int kMaxFields = 8;   // with three passive tracers

// Elements [e0, e0 + count) of a mesh whose per-point planes hold M values.
struct ElemRange {
    int64_t e0, count, M;
};

// Device-side geometry of one handle. Every per-point array has M entries,
// padded so that each starts on a 256-byte boundary.
struct DeviceGeometry {
    const double *g[9];      // metric terms g[3*d + a]
    const double *Jinv;      // 1 / J
    const double *rho_ref;   // reference density
    const double *theta_ref; // reference Theta
    const double *w;         // 1 / Theta_ref
    const double *A;         // p(Theta_ref) / Theta_ref
    const double *D;         // (N+1)^2, row-major D[i*Nq + n]
};

struct EosConstants {
    double p0, R, gamma, grav;
};

// Parameters of the native kernel: EOS constants, c[k] = binom(gamma, k+1)
// (k = 0..14, the coefficients of the p' series), and the even-odd pieces of D
// for r, m < Nq/2: De = (D[r][m] + D[r][N-m])/2, Do = (D[r][m] - D[r][N-m])/2,
// Dc[r] = D[r][c] and Dcr[m] = D[c][m] (centre column and row, odd Nq).
// Uniform across threads, so the kernel reads them as constant-bank operands.
struct NativeParams {
    EosConstants eos;
    double c[15];
    double De[16], Do[16], Dc[4], Dcr[4];
};

// Parameters of the native kernel for orders N = 8..15 (Nq = 9..16): the same
// quantities as NativeParams with even-odd tables up to (Nq/2)^2 = 64 entries.
struct HighParams {
    EosConstants eos;
    double c[15];
    double De[64], Do[64], Dc[8], Dcr[8];
};

// The same for the mixed-precision mode at N = 8..15: FP32 tables and the FP32
// EOS constants of MixedParams (c[k] = binom(gamma, k+1)).
struct HighParams32 {
    float De[64], Do[64], Dc[8], Dcr[8];
    float c[16];
    float K, gm1, gamma, grav;
};

// Per-point arrays of the double-float path (N = 1..7): float2 (h, l) pairs, and
// the reference state in FP64, so that rho - rho_ref and Theta - Theta_ref are
// exact FP64 differences before they are split.
struct DfGeometry {
    const float2 *g[9];      // metric terms
    const float2 *Jinv;      // 1 / J
    const double *rho_ref;   // reference density
    const double *theta_ref; // reference Theta
    const float2 *w;         // 1 / Theta_ref
    const float2 *A;         // p(Theta_ref) / Theta_ref
};

// Per-point arrays of the mixed-precision path, FP32.
struct MixedGeometry {
    const float *g[9];
    const float *Jinv;
    const float *rho_ref;
    const float *theta_ref;
};

// Parameters of the mixed-precision kernel: even-odd pieces of D (as in
// NativeParams), c[k] = binom(gamma, k+1) for k = 0..15, K = p0^(1-gamma) R^gamma
// (so p(Theta) = K Theta^gamma), gamma - 1, gamma and gravity.
struct MixedParams {
    float De[16], Do[16], Dc[4], Dcr[4];
    float c[16];
    float K, gm1, gamma, grav;
};

// Double-float value: the unevaluated sum h + l of two floats.
struct df {
    float h, l;
};

struct DfParams {
    df De[4][4];       // (D[i][m] + D[i][N-m]) / 2, i, m < Nq/2
    df Do[4][4];       // (D[i][m] - D[i][N-m]) / 2
    df Dc[4];          // D[i][c], the centre column (odd Nq), i < Nq/2
    df Dcr[4];         // D[c][m], the centre row (odd Nq), m < Nq/2
    df c1, c2, c3;     // binom(gamma, k), k = 1..3
    float ct[6];       // binom(gamma, k), k = 4..9
    df grav_df;        // gravity
    double grav, p0, R, gamma;
    double D[64];      // D, row-major D[i Nq + n], for the native fallback
};

}  // namespace numa
