// Internal declarations of the numa_vol library (not part of the C ABI).
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "numa_vol.h"

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

// Per-point arrays of the double-float path (N = 7): float2 (h, l) pairs, and
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

// Kernel parameters of the double-float path.
struct DfParams;  // defined below

// Launchers (vol_fp64.cu). They return a cudaError_t from the launch.
// reference_eos: w = 1/Theta_ref, A = p(Theta_ref)/Theta_ref per point.
cudaError_t launch_reference_eos(const double *theta_ref, double *w, double *A, int64_t M,
                                 EosConstants c, cudaStream_t s);
// Native FP64 for N = 8..15 (vol_fp64_high.cu): one CTA of Nq^2 threads per
// element, one pass per field.
// nf: 5 fields, or 5 + tracers (nf <= 8).
cudaError_t launch_vol_rhs_fp64_high(int N, int nf, ElemRange r, const DeviceGeometry &geo,
                                     const HighParams &P, const double *q, double *rhs,
                                     cudaStream_t s);
// Mixed precision for N = 8..15 (vol_fp64_high.cu, FP32 instantiation).
cudaError_t launch_vol_rhs_mixed_high(int N, int nf, ElemRange r, const MixedGeometry &geo,
                                      const HighParams32 &P, const float *q, float *rhs,
                                      cudaStream_t s);
cudaError_t launch_vol_rhs_fp64(int N, int nf, ElemRange r, const DeviceGeometry &geo,
                                const NativeParams &P, const double *q, double *rhs,
                                cudaStream_t s);

// Launchers of the double-float path (vol_df64.cu).  abs_max: max |src| into
// *amax_bits (the bit pattern of a nonnegative double).  to_df: split src
// into (h, l) pairs, flushing |x| < thresh to zero and flagging values left
// outside the fast-path range in *bad.
cudaError_t launch_abs_max(const double *src, int64_t M, unsigned long long *amax_bits,
                           cudaStream_t s);
cudaError_t launch_to_df(const double *src, float2 *dst, int64_t M, double thresh, int *bad,
                         cudaStream_t s);
cudaError_t launch_vol_rhs_df64(ElemRange r, const DfGeometry &geo, const DfParams &P,
                                const double *q, double *rhs, int num_sms, cudaStream_t s);

// Launchers of the mixed-precision path (vol_mixed.cu).
cudaError_t launch_to_f32(const double *src, float *dst, int64_t M, cudaStream_t s);
// N = 7 launches the persistent bulk-copy kernel (2 CTAs per SM); it sets
// bit 0 of *err if a bounded wait on its copies times out.
cudaError_t launch_vol_rhs_mixed(int N, int nf, ElemRange r, const MixedGeometry &geo,
                                 const MixedParams &P, const float *q, float *rhs, int *err,
                                 int num_sms, cudaStream_t s);

// GLL points and differentiation matrix on the host (gll.cpp).
int gll_diff_matrix(int N, double *D);

// Even-odd sweep tables of the order-N GLL D (Nq = N + 1): De, Do
// ((Nq/2)^2, row-major), Dc, Dcr (odd Nq).  Unused entries are zero.
void sweep_tables(int N, const double *D, double De[16], double Do[16], double Dc[4],
                  double Dcr[4]);

// Double-float value: the unevaluated sum h + l of two floats.
struct df {
    float h, l;
};

struct DfParams {
    df De[4][4];       // (D[i][m] + D[i][7-m]) / 2, i, m < 4
    df Do[4][4];       // (D[i][m] - D[i][7-m]) / 2
    df c1, c2, c3;     // binom(gamma, k), k = 1..3
    float ct[6];       // binom(gamma, k), k = 4..9
    df grav_df;        // gravity
    double grav, p0, R, gamma;
    double D[64];      // D for the native fallback
};

// Native: vol_rhs_fp64_kernel (N <= 7); NativeHigh: vol_rhs_high_kernel<Nq, double>
// (N = 8..15); DoubleFloat (N = 7); Mixed (N <= 7) and MixedHigh:
// vol_rhs_high_kernel<Nq, float> (N = 8..15).
enum class Kernel { Native, NativeHigh, DoubleFloat, Mixed, MixedHigh };

// Device-side description of one instance of a batch: its order, size, state
// and the geometry/parameters of its handle (FP64 or mixed, per the batch).
struct BatchInstance {
    int N, nq;
    int64_t M;
    void *q;
    DeviceGeometry geo;
    NativeParams np;
    MixedGeometry mgeo;
    MixedParams mp;
    int nsteps;   // steps of this instance in the launch; 0: the launch's step count
};

// One work item: elements [e0, e0 + count) of an instance.
struct BatchItem {
    int instance;
    int nq;
    int64_t e0;
    int64_t count;
};

// Coefficients of the five-stage fourth-order 2N-storage Runge-Kutta scheme.
struct LsrkCoef {
    double A[5], B[5];
};

// Launch of the persistent batched integrator (batch_lsrk.cu): items are
// claimed through *counter (reset to 0 by the caller before the launch).
// prepare_batch_lsrk() sets the kernels' shared-memory opt-in on the current
// device; call it before the first launch (and outside stream capture).
cudaError_t prepare_batch_lsrk();
// The grid is num_sms times the CTAs per SM the kernel is built for.
cudaError_t launch_batch_lsrk(bool mixed, const BatchInstance *inst, const BatchItem *items,
                              int num_items, int *counter, const LsrkCoef &co, int nsteps,
                              double dt, int num_sms, cudaStream_t s);

// Elements one CTA pass holds for order Nq (512 threads, one per point).
inline int elements_per_pass(int nq) { return 512 / (nq * nq * nq); }

// Work list for instances with tile_mult[nq] passes per item (batch_abi.cu).
std::vector<BatchItem> build_items(const std::vector<BatchInstance> &inst, const int *tile_mult);

}  // namespace numa

struct numa_vol {
    int N = 0;
    int Nq = 0;
    int nf = 5;   // fields of the state: 5 + tracers
    int64_t Ne = 0;
    int64_t M = 0;
    int device = 0;
    int num_sms = 0;
    int *d_err = nullptr;           // device status word: bit 0 = a bounded wait timed out
    numa_precision prec = NUMA_FP64;
    numa::EosConstants eos{};
    void *d_block = nullptr;        // one allocation: geometry, reference state, D
    size_t block_bytes = 0;
    numa::Kernel kernel = numa::Kernel::Native;
    numa::DeviceGeometry geo{};     // native path
    numa::DfGeometry dgeo{};        // double-float path
    numa::DfParams dparams{};
    numa::NativeParams nparams{};
    numa::HighParams hparams{};      // NUMA_FP64, N >= 8
    numa::HighParams32 hmparams{};   // NUMA_MIXED, N >= 8
    numa::MixedGeometry mgeo{};     // mixed-precision path
    numa::MixedParams mparams{};
    size_t elem = sizeof(double);   // bytes per state/rhs value (4 for NUMA_MIXED)
    void *d_stage = nullptr;        // host entry point: q and rhs staging, 2 * 5 * M values
    // host entry point: copy-in, compute and copy-out streams, per-chunk events
    // host path: two compute streams (alternate chunks, so one chunk's tail
    // overlaps the next chunk's start), copy-in and copy-out streams
    cudaStream_t host_stream = nullptr, host_stream2 = nullptr, h2d_stream = nullptr,
                 d2h_stream = nullptr;
    static constexpr int kChunks = 32;   // chunks of the host path: short pipeline fill and drain
    cudaEvent_t ev_in[kChunks] = {}, ev_out[kChunks] = {};
};
