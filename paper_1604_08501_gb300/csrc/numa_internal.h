// Internal declarations of the numa_vol library (not part of the C ABI).
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "kernel_params.h"
#include "numa_vol.h"

namespace numa {

// Launchers (vol_fp64.cu). They return a cudaError_t from the launch.
// reference_eos: w = 1/Theta_ref, A = p(Theta_ref)/Theta_ref per point.
cudaError_t launch_reference_eos(const double *theta_ref, double *w, double *A, int64_t M,
                                 EosConstants c, cudaStream_t s);
// Native FP64 for N = 8..15 (vol_fp64_high.cu): one CTA of 3 Nq^2 threads
// per element, one pass per field.
// nf: 5 fields, or 5 + tracers (nf <= 8).
cudaError_t launch_vol_rhs_fp64_high(int N, int nf, ElemRange r, const DeviceGeometry &geo,
                                     const HighParams &P, const double *q, double *rhs,
                                     cudaStream_t s);
// Mixed precision for N = 8..15 (vol_fp64_high.cu, FP32 instantiation: a
// five-field and an eight-field form, chosen by nf; num_sms sets the
// distance of its L2 prefetch, one wave of resident CTAs).
cudaError_t launch_vol_rhs_mixed_high(int N, int nf, ElemRange r, const MixedGeometry &geo,
                                      const HighParams32 &P, const float *q, float *rhs,
                                      int num_sms, cudaStream_t s);
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
// nf: 5 fields, or 5 + tracers (nf <= 8).
cudaError_t launch_vol_rhs_df64(int N, int nf, ElemRange r, const DfGeometry &geo,
                                const DfParams &P, const double *q, double *rhs, int num_sms,
                                cudaStream_t s);

// Launchers of the mixed-precision path (vol_mixed.cu).
cudaError_t launch_to_f32(const double *src, float *dst, int64_t M, cudaStream_t s);
// One CTA per element (vol_rhs_mixed_kernel<Nq>), with an L2 prefetch of the
// element one wave ahead; num_sms sizes that wave.
cudaError_t launch_vol_rhs_mixed(int N, int nf, ElemRange r, const MixedGeometry &geo,
                                 const MixedParams &P, const float *q, float *rhs, int num_sms,
                                 cudaStream_t s);

// The mixed-precision kernel at N = 7 with the D sums on the tensor cores
// (vol_mixed_tc.cu): a persistent grid; a bounded wait that runs out sets
// bit 0 of *err.  prepare_vol_rhs_mixed_tc() once per device first (outside
// stream capture).
cudaError_t prepare_vol_rhs_mixed_tc();
cudaError_t launch_vol_rhs_mixed_tc(ElemRange r, const MixedGeometry &geo, const MixedParams &P,
                                    const float *q, float *rhs, int num_sms, int *err,
                                    cudaStream_t s);

// GLL points and differentiation matrix on the host (gll.cpp).
int gll_diff_matrix(int N, double *D);

// Even-odd sweep tables of the order-N GLL D (Nq = N + 1): De, Do
// ((Nq/2)^2, row-major), Dc, Dcr (odd Nq).  Unused entries are zero.
void sweep_tables(int N, const double *D, double De[16], double Do[16], double Dc[4],
                  double Dcr[4]);

// Native: vol_rhs_fp64_kernel (N <= 7); NativeHigh: vol_rhs_high_kernel<Nq, double>
// (N = 8..15); DoubleFloat (vol_rhs_df64_kernel<Nq>, N <= 7); Mixed (N <= 7) and MixedHigh:
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
    int nf;       // fields: 5, or 5 + tracers (the tracer forms of the tiles only)
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
// The grid is num_sms times the CTAs per SM the kernel is built for.  tc_mask
// (mixed only): bit Nq set = order Nq takes its D contractions as TF32 split
// products on the tensor cores (batch_tile_tc.cuh); counter[1] then receives
// the kernel's status bits.
constexpr unsigned kTcAllOrders = 0x1FCu;   // bits 2..8
// ctas_per_sm: CTAs per SM of the persistent grid, 1 .. the kernel's maximum
// (batch_max_ctas_per_sm); 0 takes the maximum.  tmem_state (mixed): the
// CUDA-core tiles keep each point's state in tensor memory instead of shared
// memory (the tensor-core kernel's CUDA-core path).  tracers: some instance
// has nf > 5; the launch then runs the shared-memory-state tiles' tracer forms
// and tc_mask and tmem_state have no effect.
cudaError_t launch_batch_lsrk(bool mixed, const BatchInstance *inst, const BatchItem *items,
                              int num_items, int *counter, const LsrkCoef &co, int nsteps,
                              double dt, int num_sms, cudaStream_t s, unsigned tc_mask = 0,
                              int ctas_per_sm = 0, bool tmem_state = false,
                              bool tracers = false);
int batch_max_ctas_per_sm(bool mixed);

// Elements one CTA pass holds for order Nq (512 threads, one per point).
inline int elements_per_pass(int nq) { return 512 / (nq * nq * nq); }

// Work list for instances with tile_mult[nq] passes per item (batch_abi.cu);
// costliest_first: items sorted by points, largest first (stable).
std::vector<BatchItem> build_items(const std::vector<BatchInstance> &inst, const int *tile_mult,
                                   bool costliest_first = false);

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
    bool tc_sweep = false;          // NUMA_MIXED, N = 7: the D sums on the tensor cores
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
    static constexpr int kChunks = 64;   // host path: at most this many chunks (short fill and drain)
    cudaEvent_t ev_in[kChunks] = {}, ev_out[kChunks] = {};
};
