// Internal declarations of the numa_vol library (not part of the C ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "numa_vol.h"

namespace numa {

constexpr int kFields = 5;

// Device-side geometry of one handle. Every per-point array has M entries,
// padded so that each starts on a 256-byte boundary.
struct DeviceGeometry {
    const double *g[9];     // metric terms g[3*d + a]
    const double *Jinv;     // 1 / J
    const double *rho_ref;  // reference density
    const double *p_ref;    // p(Theta_ref), evaluated once at create time
    const double *D;        // (N+1)^2, row-major D[i*Nq + n]
};

struct EosConstants {
    double p0, R, gamma, grav;
};

// Launchers (vol_fp64.cu). They return a cudaError_t from the launch.
cudaError_t launch_pref_fp64(const double *rhotheta_ref, double *p_ref, int64_t M,
                             EosConstants c, cudaStream_t s);
cudaError_t launch_vol_rhs_fp64(int N, int64_t Ne, const DeviceGeometry &geo, EosConstants c,
                                const double *q, double *rhs, cudaStream_t s);

// GLL points and differentiation matrix on the host (gll.cpp).
int gll_diff_matrix(int N, double *D);

}  // namespace numa

struct numa_vol {
    int N = 0;
    int Nq = 0;
    int64_t Ne = 0;
    int64_t M = 0;
    int device = 0;
    numa_precision prec = NUMA_FP64;
    numa::EosConstants eos{};
    void *d_block = nullptr;        // one allocation: geometry, reference state, D
    size_t block_bytes = 0;
    numa::DeviceGeometry geo{};
    double *d_stage = nullptr;      // host entry point: q and rhs staging, 2 * 5 * M
    cudaStream_t host_stream = nullptr;
};
