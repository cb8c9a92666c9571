// C ABI of the element volume term: argument checks, device memory of a
// handle, and dispatch to the kernels.  See include/numa_vol.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>

#include "numa_internal.h"
#include "numa_vol.h"

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

int fail_cuda(cudaError_t e, const char *where) {
    // Reset the runtime's last-error state: a non-sticky error (an allocation
    // refused) is reported here, not again by the next unrelated launch check.
    cudaGetLastError();
    int code = (e == cudaErrorMemoryAllocation) ? NUMA_ENOMEM : NUMA_ECUDA;
    return fail(code, std::string(where) + ": " + cudaGetErrorName(e) + " (" +
                          cudaGetErrorString(e) + ")");
}

// Per-point arrays start on 256-byte boundaries inside the handle's block.
int64_t padded(int64_t M) { return (M + 31) / 32 * 32; }

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

bool overlap(const void *a, const void *b, size_t bytes) {
    auto x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + bytes && y < x + bytes;
}

// Device (or managed) memory the current device can address directly.
bool is_device_pointer(const void *p) {
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();  // clear the sticky-free error of an unknown pointer
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

const char *numa_vol_last_error(void) { return g_last_error.c_str(); }

const char *numa_vol_kernel_name(const numa_vol *h) {
    static const char *native[] = {"", "vol_rhs_fp64_kernel<2>", "vol_rhs_fp64_kernel<3>",
                                   "vol_rhs_fp64_kernel<4>", "vol_rhs_fp64_kernel<5>",
                                   "vol_rhs_fp64_kernel<6>", "vol_rhs_fp64_kernel<7>",
                                   "vol_rhs_fp64_kernel<8>", "vol_rhs_high_kernel<9, double>",
                                   "vol_rhs_high_kernel<10, double>", "vol_rhs_high_kernel<11, double>",
                                   "vol_rhs_high_kernel<12, double>", "vol_rhs_high_kernel<13, double>",
                                   "vol_rhs_high_kernel<14, double>", "vol_rhs_high_kernel<15, double>",
                                   "vol_rhs_high_kernel<16, double>"};
    if (!h) return "";
    static const char *mixed[] = {"", "vol_rhs_mixed_kernel<2>", "vol_rhs_mixed_kernel<3>",
                                  "vol_rhs_mixed_kernel<4>", "vol_rhs_mixed_kernel<5>",
                                  "vol_rhs_mixed_kernel<6>", "vol_rhs_mixed_kernel<7>",
                                  "vol_rhs_mixed_kernel<8>"};
    static const char *dfk[] = {"", "vol_rhs_df64_kernel<2>", "vol_rhs_df64_kernel<3>",
                                "vol_rhs_df64_kernel<4>", "vol_rhs_df64_kernel<5>",
                                "vol_rhs_df64_kernel<6>", "vol_rhs_df64_kernel<7>",
                                "vol_rhs_df64_kernel<8>"};
    if (h->kernel == numa::Kernel::DoubleFloat) return dfk[h->N];
    if (h->kernel == numa::Kernel::Mixed && h->tc_sweep) return "vol_rhs_mixed_tc_kernel<8>";
    if (h->kernel == numa::Kernel::Mixed) return mixed[h->N];
    if (h->kernel == numa::Kernel::MixedHigh) {
        static const char *mixed_high[] = {"vol_rhs_high_kernel<9, float>", "vol_rhs_high_kernel<10, float>",
                                           "vol_rhs_high_kernel<11, float>", "vol_rhs_high_kernel<12, float>",
                                           "vol_rhs_high_kernel<13, float>", "vol_rhs_high_kernel<14, float>",
                                           "vol_rhs_high_kernel<15, float>", "vol_rhs_high_kernel<16, float>"};
        return mixed_high[h->N - 8];
    }
    return native[h->N];
}

int numa_vol_set_sweep(numa_vol *h, numa_sweep sweep) {
    g_last_error.clear();
    if (!h) return fail(NUMA_EINVAL, "numa_vol_set_sweep: NULL handle");
    if (sweep != NUMA_SWEEP_CUDA_CORES && sweep != NUMA_SWEEP_TENSOR_TF32)
        return fail(NUMA_EINVAL, "numa_vol_set_sweep: NUMA_SWEEP_CUDA_CORES or NUMA_SWEEP_TENSOR_TF32");
    if (sweep == NUMA_SWEEP_CUDA_CORES) {
        h->tc_sweep = false;
        return NUMA_OK;
    }
    if (h->kernel != numa::Kernel::Mixed || h->N != 7 || h->nf != numa::kFields)
        return fail(NUMA_EUNSUPPORTED, "numa_vol_set_sweep: the tensor-core sweep takes NUMA_MIXED "
                                       "handles of N = 7 without tracers");
    const cudaError_t e = numa::prepare_vol_rhs_mixed_tc();
    if (e != cudaSuccess) return fail_cuda(e, "numa_vol_set_sweep");
    h->tc_sweep = true;
    return NUMA_OK;
}

int numa_vol_diff_matrix(int N, double *D_out) {
    g_last_error.clear();
    if (!D_out) return fail(NUMA_EINVAL, "numa_vol_diff_matrix: D_out is NULL");
    if (N < 1 || N > NUMA_MAX_N_FP64)
        return fail(NUMA_EINVAL, "numa_vol_diff_matrix: N must be in [1, 15]");
    return numa::gll_diff_matrix(N, D_out);
}

}  // extern "C"

namespace {

// Host split of a double into a df constant (round-to-nearest pieces).
numa::df split_host(long double x) {
    const float h = static_cast<float>(x);
    const float l = static_cast<float>(x - static_cast<long double>(h));
    return numa::df{h, l};
}

// binom(gamma, k) for k = 0..16, in long double.
void binomial_coefficients(double gamma, long double c[17]) {
    c[0] = 1.0L;
    for (int k = 1; k < 17; ++k) c[k] = c[k - 1] * ((long double)gamma - (k - 1)) / k;
}

void build_params(numa_vol *h, const double *D) {
    long double c[17];
    binomial_coefficients(h->eos.gamma, c);
    h->nparams.eos = h->eos;
    for (int k = 0; k < 15; ++k) h->nparams.c[k] = static_cast<double>(c[k + 1]);
    const long double g = h->eos.gamma;
    const float K = static_cast<float>(std::pow((long double)h->eos.p0, 1.0L - g) *
                                       std::pow((long double)h->eos.R, g));
    if (h->N >= 8) {   // the high-order kernels' parameters (FP64 and mixed)
        h->hparams.eos = h->eos;
        for (int k = 0; k < 15; ++k) h->hparams.c[k] = h->nparams.c[k];
        numa::sweep_tables(h->N, D, h->hparams.De, h->hparams.Do, h->hparams.Dc, h->hparams.Dcr);
        numa::HighParams32 &m = h->hmparams;
        for (int t = 0; t < 64; ++t) {
            m.De[t] = static_cast<float>(h->hparams.De[t]);
            m.Do[t] = static_cast<float>(h->hparams.Do[t]);
        }
        for (int t = 0; t < 8; ++t) {
            m.Dc[t] = static_cast<float>(h->hparams.Dc[t]);
            m.Dcr[t] = static_cast<float>(h->hparams.Dcr[t]);
        }
        for (int k = 0; k < 16; ++k) m.c[k] = static_cast<float>(c[k + 1]);
        m.K = K;
        m.gm1 = static_cast<float>(g - 1.0L);
        m.gamma = static_cast<float>(g);
        m.grav = static_cast<float>(h->eos.grav);
        return;
    }
    numa::sweep_tables(h->N, D, h->nparams.De, h->nparams.Do, h->nparams.Dc, h->nparams.Dcr);
    {
        numa::MixedParams &m = h->mparams;
        for (int t = 0; t < 16; ++t) {
            m.De[t] = static_cast<float>(h->nparams.De[t]);
            m.Do[t] = static_cast<float>(h->nparams.Do[t]);
        }
        for (int t = 0; t < 4; ++t) {
            m.Dc[t] = static_cast<float>(h->nparams.Dc[t]);
            m.Dcr[t] = static_cast<float>(h->nparams.Dcr[t]);
        }
        for (int k = 0; k < 16; ++k) m.c[k] = static_cast<float>(c[k + 1]);
        m.K = K;
        m.gm1 = static_cast<float>(g - 1.0L);
        m.gamma = static_cast<float>(g);
        m.grav = static_cast<float>(h->eos.grav);
    }
    if (h->N > NUMA_MAX_N) return;
    numa::DfParams &P = h->dparams;
    const int nq = h->Nq, N = h->N, half = nq / 2, cc = nq / 2;
    for (int i = 0; i < half; ++i) {
        for (int m = 0; m < half; ++m) {
            const long double a = D[i * nq + m], b = D[i * nq + N - m];
            P.De[i][m] = split_host((a + b) / 2);
            P.Do[i][m] = split_host((a - b) / 2);
        }
        if (nq & 1) {
            P.Dc[i] = split_host(D[i * nq + cc]);
            P.Dcr[i] = split_host(D[cc * nq + i]);
        }
    }
    P.c1 = split_host(c[1]);
    P.c2 = split_host(c[2]);
    P.c3 = split_host(c[3]);
    for (int k = 4; k < 10; ++k) P.ct[k - 4] = static_cast<float>(c[k]);
    P.grav_df = split_host(h->eos.grav);
    P.grav = h->eos.grav;
    P.p0 = h->eos.p0;
    P.R = h->eos.R;
    P.gamma = h->eos.gamma;
    for (int t = 0; t < nq * nq; ++t) P.D[t] = D[t];
}

// Per-point arrays of a handle, in order: g[0..8], Jinv, rho_ref, theta_ref,
// w = 1/theta_ref, A = p(theta_ref)/theta_ref.
constexpr int kArrays = 14;

// Stage the caller's arrays and the derived reference arrays as FP64 in
// `dst` (kArrays slots of P doubles each).
cudaError_t stage_fp64(numa_vol *h, const numa_geometry *geo, double *const *dst) {
    const size_t bytes = sizeof(double) * h->M;
    const double *src[12] = {geo->g[0], geo->g[1], geo->g[2], geo->g[3], geo->g[4], geo->g[5],
                             geo->g[6], geo->g[7], geo->g[8], geo->Jinv, geo->rho_ref,
                             geo->rhotheta_ref};
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < 12 && e == cudaSuccess; ++s)
        if (bytes) e = cudaMemcpy(dst[s], src[s], bytes, cudaMemcpyDefault);
    if (e == cudaSuccess) e = numa::launch_reference_eos(dst[11], dst[12], dst[13], h->M, h->eos, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    return e;
}

// Native layout: kArrays FP64 arrays (each padded(M)), then D.
cudaError_t create_native(numa_vol *h, const numa_geometry *geo, const double *D) {
    const int64_t P = padded(h->M);
    h->block_bytes = sizeof(double) * (kArrays * P + h->Nq * h->Nq);
    cudaError_t e = cudaMalloc(&h->d_block, h->block_bytes);
    if (e != cudaSuccess) {
        h->d_block = nullptr;
        return e;
    }
    double *base = static_cast<double *>(h->d_block);
    double *slots[kArrays];
    for (int s = 0; s < kArrays; ++s) slots[s] = base + s * P;
    double *dD = base + kArrays * P;
    e = stage_fp64(h, geo, slots);
    if (e == cudaSuccess)
        e = cudaMemcpy(dD, D, sizeof(double) * h->Nq * h->Nq, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    for (int s = 0; s < 9; ++s) h->geo.g[s] = slots[s];
    h->geo.Jinv = slots[9];
    h->geo.rho_ref = slots[10];
    h->geo.theta_ref = slots[11];
    h->geo.w = slots[12];
    h->geo.A = slots[13];
    h->geo.D = dD;
    h->kernel = h->N > NUMA_MAX_N ? numa::Kernel::NativeHigh : numa::Kernel::Native;
    return cudaSuccess;
}

// Mixed layout: 12 FP32 arrays (g[0..8], Jinv, rho_ref, theta_ref).
cudaError_t create_mixed(numa_vol *h, const numa_geometry *geo) {
    const int64_t P = padded(h->M);
    h->block_bytes = sizeof(float) * 12 * P;
    cudaError_t e = cudaMalloc(&h->d_block, h->block_bytes);
    if (e != cudaSuccess) {
        h->d_block = nullptr;
        return e;
    }
    double *tmp = nullptr;
    e = cudaMalloc(&tmp, sizeof(double) * (P > 0 ? P : 1));
    if (e != cudaSuccess) return e;
    float *base = static_cast<float *>(h->d_block);
    float *slots[12];
    for (int s = 0; s < 12; ++s) slots[s] = base + s * P;
    const double *src[12] = {geo->g[0], geo->g[1], geo->g[2], geo->g[3], geo->g[4], geo->g[5],
                             geo->g[6], geo->g[7], geo->g[8], geo->Jinv, geo->rho_ref,
                             geo->rhotheta_ref};
    const size_t bytes = sizeof(double) * h->M;
    for (int s = 0; s < 12 && e == cudaSuccess; ++s) {
        if (bytes) e = cudaMemcpy(tmp, src[s], bytes, cudaMemcpyDefault);
        if (e == cudaSuccess) e = numa::launch_to_f32(tmp, slots[s], h->M, 0);
        if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    }
    cudaFree(tmp);
    if (e != cudaSuccess) return e;
    for (int s = 0; s < 9; ++s) h->mgeo.g[s] = slots[s];
    h->mgeo.Jinv = slots[9];
    h->mgeo.rho_ref = slots[10];
    h->mgeo.theta_ref = slots[11];
    h->kernel = h->N > NUMA_MAX_N ? numa::Kernel::MixedHigh : numa::Kernel::Mixed;
    h->elem = sizeof(float);
    return cudaSuccess;
}

// Double-float layout: kArrays float2 arrays.  Sets *in_range = false (and
// keeps nothing) if a value stays outside the fast-path range after the
// relative flush of rounding noise.
cudaError_t create_df(numa_vol *h, const numa_geometry *geo, bool *in_range) {
    *in_range = true;
    const int64_t P = padded(h->M);
    h->block_bytes = sizeof(float2) * kArrays * P;
    cudaError_t e = cudaMalloc(&h->d_block, h->block_bytes);
    if (e != cudaSuccess) {
        h->d_block = nullptr;
        return e;
    }
    void *tmp = nullptr;
    e = cudaMalloc(&tmp, sizeof(double) * kArrays * P + 256);
    if (e != cudaSuccess) {
        cudaFree(h->d_block);
        h->d_block = nullptr;
        return e;
    }
    double *staged[kArrays];
    for (int s = 0; s < kArrays; ++s) staged[s] = static_cast<double *>(tmp) + s * P;
    unsigned long long *d_amax = reinterpret_cast<unsigned long long *>(
        static_cast<double *>(tmp) + kArrays * P);
    int *d_bad = reinterpret_cast<int *>(d_amax + kArrays);
    float2 *base = static_cast<float2 *>(h->d_block);
    float2 *slots[kArrays];
    for (int s = 0; s < kArrays; ++s) slots[s] = base + s * P;
    e = stage_fp64(h, geo, staged);
    if (e == cudaSuccess) e = cudaMemset(d_amax, 0, sizeof(unsigned long long) * kArrays + sizeof(int));
    for (int s = 0; s < kArrays && e == cudaSuccess; ++s)
        e = numa::launch_abs_max(staged[s], h->M, d_amax + s, 0);
    unsigned long long amax[kArrays] = {};
    if (e == cudaSuccess)
        e = cudaMemcpy(amax, d_amax, sizeof(amax), cudaMemcpyDeviceToHost);
    for (int s = 0; s < kArrays && e == cudaSuccess; ++s) {
        if (s == 10 || s == 11) {   // rho_ref and theta_ref stay FP64
            if (h->M) e = cudaMemcpy(slots[s], staged[s], sizeof(double) * h->M,
                                     cudaMemcpyDeviceToDevice);
            continue;
        }
        double mx;
        std::memcpy(&mx, &amax[s], sizeof(double));
        e = numa::launch_to_df(staged[s], slots[s], h->M, std::ldexp(mx, -50), d_bad, 0);
    }
    int bad = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(tmp);
    if (e != cudaSuccess || bad) {
        cudaFree(h->d_block);
        h->d_block = nullptr;
        *in_range = (e != cudaSuccess) || !bad;
        return e;
    }
    for (int s = 0; s < 9; ++s) h->dgeo.g[s] = slots[s];
    h->dgeo.Jinv = slots[9];
    h->dgeo.rho_ref = reinterpret_cast<const double *>(slots[10]);
    h->dgeo.theta_ref = reinterpret_cast<const double *>(slots[11]);
    h->dgeo.w = slots[12];
    h->dgeo.A = slots[13];
    h->kernel = numa::Kernel::DoubleFloat;
    return cudaSuccess;
}

}  // namespace

extern "C" {

int numa_vol_create(const numa_mesh *mesh, const numa_geometry *geo, const numa_constants *c,
                    numa_precision prec, numa_vol **out) {
    g_last_error.clear();
    if (!out) return fail(NUMA_EINVAL, "numa_vol_create: out is NULL");
    *out = nullptr;
    if (!mesh || !geo || !c) return fail(NUMA_EINVAL, "numa_vol_create: NULL argument");
    if (mesh->N < 1 || mesh->N > NUMA_MAX_N_FP64)
        return fail(NUMA_EINVAL, "numa_vol_create: N must be in [1, 15]");
    if (mesh->N > NUMA_MAX_N && prec == NUMA_DF64)
        return fail(NUMA_EUNSUPPORTED, "numa_vol_create: NUMA_DF64 is implemented for N = 1..7");
    if (mesh->num_tracers < 0 || mesh->num_tracers > NUMA_MAX_TRACERS)
        return fail(NUMA_EINVAL, "numa_vol_create: num_tracers must be in [0, 3]");
    if (mesh->num_elements < 0)
        return fail(NUMA_EINVAL, "numa_vol_create: num_elements must be >= 0");
    if (mesh->num_elements > (int64_t)INT32_MAX)
        return fail(NUMA_EINVAL, "numa_vol_create: num_elements exceeds 2^31 - 1");
    if (!(c->p0 > 0) || !(c->R > 0) || !(c->cp > c->R))
        return fail(NUMA_EINVAL, "numa_vol_create: need p0 > 0 and cp > R > 0");
    for (int s = 0; s < 9; ++s)
        if (!geo->g[s]) return fail(NUMA_EINVAL, "numa_vol_create: NULL metric array");
    if (!geo->Jinv || !geo->rho_ref || !geo->rhotheta_ref)
        return fail(NUMA_EINVAL, "numa_vol_create: NULL Jinv or reference array");
    if (prec != NUMA_FP64 && prec != NUMA_DF64 && prec != NUMA_MIXED)
        return fail(NUMA_EINVAL, "numa_vol_create: unknown precision");

    numa_vol *h = new (std::nothrow) numa_vol();
    if (!h) return fail(NUMA_ENOMEM, "numa_vol_create: host allocation failed");
    h->N = mesh->N;
    h->Nq = mesh->N + 1;
    h->nf = numa::kFields + mesh->num_tracers;
    h->Ne = mesh->num_elements;
    h->M = h->Ne * h->Nq * h->Nq * h->Nq;
    h->prec = prec;
    h->eos = numa::EosConstants{c->p0, c->R, c->cp / (c->cp - c->R), c->grav};

    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) {
        delete h;
        return fail_cuda(e, "numa_vol_create: cudaGetDevice");
    }
    e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_err, 256);
    if (e == cudaSuccess) e = cudaMemset(h->d_err, 0, 256);
    if (e != cudaSuccess) {
        cudaFree(h->d_err);
        delete h;
        return fail_cuda(e, "numa_vol_create: status word");
    }
    double D[(NUMA_MAX_N_FP64 + 1) * (NUMA_MAX_N_FP64 + 1)];
    numa::gll_diff_matrix(h->N, D);

    build_params(h, D);
    bool use_native = prec == NUMA_FP64;
    if (prec == NUMA_MIXED) {
        e = create_mixed(h, geo);
        use_native = false;
    } else if (!use_native) {
        bool in_range = true;
        e = create_df(h, geo, &in_range);
        if (e == cudaSuccess && !in_range) use_native = true;   // geometry out of range
    }
    if (use_native && e == cudaSuccess) e = create_native(h, geo, D);
    if (e != cudaSuccess) {
        cudaFree(h->d_block);
        cudaFree(h->d_err);
        delete h;
        return fail_cuda(e, "numa_vol_create: upload of geometry");
    }
    *out = h;
    return NUMA_OK;
}

}  // extern "C"

namespace {

// Elements [e0, e0 + count) of the handle's mesh.
cudaError_t launch(numa_vol *h, const void *q, void *rhs, int64_t e0, int64_t count,
                   cudaStream_t s) {
    const numa::ElemRange r{e0, count, h->M};
    if (h->kernel == numa::Kernel::MixedHigh)
        return numa::launch_vol_rhs_mixed_high(h->N, h->nf, r, h->mgeo, h->hmparams,
                                               static_cast<const float *>(q),
                                               static_cast<float *>(rhs), h->num_sms, s);
    if (h->kernel == numa::Kernel::Mixed && h->tc_sweep)
        return numa::launch_vol_rhs_mixed_tc(r, h->mgeo, h->mparams, static_cast<const float *>(q),
                                             static_cast<float *>(rhs), h->num_sms, h->d_err, s);
    if (h->kernel == numa::Kernel::Mixed)
        return numa::launch_vol_rhs_mixed(h->N, h->nf, r, h->mgeo, h->mparams,
                                          static_cast<const float *>(q), static_cast<float *>(rhs),
                                          h->num_sms, s);
    if (h->kernel == numa::Kernel::DoubleFloat)
        return numa::launch_vol_rhs_df64(h->N, h->nf, r, h->dgeo, h->dparams,
                                         static_cast<const double *>(q),
                                         static_cast<double *>(rhs), h->num_sms, s);
    if (h->kernel == numa::Kernel::NativeHigh)
        return numa::launch_vol_rhs_fp64_high(h->N, h->nf, r, h->geo, h->hparams,
                                              static_cast<const double *>(q),
                                              static_cast<double *>(rhs), s);
    return numa::launch_vol_rhs_fp64(h->N, h->nf, r, h->geo, h->nparams,
                                     static_cast<const double *>(q), static_cast<double *>(rhs), s);
}

}  // namespace

extern "C" {

int numa_vol_rhs(numa_vol *h, const void *q, void *rhs, void *stream) {
    g_last_error.clear();
    if (!h) return fail(NUMA_EINVAL, "numa_vol_rhs: NULL handle");
    if (h->Ne == 0) return NUMA_OK;
    if (!q || !rhs) return fail(NUMA_EINVAL, "numa_vol_rhs: NULL q or rhs");
    if (!aligned16(q) || !aligned16(rhs))
        return fail(NUMA_EINVAL, "numa_vol_rhs: q and rhs must be 16-byte aligned");
    const size_t bytes = h->elem * h->nf * h->M;
    if (overlap(q, rhs, bytes)) return fail(NUMA_EINVAL, "numa_vol_rhs: q and rhs overlap");
    if (!is_device_pointer(q) || !is_device_pointer(rhs))
        return fail(NUMA_EINVAL, "numa_vol_rhs: q and rhs must be device pointers");
    cudaError_t e = launch(h, q, rhs, 0, h->Ne, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail_cuda(e, "numa_vol_rhs: launch");
    return NUMA_OK;
}

int numa_vol_rhs_host(numa_vol *h, const void *q, void *rhs) {
    g_last_error.clear();
    if (!h) return fail(NUMA_EINVAL, "numa_vol_rhs_host: NULL handle");
    if (h->Ne == 0) return NUMA_OK;
    if (!q || !rhs) return fail(NUMA_EINVAL, "numa_vol_rhs_host: NULL q or rhs");
    const size_t bytes = h->elem * h->nf * h->M;
    if (overlap(q, rhs, bytes)) return fail(NUMA_EINVAL, "numa_vol_rhs_host: q and rhs overlap");
    cudaError_t e = cudaSuccess;
    if (!h->host_stream) {
        e = cudaStreamCreateWithFlags(&h->host_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->host_stream2, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->h2d_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->d2h_stream, cudaStreamNonBlocking);
        for (int c = 0; c < numa_vol::kChunks && e == cudaSuccess; ++c) {
            e = cudaEventCreateWithFlags(&h->ev_in[c], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_out[c], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return fail_cuda(e, "numa_vol_rhs_host: streams");
    }
    if (!h->d_stage) {
        e = cudaMalloc(&h->d_stage, 2 * bytes);
        if (e != cudaSuccess) {
            h->d_stage = nullptr;
            return fail_cuda(e, "numa_vol_rhs_host: staging allocation");
        }
    }
    // Chunks of elements flow through four streams: copy-in of chunk c + 1,
    // compute of chunk c (two compute streams in turn, so that consecutive
    // chunks' kernels overlap at their ends) and copy-out of chunk c - 1.
    char *dq = static_cast<char *>(h->d_stage);
    char *dr = dq + bytes;
    const char *hq = static_cast<const char *>(q);
    char *hr = static_cast<char *>(rhs);
    const int64_t n3 = (int64_t)h->Nq * h->Nq * h->Nq;
    // Native FP64: 64 chunks (the kernel dominates; a shorter fill and drain).
    // Double-float and FP32 states: 16 (the copies dominate; fewer, larger
    // copies).  Measured on GB300 (pinned host memory, 193-210 GB/s each way,
    // 341 GB/s both at once): double-float 3.84 GDOF/s end to end against
    // 3.15-3.64 with 64 chunks, mixed 7.38 against 7.08 with 32.
    const int64_t target =
        h->elem == sizeof(double) && h->kernel != numa::Kernel::DoubleFloat ? numa_vol::kChunks : 16;
    const int chunks = (int)std::min<int64_t>(target, h->Ne);
    const size_t plane = h->elem * h->M;
    // One 2D copy per chunk and direction moves the chunk's slice of every
    // field plane (pitch = the plane stride).
    for (int c = 0; c < chunks && e == cudaSuccess; ++c) {
        const int64_t e0 = h->Ne * c / chunks, e1 = h->Ne * (c + 1) / chunks;
        const size_t off = h->elem * e0 * n3, len = h->elem * (e1 - e0) * n3;
        e = cudaMemcpy2DAsync(dq + off, plane, hq + off, plane, len, (size_t)h->nf,
                              cudaMemcpyHostToDevice, h->h2d_stream);
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_in[c], h->h2d_stream);
        cudaStream_t cs = (c & 1) ? h->host_stream2 : h->host_stream;
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, h->ev_in[c], 0);
        if (e == cudaSuccess) e = launch(h, dq, dr, e0, e1 - e0, cs);
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_out[c], cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->d2h_stream, h->ev_out[c], 0);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(hr + off, plane, dr + off, plane, len, (size_t)h->nf,
                                  cudaMemcpyDeviceToHost, h->d2h_stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->d2h_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->host_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->host_stream2);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->h2d_stream);
    if (e != cudaSuccess) return fail_cuda(e, "numa_vol_rhs_host");
    return numa_vol_status(h, h->host_stream);
}

int numa_vol_status(numa_vol *h, void *stream) {
    if (!h) return fail(NUMA_EINVAL, "numa_vol_status: NULL handle");
    int flag = 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(&flag, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && flag) e = cudaMemsetAsync(h->d_err, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda(e, "numa_vol_status");
    if (flag) return fail(NUMA_ETIMEOUT, "numa_vol_status: a kernel gave up a bounded device-side "
                                         "wait; its results are incomplete");
    return NUMA_OK;
}

void numa_vol_destroy(numa_vol *h) {
    if (!h) return;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != h->device) cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    if (h->host_stream) cudaStreamDestroy(h->host_stream);
    if (h->host_stream2) cudaStreamDestroy(h->host_stream2);
    if (h->h2d_stream) cudaStreamDestroy(h->h2d_stream);
    if (h->d2h_stream) cudaStreamDestroy(h->d2h_stream);
    for (int c = 0; c < numa_vol::kChunks; ++c) {
        if (h->ev_in[c]) cudaEventDestroy(h->ev_in[c]);
        if (h->ev_out[c]) cudaEventDestroy(h->ev_out[c]);
    }
    cudaFree(h->d_stage);
    cudaFree(h->d_block);
    cudaFree(h->d_err);
    if (cur != h->device) cudaSetDevice(cur);
    delete h;
}

}  // extern "C"
