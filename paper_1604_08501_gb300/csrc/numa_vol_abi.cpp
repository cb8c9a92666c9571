// C ABI of the element volume term: argument checks, device memory of a
// handle, and dispatch to the kernels.  See include/numa_vol.h.
#include <cuda_runtime.h>

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

int numa_vol_diff_matrix(int N, double *D_out) {
    g_last_error.clear();
    if (!D_out) return fail(NUMA_EINVAL, "numa_vol_diff_matrix: D_out is NULL");
    if (N < 1 || N > NUMA_MAX_N)
        return fail(NUMA_EINVAL, "numa_vol_diff_matrix: N must be in [1, 7]");
    return numa::gll_diff_matrix(N, D_out);
}

int numa_vol_create(const numa_mesh *mesh, const numa_geometry *geo, const numa_constants *c,
                    numa_precision prec, numa_vol **out) {
    g_last_error.clear();
    if (!out) return fail(NUMA_EINVAL, "numa_vol_create: out is NULL");
    *out = nullptr;
    if (!mesh || !geo || !c) return fail(NUMA_EINVAL, "numa_vol_create: NULL argument");
    if (mesh->N < 1 || mesh->N > NUMA_MAX_N)
        return fail(NUMA_EINVAL, "numa_vol_create: N must be in [1, 7]");
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
    if (prec != NUMA_FP64)
        return fail(NUMA_EUNSUPPORTED, "numa_vol_create: only NUMA_FP64 is implemented");

    numa_vol *h = new (std::nothrow) numa_vol();
    if (!h) return fail(NUMA_ENOMEM, "numa_vol_create: host allocation failed");
    h->N = mesh->N;
    h->Nq = mesh->N + 1;
    h->Ne = mesh->num_elements;
    h->M = h->Ne * h->Nq * h->Nq * h->Nq;
    h->prec = prec;
    h->eos = numa::EosConstants{c->p0, c->R, c->cp / (c->cp - c->R), c->grav};

    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) {
        delete h;
        return fail_cuda(e, "numa_vol_create: cudaGetDevice");
    }

    double D[(NUMA_MAX_N + 1) * (NUMA_MAX_N + 1)];
    numa::gll_diff_matrix(h->N, D);

    // Block layout: g[0..8], Jinv, rho_ref, p_ref (each padded(M)), then D.
    const int64_t P = padded(h->M);
    h->block_bytes = sizeof(double) * (12 * P + h->Nq * h->Nq);
    e = cudaMalloc(&h->d_block, h->block_bytes);
    if (e != cudaSuccess) {
        delete h;
        return fail_cuda(e, "numa_vol_create: cudaMalloc of geometry");
    }
    double *base = static_cast<double *>(h->d_block);
    double *slots[12];
    for (int s = 0; s < 12; ++s) slots[s] = base + s * P;
    double *dD = base + 12 * P;
    const size_t bytes = sizeof(double) * h->M;
    const double *src[11] = {geo->g[0], geo->g[1], geo->g[2], geo->g[3], geo->g[4], geo->g[5],
                             geo->g[6], geo->g[7], geo->g[8], geo->Jinv, geo->rho_ref};
    for (int s = 0; s < 11 && e == cudaSuccess; ++s)
        if (bytes) e = cudaMemcpy(slots[s], src[s], bytes, cudaMemcpyDefault);
    if (e == cudaSuccess) e = cudaMemcpy(dD, D, sizeof(double) * h->Nq * h->Nq, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = numa::launch_pref_fp64(geo->rhotheta_ref, slots[11], h->M, h->eos, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) {
        cudaFree(h->d_block);
        delete h;
        return fail_cuda(e, "numa_vol_create: upload of geometry");
    }
    for (int s = 0; s < 9; ++s) h->geo.g[s] = slots[s];
    h->geo.Jinv = slots[9];
    h->geo.rho_ref = slots[10];
    h->geo.p_ref = slots[11];
    h->geo.D = dD;
    *out = h;
    return NUMA_OK;
}

int numa_vol_rhs(numa_vol *h, const void *q, void *rhs, void *stream) {
    g_last_error.clear();
    if (!h) return fail(NUMA_EINVAL, "numa_vol_rhs: NULL handle");
    if (h->Ne == 0) return NUMA_OK;
    if (!q || !rhs) return fail(NUMA_EINVAL, "numa_vol_rhs: NULL q or rhs");
    if (!aligned16(q) || !aligned16(rhs))
        return fail(NUMA_EINVAL, "numa_vol_rhs: q and rhs must be 16-byte aligned");
    const size_t bytes = sizeof(double) * numa::kFields * h->M;
    if (overlap(q, rhs, bytes)) return fail(NUMA_EINVAL, "numa_vol_rhs: q and rhs overlap");
    if (!is_device_pointer(q) || !is_device_pointer(rhs))
        return fail(NUMA_EINVAL, "numa_vol_rhs: q and rhs must be device pointers");
    cudaError_t e = numa::launch_vol_rhs_fp64(h->N, h->Ne, h->geo, h->eos,
                                              static_cast<const double *>(q),
                                              static_cast<double *>(rhs),
                                              static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail_cuda(e, "numa_vol_rhs: launch");
    return NUMA_OK;
}

int numa_vol_rhs_host(numa_vol *h, const double *q, double *rhs) {
    g_last_error.clear();
    if (!h) return fail(NUMA_EINVAL, "numa_vol_rhs_host: NULL handle");
    if (h->Ne == 0) return NUMA_OK;
    if (!q || !rhs) return fail(NUMA_EINVAL, "numa_vol_rhs_host: NULL q or rhs");
    const size_t bytes = sizeof(double) * numa::kFields * h->M;
    if (overlap(q, rhs, bytes)) return fail(NUMA_EINVAL, "numa_vol_rhs_host: q and rhs overlap");
    cudaError_t e = cudaSuccess;
    if (!h->host_stream) e = cudaStreamCreateWithFlags(&h->host_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return fail_cuda(e, "numa_vol_rhs_host: stream");
    if (!h->d_stage) {
        e = cudaMalloc(&h->d_stage, 2 * bytes);
        if (e != cudaSuccess) {
            h->d_stage = nullptr;
            return fail_cuda(e, "numa_vol_rhs_host: staging allocation");
        }
    }
    double *dq = h->d_stage;
    double *dr = h->d_stage + numa::kFields * h->M;
    e = cudaMemcpyAsync(dq, q, bytes, cudaMemcpyHostToDevice, h->host_stream);
    if (e == cudaSuccess)
        e = numa::launch_vol_rhs_fp64(h->N, h->Ne, h->geo, h->eos, dq, dr, h->host_stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(rhs, dr, bytes, cudaMemcpyDeviceToHost, h->host_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->host_stream);
    if (e != cudaSuccess) return fail_cuda(e, "numa_vol_rhs_host");
    return NUMA_OK;
}

void numa_vol_destroy(numa_vol *h) {
    if (!h) return;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != h->device) cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    if (h->host_stream) cudaStreamDestroy(h->host_stream);
    cudaFree(h->d_stage);
    cudaFree(h->d_block);
    if (cur != h->device) cudaSetDevice(cur);
    delete h;
}

}  // extern "C"
