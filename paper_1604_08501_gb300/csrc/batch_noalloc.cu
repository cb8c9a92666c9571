// A variant of the batched integrator (numa_batch_advance) that allocates no
// memory: for callers that must not call cudaMalloc once they are running.
// An example is a serving process that has committed its whole HBM budget to
// resident ensemble states, or an application whose allocator forbids growth
// after start-up.
//
// numa_batch_advance keeps its work list in device memory it allocates.  This
// variant keeps its scratch (the work counter and the instance table) in one
// file-scope __device__ array of fixed size, sized for at most
// NUMA_NOALLOC_MAX_INSTANCES instances.  The host side builds the table on its
// own stack, and the kernel derives each work item from per-instance offsets
// in the table.  The per-tile arithmetic is the same device code as the
// allocating entry point's (batch_tile.cuh), with the same tiles.
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <mutex>

#include "batch_tile.cuh"
#include "numa_vol.h"

namespace numa {

namespace {

constexpr int kMaxInst = NUMA_NOALLOC_MAX_INSTANCES;
constexpr int kPassesPerItem = 4;   // elements per work item = 4 passes, the batch's default

struct NoallocTable {
    int count;                      // instances
    int num_items;                  // work items in total
    int first_item[kMaxInst + 1];   // work items before instance k (prefix sums)
    BatchInstance inst[kMaxInst];
};

// Scratch layout: the claim counter in the first 256 bytes, then the table.
constexpr size_t kCounterBytes = 256;
constexpr size_t kScratchBytes = kCounterBytes + (sizeof(NoallocTable) + 255) / 256 * 256;

// The only device memory this entry point uses.  Every GPU that loads the
// library holds it (about 57 KB) until the process exits.  Host code never
// dereferences this name: it stands in for the device address, which
// setup() obtains with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// TR: the tiles' tracer forms, for a call that holds an instance with tracers.
template <bool MIXED, bool TR>
__global__ void __launch_bounds__(kThreads, tile_ctas_per_sm<MIXED>())
batch_lsrk_noalloc_kernel(unsigned char *scratch, LsrkCoef co, int nsteps, double dt) {
    int *counter = reinterpret_cast<int *>(scratch);
    const NoallocTable *tab = reinterpret_cast<const NoallocTable *>(scratch + kCounterBytes);
    extern __shared__ __align__(16) double smem_d[];
    __shared__ BatchInstance sI;
    __shared__ int s_item;
    __shared__ tile_t<MIXED> sco[10];
    load_stage_coefficients<MIXED>(co, sco);   // visible after the first barrier below
    const int num_items = tab->num_items;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= num_items) break;
        int k = 0;   // the instance of item it: the last k with first_item[k] <= it
        while (k + 1 < tab->count && tab->first_item[k + 1] <= it) ++k;
        {
            const int *src = reinterpret_cast<const int *>(&tab->inst[k]);
            int *dst = reinterpret_cast<int *>(&sI);
            for (int w = threadIdx.x; w < (int)(sizeof(BatchInstance) / sizeof(int)); w += kThreads)
                dst[w] = src[w];
        }
        __syncthreads();
        const int nq = sI.nq;
        const int64_t ne = sI.M / ((int64_t)nq * nq * nq);
        const int64_t tile = (int64_t)(kThreads / (nq * nq * nq)) * kPassesPerItem;
        const int64_t e0 = (int64_t)(it - tab->first_item[k]) * tile;
        const int64_t count = ne - e0 < tile ? ne - e0 : tile;
        const int ns = sI.nsteps > 0 ? sI.nsteps : nsteps;
        switch (nq) {
            case 2: run_tile<2, MIXED, TR>(sI, e0, count, sco, ns, dt, smem_d); break;
            case 3: run_tile<3, MIXED, TR>(sI, e0, count, sco, ns, dt, smem_d); break;
            case 4: run_tile<4, MIXED, TR>(sI, e0, count, sco, ns, dt, smem_d); break;
            case 5: run_tile<5, MIXED, TR>(sI, e0, count, sco, ns, dt, smem_d); break;
            case 6: run_tile<6, MIXED, TR>(sI, e0, count, sco, ns, dt, smem_d); break;
            case 7: run_tile<7, MIXED, TR>(sI, e0, count, sco, ns, dt, smem_d); break;
            case 8: run_tile<8, MIXED, TR>(sI, e0, count, sco, ns, dt, smem_d); break;
            default: break;
        }
        __syncthreads();   // sI and s_item are rewritten by the next claim
    }
}

// Five-stage fourth-order 2N-storage coefficients (Carpenter and Kennedy,
// NASA TM-109112, 1994), as in numa_batch_advance.
const LsrkCoef kCoef = {
    {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
     -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0},
    {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
     1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
     2277821191437.0 / 14882151754819.0}};

// One-time set-up per device, with that device current: the device address of
// the scratch array, the sweep tables and the kernels' shared-memory opt-in.
constexpr int kMaxDevices = 64;
struct DeviceSetup {
    bool done;
    unsigned char *scratch;
    int num_sms;
};
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

cudaError_t setup(int dev, DeviceSetup *out) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup &s = g_setup[dev];
    if (!s.done) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&s.num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        e = upload_sweep_tables();
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(batch_lsrk_noalloc_kernel<false, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tile_smem_bytes<false>());
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(batch_lsrk_noalloc_kernel<true, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tile_smem_bytes<true>());
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(batch_lsrk_noalloc_kernel<false, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tile_smem_bytes<false, true>());
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(batch_lsrk_noalloc_kernel<true, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tile_smem_bytes<true, true>());
        if (e != cudaSuccess) return e;
        s.scratch = static_cast<unsigned char *>(p);
        s.done = true;
    }
    *out = s;
    return cudaSuccess;
}

}  // namespace

}  // namespace numa

extern "C" int numa_batch_advance_noalloc(const numa_vol *const *handles, void *const *states,
                                          int count, int nsteps, double dt, void *stream) {
    using namespace numa;
    if (!handles || !states || count < 1 || nsteps < 0) return NUMA_EINVAL;
    if (count > kMaxInst) return NUMA_ELIMIT;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return NUMA_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // The table is copied from this call's stack frame: a captured copy would
    // keep a pointer into a frame that is gone by the time the graph runs.
    // So a stream that is being captured is refused before anything is
    // enqueued (the capture stays valid).
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return NUMA_ECUDA;
    if (cap != cudaStreamCaptureStatusNone) return NUMA_EINVAL;
    const bool mixed = handles[0] && handles[0]->kernel == Kernel::Mixed;
    NoallocTable tab;   // on the stack: no heap
    bool tracers = false;   // some instance has tracers: the tiles' tracer forms
    tab.count = count;
    tab.first_item[0] = 0;
    for (int k = 0; k < count; ++k) {
        const numa_vol *h = handles[k];
        if (!h || !states[k] || (reinterpret_cast<uintptr_t>(states[k]) & 15u) != 0 ||
            h->device != dev)
            return NUMA_EINVAL;
        if (h->N > NUMA_MAX_N) return NUMA_EUNSUPPORTED;
        if (mixed ? h->kernel != Kernel::Mixed : h->kernel != Kernel::Native) return NUMA_EINVAL;
        BatchInstance &I = tab.inst[k];
        I = BatchInstance{};
        I.N = h->N;
        I.nq = h->Nq;
        I.nf = h->nf;
        tracers = tracers || h->nf > kFields;
        I.M = h->M;
        I.q = states[k];
        I.geo = h->geo;
        I.np = h->nparams;
        I.mgeo = h->mgeo;
        I.mp = h->mparams;
        const int64_t tile = (int64_t)elements_per_pass(h->Nq) * kPassesPerItem;
        const int64_t items = (h->Ne + tile - 1) / tile;
        if ((int64_t)tab.first_item[k] + items > INT32_MAX) return NUMA_ELIMIT;
        tab.first_item[k + 1] = tab.first_item[k] + (int)items;
    }
    tab.num_items = tab.first_item[count];
    if (nsteps == 0 || tab.num_items == 0) return NUMA_OK;

    DeviceSetup ds;
    if (setup(dev, &ds) != cudaSuccess) return NUMA_ECUDA;
    // The table's used part, from this stack frame (a pageable source is staged
    // before cudaMemcpyAsync returns), and a zeroed claim counter.
    const size_t used = offsetof(NoallocTable, inst) + sizeof(BatchInstance) * (size_t)count;
    if (cudaMemcpyAsync(ds.scratch + kCounterBytes, &tab, used, cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemsetAsync(ds.scratch, 0, sizeof(int), s) != cudaSuccess)
        return NUMA_ECUDA;
    const int g_mixed = ds.num_sms * tile_ctas_per_sm<true>();
    const int g_fp64 = ds.num_sms * tile_ctas_per_sm<false>();
    if (mixed && tracers)
        batch_lsrk_noalloc_kernel<true, true><<<g_mixed, kThreads, tile_smem_bytes<true, true>(), s>>>(
            ds.scratch, kCoef, nsteps, dt);
    else if (mixed)
        batch_lsrk_noalloc_kernel<true, false><<<g_mixed, kThreads, tile_smem_bytes<true>(), s>>>(
            ds.scratch, kCoef, nsteps, dt);
    else if (tracers)
        batch_lsrk_noalloc_kernel<false, true><<<g_fp64, kThreads, tile_smem_bytes<false, true>(),
                                                 s>>>(ds.scratch, kCoef, nsteps, dt);
    else
        batch_lsrk_noalloc_kernel<false, false><<<g_fp64, kThreads, tile_smem_bytes<false>(), s>>>(
            ds.scratch, kCoef, nsteps, dt);
    return cudaGetLastError() == cudaSuccess ? NUMA_OK : NUMA_ECUDA;
}
