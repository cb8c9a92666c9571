// Batched explicit time integration of dq/dt = v(q), v the element volume term
// (Sec. 2, Eq. (2)), for many independent instances of mixed order and size in
// one persistent launch.
//
// Scheme: the five-stage fourth-order 2N-storage Runge-Kutta method of
// Carpenter and Kennedy (NASA TM-109112, 1994): per stage s,
//   dq <- A_s dq + dt v(q),  q <- q + B_s dq,   dq = 0 at the start.
// The paper frames the volume term as the rate function of such an explicit
// solver (Sec. 2); the scheme is the benchmark's choice.
//
// The volume term couples only the points of one element.  So a CTA can take
// a tile of elements through all 5 * nsteps stages with q and dq of its
// points in registers: q is read from and written to HBM once, and there is
// no grid-wide synchronisation.  The tile's geometry (56 KB in FP64 for one
// Nq = 8 element) is re-read every stage; after the first stage it comes from
// L2.  Each stage
// runs the same three phases as the single-evaluation kernels: fluxes by point
// into shared memory, even-odd D sweeps by line in place, combination by point.
//
// Work items (instance, element range) are claimed dynamically through an
// atomic counter.  Orders are mixed within one launch: a CTA of 512 threads
// holds 512 / Nq^3 elements per pass.  Tile sizes (elements per item) come
// from the batch's autotuner.
#include <cuda_runtime.h>

#include <mutex>

#include "batch_tile.cuh"
#include "batch_tile_tc.cuh"

namespace numa {

namespace {

// TR: the tiles' tracer forms, for batches that hold instances with tracers.
template <bool MIXED, bool TR = false>
__global__ void __launch_bounds__(kThreads, tile_ctas_per_sm<MIXED>())
batch_lsrk_kernel(const BatchInstance *__restrict__ inst, const BatchItem *__restrict__ items,
                  int num_items, int *counter, LsrkCoef co, int nsteps, double dt) {
    extern __shared__ __align__(16) double smem_d[];
    __shared__ BatchInstance sI;
    __shared__ int s_item;
    __shared__ tile_t<MIXED> sco[10];
    load_stage_coefficients<MIXED>(co, sco);   // visible after the first barrier below
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= num_items) break;
        const BatchItem item = items[it];
        {
            // instance description into shared memory, word by word
            const int *src = reinterpret_cast<const int *>(inst + item.instance);
            int *dst = reinterpret_cast<int *>(&sI);
            for (int w = threadIdx.x; w < (int)(sizeof(BatchInstance) / sizeof(int)); w += kThreads)
                dst[w] = src[w];
        }
        __syncthreads();
        const int ns = sI.nsteps > 0 ? sI.nsteps : nsteps;
        switch (item.nq) {
            case 2: run_tile<2, MIXED, TR>(sI, item.e0, item.count, sco, ns, dt, smem_d); break;
            case 3: run_tile<3, MIXED, TR>(sI, item.e0, item.count, sco, ns, dt, smem_d); break;
            case 4: run_tile<4, MIXED, TR>(sI, item.e0, item.count, sco, ns, dt, smem_d); break;
            case 5: run_tile<5, MIXED, TR>(sI, item.e0, item.count, sco, ns, dt, smem_d); break;
            case 6: run_tile<6, MIXED, TR>(sI, item.e0, item.count, sco, ns, dt, smem_d); break;
            case 7: run_tile<7, MIXED, TR>(sI, item.e0, item.count, sco, ns, dt, smem_d); break;
            case 8: run_tile<8, MIXED, TR>(sI, item.e0, item.count, sco, ns, dt, smem_d); break;
            default: break;
        }
        __syncthreads();   // sI and s_item are rewritten by the next claim
    }
}


// Mixed precision with the D contractions on the tensor cores (batch_tile_tc.cuh)
// for the orders whose bit Nq is set in tc_mask, on the CUDA cores for the
// others (run_tile_cc_tm: run_tile's phases with the state in tensor memory):
// the autotuner picks per order.  counter[1] is the batch's
// status word: bit 0 is set when a wait for the tensor core ran out; the CTA
// then stops claiming work.
static_assert(sizeof(float) * kMixedFluxWords <= (size_t)kTcOperandBytes,
              "the CUDA-core tile's fluxes fit the tensor tile's operand region");

// Separate functions (not inlined), so that each tile is register-allocated on
// its own: inlined together they spill.
template <int NQ>
__device__ __noinline__ bool run_tile_tc_call(const BatchInstance &I, int64_t e0, int64_t count,
                                              const float *sco, int ns, double dt,
                                              unsigned char *sm, uint32_t tmem, uint64_t *bar,
                                              uint32_t &phase, int *s_nq) {
    return run_tile_tc<NQ>(I, e0, count, sco, ns, dt, sm, tmem, bar, phase, s_nq);
}
template <int NQ>
__device__ __noinline__ void run_tile_cc_call(const BatchInstance &I, int64_t e0, int64_t count,
                                              const float *sco, int ns, double dt,
                                              unsigned char *sm, uint32_t tmem) {
    run_tile_cc_tm<NQ>(I, e0, count, sco, ns, dt, sm, tmem);
}

template <int NQ>
__device__ __forceinline__ bool run_tile_either(unsigned tc_mask, const BatchInstance &I,
                                                int64_t e0, int64_t count, const float *sco,
                                                int ns, double dt, unsigned char *sm,
                                                uint32_t tmem, uint64_t *bar, uint32_t &phase,
                                                int *s_nq) {
    if ((tc_mask >> NQ) & 1u)
        return run_tile_tc_call<NQ>(I, e0, count, sco, ns, dt, sm, tmem, bar, phase, s_nq);
    run_tile_cc_call<NQ>(I, e0, count, sco, ns, dt, sm, tmem);
    __syncthreads();
    if (threadIdx.x == 0) *s_nq = 0;   // the operands were overwritten
    return true;
}

__global__ void __launch_bounds__(kThreads, 2)
batch_lsrk_tc_kernel(const BatchInstance *__restrict__ inst, const BatchItem *__restrict__ items,
                     int num_items, int *counter, LsrkCoef co, int nsteps, double dt,
                     unsigned tc_mask) {
    extern __shared__ __align__(1024) unsigned char smem_tc[];
    __shared__ BatchInstance sI;
    __shared__ int s_item, s_nq;
    __shared__ float sco[10];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t s_tmem;
    load_stage_coefficients<true>(co, sco);
    if (threadIdx.x < 32) tc::tmem_alloc(&s_tmem, kTcCols);
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        s_nq = 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = s_tmem;
    uint32_t phase = 0;
    bool ok = true;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= num_items) break;
        const BatchItem item = items[it];
        {
            const int *src = reinterpret_cast<const int *>(inst + item.instance);
            int *dst = reinterpret_cast<int *>(&sI);
            for (int w = threadIdx.x; w < (int)(sizeof(BatchInstance) / sizeof(int)); w += kThreads)
                dst[w] = src[w];
        }
        __syncthreads();
        const int ns = sI.nsteps > 0 ? sI.nsteps : nsteps;
        switch (item.nq) {
            case 2: ok = run_tile_either<2>(tc_mask, sI, item.e0, item.count, sco, ns, dt, smem_tc, tmem, &bar, phase, &s_nq); break;
            case 3: ok = run_tile_either<3>(tc_mask, sI, item.e0, item.count, sco, ns, dt, smem_tc, tmem, &bar, phase, &s_nq); break;
            case 4: ok = run_tile_either<4>(tc_mask, sI, item.e0, item.count, sco, ns, dt, smem_tc, tmem, &bar, phase, &s_nq); break;
            case 5: ok = run_tile_either<5>(tc_mask, sI, item.e0, item.count, sco, ns, dt, smem_tc, tmem, &bar, phase, &s_nq); break;
            case 6: ok = run_tile_either<6>(tc_mask, sI, item.e0, item.count, sco, ns, dt, smem_tc, tmem, &bar, phase, &s_nq); break;
            case 7: ok = run_tile_either<7>(tc_mask, sI, item.e0, item.count, sco, ns, dt, smem_tc, tmem, &bar, phase, &s_nq); break;
            case 8: ok = run_tile_either<8>(tc_mask, sI, item.e0, item.count, sco, ns, dt, smem_tc, tmem, &bar, phase, &s_nq); break;
            default: break;
        }
        __syncthreads();   // sI and s_item are rewritten by the next claim
        if (!ok) break;    // uniform: run_tile_tc decides it with a barrier
    }
    if (!ok) {
        if (threadIdx.x == 0) atomicOr(counter + 1, 1);
        bulk_wait(&bar, phase);   // the MMAs in flight, bounded again
    }
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, kTcCols);
    }
}

}  // namespace

cudaError_t prepare_batch_lsrk() {
    // once per device: the sweep tables into this unit's constant memory
    static std::mutex mu;
    static bool uploaded[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!uploaded[dev]) {
            e = upload_sweep_tables();
            if (e == cudaSuccess) e = upload_tc_tables();
            if (e != cudaSuccess) return e;
            uploaded[dev] = true;
        }
    }
    e = cudaFuncSetAttribute(batch_lsrk_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tile_smem_bytes<false>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(batch_lsrk_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tile_smem_bytes<true>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(batch_lsrk_kernel<false, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tile_smem_bytes<false, true>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(batch_lsrk_kernel<true, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tile_smem_bytes<true, true>());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(batch_lsrk_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kTcSmemBytes);
}

int batch_max_ctas_per_sm(bool mixed) { return mixed ? 2 : tile_ctas_per_sm<false>(); }

cudaError_t launch_batch_lsrk(bool mixed, const BatchInstance *inst, const BatchItem *items,
                              int num_items, int *counter, const LsrkCoef &co, int nsteps,
                              double dt, int num_sms, cudaStream_t s, unsigned tc_mask,
                              int ctas_per_sm, bool tmem_state, bool tracers) {
    if (num_items <= 0 || nsteps <= 0) return cudaSuccess;
    const int kmax = batch_max_ctas_per_sm(mixed);
    const int k = ctas_per_sm > 0 && ctas_per_sm < kmax ? ctas_per_sm : kmax;
    if (tracers && mixed)   // the shared-memory-state tile's tracer form
        batch_lsrk_kernel<true, true><<<num_sms * k, kThreads, tile_smem_bytes<true, true>(), s>>>(
            inst, items, num_items, counter, co, nsteps, dt);
    else if (tracers)
        batch_lsrk_kernel<false, true><<<num_sms * k, kThreads, tile_smem_bytes<false, true>(), s>>>(
            inst, items, num_items, counter, co, nsteps, dt);
    else if (mixed && (tc_mask != 0 || tmem_state))
        batch_lsrk_tc_kernel<<<num_sms * k, kThreads, kTcSmemBytes, s>>>(
            inst, items, num_items, counter, co, nsteps, dt, tc_mask);
    else if (mixed)
        batch_lsrk_kernel<true><<<num_sms * k, kThreads, tile_smem_bytes<true>(), s>>>(
            inst, items, num_items, counter, co, nsteps, dt);
    else
        batch_lsrk_kernel<false><<<num_sms * k, kThreads, tile_smem_bytes<false>(), s>>>(
            inst, items, num_items, counter, co, nsteps, dt);
    return cudaGetLastError();
}

}  // namespace numa
