// C ABI of batched time integration: many volume-term instances (handles of
// mixed order and size) advanced together by the low-storage Runge-Kutta
// scheme in one persistent, graph-captured launch.  See include/numa_vol.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "numa_internal.h"
#include "numa_vol.h"

namespace {

// The five-stage fourth-order 2N-storage coefficients of Carpenter and
// Kennedy (NASA TM-109112, 1994).
const numa::LsrkCoef kLsrk = {
    {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
     -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0},
    {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
     1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
     2277821191437.0 / 14882151754819.0}};

thread_local std::string g_batch_error;

int bfail(int code, const std::string &msg) {
    g_batch_error = msg;
    return code;
}

int bfail_cuda(cudaError_t e, const char *where) {
    // Reset the runtime's last-error state: a non-sticky error (an allocation
    // refused) is reported here, not again by the next unrelated launch check.
    cudaGetLastError();
    int code = (e == cudaErrorMemoryAllocation) ? NUMA_ENOMEM : NUMA_ECUDA;
    return bfail(code, std::string(where) + ": " + cudaGetErrorName(e) + " (" +
                           cudaGetErrorString(e) + ")");
}

// Some instance has tracers: the launch runs the tiles' tracer forms.
bool has_tracers(const std::vector<numa::BatchInstance> &v) {
    for (const auto &I : v)
        if (I.nf > numa::kFields) return true;
    return false;
}

}  // namespace

struct numa_batch {
    numa_precision prec = NUMA_FP64;
    int device = 0;
    int num_sms = 0;
    std::vector<numa::BatchInstance> inst;
    int tile_mult[9] = {4, 4, 4, 4, 4, 4, 4, 4, 4};   // elements per item / elements per pass, by Nq
    numa_sweep sweep = NUMA_SWEEP_CUDA_CORES;
    unsigned tc_mask = 0;  // orders (bit Nq) whose D sums run on the tensor cores (mixed only)
    int ctas_per_sm = 0;   // CTAs per SM of the persistent grid (0: the kernel's maximum)
    bool costliest_first = false;   // work items sorted by points, largest first
    bool tmem_state = false;        // mixed, CUDA-core tiles: the state in tensor memory
    double tuned_ms = 0.0;          // last autotune: ms per step of the chosen configuration
    int tuned_candidates = 0;       // last autotune: configurations timed
    // device scratch: instance table, work items, claim counter
    numa::BatchInstance *d_inst = nullptr;
    size_t inst_cap = 0;
    numa::BatchItem *d_items = nullptr;
    size_t items_cap = 0;
    int num_items = 0;
    int *d_counter = nullptr;
    bool dirty = true;
    // captured launch: counter reset + persistent kernel
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int g_nsteps = -1;
    double g_dt = 0.0;
    cudaEvent_t launched = nullptr;   // recorded after each launch: the tables are in use until then
};

namespace numa {

// Build the work list for `inst` with the given tiles; items of one instance
// are contiguous and instances keep their order.
std::vector<BatchItem> build_items(const std::vector<BatchInstance> &inst, const int *tile_mult,
                                   bool costliest_first) {
    std::vector<BatchItem> items;
    for (size_t k = 0; k < inst.size(); ++k) {
        const int nq = inst[k].nq;
        const int64_t ne = inst[k].M / ((int64_t)nq * nq * nq);
        const int64_t tile = (int64_t)elements_per_pass(nq) * std::max(1, tile_mult[nq]);
        for (int64_t e0 = 0; e0 < ne; e0 += tile)
            items.push_back(BatchItem{(int)k, nq, e0, std::min(tile, ne - e0)});
    }
    if (costliest_first)
        std::stable_sort(items.begin(), items.end(), [](const BatchItem &a, const BatchItem &b) {
            return a.count * a.nq * a.nq * a.nq > b.count * b.nq * b.nq * b.nq;
        });
    return items;
}

}  // namespace numa

namespace {

cudaError_t upload(numa_batch *b, const std::vector<numa::BatchInstance> &inst,
                   const std::vector<numa::BatchItem> &items, cudaStream_t s) {
    // A previous launch may still read the tables on the caller's stream.
    cudaError_t e = cudaEventSynchronize(b->launched);
    if (e != cudaSuccess) return e;
    if (inst.size() > b->inst_cap) {
        cudaFree(b->d_inst);
        b->d_inst = nullptr;
        b->inst_cap = std::max<size_t>(inst.size(), 2 * b->inst_cap);
        e = cudaMalloc(&b->d_inst, sizeof(numa::BatchInstance) * b->inst_cap);
        if (e != cudaSuccess) {
            b->inst_cap = 0;
            return e;
        }
    }
    if (items.size() > b->items_cap) {
        cudaFree(b->d_items);
        b->d_items = nullptr;
        b->items_cap = std::max<size_t>(items.size(), 2 * b->items_cap);
        e = cudaMalloc(&b->d_items, sizeof(numa::BatchItem) * b->items_cap);
        if (e != cudaSuccess) {
            b->items_cap = 0;
            return e;
        }
    }
    if (!inst.empty())
        e = cudaMemcpyAsync(b->d_inst, inst.data(), sizeof(numa::BatchInstance) * inst.size(),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !items.empty())
        e = cudaMemcpyAsync(b->d_items, items.data(), sizeof(numa::BatchItem) * items.size(),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // pageable sources
    b->num_items = (int)items.size();
    return e;
}

void drop_graph(numa_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->g_nsteps = -1;
}

int grid_of(const numa_batch *b) { return b->num_sms; }   // the launcher sizes the grid from it

}  // namespace

extern "C" {

const char *numa_batch_last_error(void) { return g_batch_error.c_str(); }

int numa_batch_create(numa_precision prec, numa_batch **out) {
    g_batch_error.clear();
    if (!out) return bfail(NUMA_EINVAL, "numa_batch_create: out is NULL");
    *out = nullptr;
    if (prec != NUMA_FP64 && prec != NUMA_MIXED)
        return bfail(NUMA_EUNSUPPORTED, "numa_batch_create: batches are NUMA_FP64 or NUMA_MIXED");
    numa_batch *b = new (std::nothrow) numa_batch();
    if (!b) return bfail(NUMA_ENOMEM, "numa_batch_create: host allocation failed");
    b->prec = prec;
    b->tmem_state = prec == NUMA_MIXED;   // the state in tensor memory: the faster tile
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e == cudaSuccess) e = numa::prepare_batch_lsrk();
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, 256);
    if (e == cudaSuccess) e = cudaMemset(b->d_counter, 0, 256);   // [0] claims, [1] status
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->launched, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(b->launched, b->cap_stream);
    if (e != cudaSuccess) {
        cudaFree(b->d_counter);
        delete b;
        return bfail_cuda(e, "numa_batch_create");
    }
    *out = b;
    return NUMA_OK;
}

int numa_batch_add(numa_batch *b, const numa_vol *h, void *q, int *index) {
    g_batch_error.clear();
    if (!b || !h || !q) return bfail(NUMA_EINVAL, "numa_batch_add: NULL argument");
    if ((reinterpret_cast<uintptr_t>(q) & 15u) != 0)
        return bfail(NUMA_EINVAL, "numa_batch_add: q must be 16-byte aligned");
    const bool mixed = b->prec == NUMA_MIXED;
    if (h->N > NUMA_MAX_N)
        return bfail(NUMA_EUNSUPPORTED, "numa_batch_add: the batch takes orders N <= 7");
    if (mixed ? h->kernel != numa::Kernel::Mixed : h->kernel != numa::Kernel::Native)
        return bfail(NUMA_EINVAL, "numa_batch_add: handle precision differs from the batch's "
                                  "(NUMA_FP64 batches take NUMA_FP64 handles)");
    if (h->device != b->device)
        return bfail(NUMA_EINVAL, "numa_batch_add: handle lives on another device");
    numa::BatchInstance I{};
    I.N = h->N;
    I.nq = h->Nq;
    I.M = h->M;
    I.q = q;
    I.geo = h->geo;
    I.np = h->nparams;
    I.mgeo = h->mgeo;
    I.mp = h->mparams;
    I.nf = h->nf;
    b->inst.push_back(I);
    b->dirty = true;
    if (index) *index = (int)b->inst.size() - 1;
    return NUMA_OK;
}

int numa_batch_clear(numa_batch *b) {
    if (!b) return bfail(NUMA_EINVAL, "numa_batch_clear: NULL batch");
    b->inst.clear();
    b->dirty = true;
    return NUMA_OK;
}

int numa_batch_size(const numa_batch *b) { return b ? (int)b->inst.size() : 0; }

int numa_batch_advance(numa_batch *b, int nsteps, double dt, void *stream) {
    g_batch_error.clear();
    if (!b) return bfail(NUMA_EINVAL, "numa_batch_advance: NULL batch");
    if (nsteps < 0) return bfail(NUMA_EINVAL, "numa_batch_advance: nsteps < 0");
    if (nsteps == 0 || b->inst.empty()) return NUMA_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (b->dirty) {
        drop_graph(b);
        e = upload(b, b->inst, numa::build_items(b->inst, b->tile_mult, b->costliest_first),
                   b->cap_stream);
        if (e != cudaSuccess) return bfail_cuda(e, "numa_batch_advance: upload of the work list");
        b->dirty = false;
    }
    if (!b->exec || b->g_nsteps != nsteps || b->g_dt != dt) {
        drop_graph(b);
        e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) e = cudaMemsetAsync(b->d_counter, 0, sizeof(int), b->cap_stream);
        if (e == cudaSuccess)
            e = numa::launch_batch_lsrk(b->prec == NUMA_MIXED, b->d_inst, b->d_items, b->num_items,
                                        b->d_counter, kLsrk, nsteps, dt, grid_of(b), b->cap_stream,
                                        b->tc_mask, b->ctas_per_sm, b->tmem_state,
                                        has_tracers(b->inst));
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &g);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
        if (e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            b->exec = nullptr;
            return bfail_cuda(e, "numa_batch_advance: graph capture");
        }
        b->graph = g;
        b->g_nsteps = nsteps;
        b->g_dt = dt;
    }
    e = cudaGraphLaunch(b->exec, s);
    if (e == cudaSuccess) e = cudaEventRecord(b->launched, s);
    if (e != cudaSuccess) return bfail_cuda(e, "numa_batch_advance: graph launch");
    return NUMA_OK;
}

namespace {

// One launch configuration of the batch.
struct TuneCfg {
    int mult[9];
    unsigned mask;
    int ctas;
    bool costliest;
    bool tmem;
};

// Best of `reps` timed launches of `nsteps` steps over instances `sub` in
// configuration c (the work list is uploaded first).
cudaError_t time_cfg(numa_batch *b, const std::vector<numa::BatchInstance> &sub, const TuneCfg &c,
                     int nsteps, int reps, cudaStream_t s, cudaEvent_t t0, cudaEvent_t t1,
                     float *ms_out) {
    cudaError_t e = upload(b, sub, numa::build_items(sub, c.mult, c.costliest), s);
    float ms = 1e30f;
    for (int rep = 0; rep < reps && e == cudaSuccess; ++rep) {
        e = cudaMemsetAsync(b->d_counter, 0, sizeof(int), s);
        if (e == cudaSuccess) e = cudaEventRecord(t0, s);
        if (e == cudaSuccess)
            e = numa::launch_batch_lsrk(b->prec == NUMA_MIXED, b->d_inst, b->d_items, b->num_items,
                                        b->d_counter, kLsrk, nsteps, 1e-6, grid_of(b), s, c.mask,
                                        c.ctas, c.tmem, has_tracers(sub));
        if (e == cudaSuccess) e = cudaEventRecord(t1, s);
        if (e == cudaSuccess) e = cudaEventRecord(b->launched, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, t0, t1);
        ms = std::min(ms, t);
    }
    ++b->tuned_candidates;
    *ms_out = ms;
    return e;
}

}  // namespace

int numa_batch_autotune(numa_batch *b, void *stream) {
    g_batch_error.clear();
    if (!b) return bfail(NUMA_EINVAL, "numa_batch_autotune: NULL batch");
    if (b->inst.empty()) return NUMA_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool mixed = b->prec == NUMA_MIXED;
    const size_t elem = mixed ? sizeof(float) : sizeof(double);
    const int mults[] = {1, 2, 4, 8, 16, 32};
    constexpr int kSteps = 2, kReps = 3;   // per timing: two steps (ten stages), best of three
    b->tuned_candidates = 0;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    cudaError_t e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    // every instance on a copy of its state
    std::vector<numa::BatchInstance> all;
    std::vector<void *> copies;
    for (const auto &I : b->inst) {
        if (e != cudaSuccess) break;
        void *c = nullptr;
        e = cudaMalloc(&c, elem * I.nf * I.M);
        if (e != cudaSuccess) break;
        copies.push_back(c);
        e = cudaMemcpyAsync(c, I.q, elem * I.nf * I.M, cudaMemcpyDeviceToDevice, s);
        numa::BatchInstance J = I;
        J.q = c;
        all.push_back(J);
    }
    TuneCfg cur{};
    std::copy(b->tile_mult, b->tile_mult + 9, cur.mult);
    cur.mask = b->tc_mask;
    cur.ctas = b->ctas_per_sm;
    cur.costliest = b->costliest_first;
    cur.tmem = b->tmem_state;
    // per-order candidates: (sweep, passes per item)
    auto order_cands = [&](int nq) {
        std::vector<std::pair<unsigned, int>> v;
        const unsigned bit = 1u << nq;
        std::vector<unsigned> masks;
        if (b->sweep == NUMA_SWEEP_AUTO) {
            masks = {0u, bit};
        } else {
            masks = {b->tc_mask & bit};
        }
        for (unsigned mk : masks)
            for (int m : mults) v.push_back({mk, m});
        return v;
    };
    // 1. each order alone: the best candidate as the starting point
    bool present[9] = {};
    for (const auto &I : all) present[I.nq] = true;
    for (int nq = 2; nq <= 8 && e == cudaSuccess; ++nq) {
        if (!present[nq]) continue;
        std::vector<numa::BatchInstance> sub;
        for (const auto &I : all)
            if (I.nq == nq) sub.push_back(I);
        float best = 1e30f;
        for (auto [mk, m] : order_cands(nq)) {
            if (e != cudaSuccess) break;
            TuneCfg c = cur;
            c.mult[nq] = m;
            c.mask = (cur.mask & ~(1u << nq)) | mk;
            float ms = 0.f;
            e = time_cfg(b, sub, c, kSteps, kReps, s, t0, t1, &ms);
            if (e == cudaSuccess && ms < best) {
                best = ms;
                cur.mult[nq] = m;
                cur.mask = c.mask;
            }
        }
    }
    // 2. the launch the batch runs (all orders together): coordinate descent
    // over each order's candidates, then CTAs per SM and the item order; a
    // change is kept when it saves at least 1 %.
    float best = 1e30f;
    if (e == cudaSuccess) e = time_cfg(b, all, cur, kSteps, kReps, s, t0, t1, &best);
    auto try_cfg = [&](const TuneCfg &c) {
        float ms = 0.f;
        if (e == cudaSuccess) e = time_cfg(b, all, c, kSteps, kReps, s, t0, t1, &ms);
        if (e == cudaSuccess && ms < 0.99f * best) {
            best = ms;
            cur = c;
        }
    };
    int present_count = 0;
    for (int nq = 2; nq <= 8; ++nq) present_count += present[nq];
    for (int nq = 2; nq <= 8 && present_count > 1; ++nq) {
        if (!present[nq]) continue;
        const TuneCfg base = cur;
        for (auto [mk, m] : order_cands(nq)) {
            TuneCfg c = base;
            c.mult[nq] = m;
            c.mask = (base.mask & ~(1u << nq)) | mk;
            if (c.mult[nq] == base.mult[nq] && c.mask == base.mask) continue;
            try_cfg(c);
        }
    }
    for (int k = 1; k <= numa::batch_max_ctas_per_sm(mixed); ++k) {
        TuneCfg c = cur;
        c.ctas = k == numa::batch_max_ctas_per_sm(mixed) ? 0 : k;
        if (c.ctas != cur.ctas) try_cfg(c);
    }
    {
        TuneCfg c = cur;
        c.costliest = !cur.costliest;
        try_cfg(c);
    }
    if (mixed) {   // the CUDA-core tiles' state in tensor memory or shared memory
        TuneCfg c = cur;
        c.tmem = !cur.tmem;
        try_cfg(c);
    }
    for (void *c : copies) cudaFree(c);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (e != cudaSuccess) return bfail_cuda(e, "numa_batch_autotune");
    std::copy(cur.mult, cur.mult + 9, b->tile_mult);
    b->tc_mask = cur.mask;
    b->ctas_per_sm = cur.ctas;
    b->costliest_first = cur.costliest;
    b->tmem_state = cur.tmem;
    b->tuned_ms = best / kSteps;
    b->dirty = true;   // the work list is rebuilt with the chosen tiles
    drop_graph(b);     // and the launch recaptured with the chosen kernel and grid
    return NUMA_OK;
}

int numa_batch_get_config(const numa_batch *b, numa_batch_config *out) {
    if (!b || !out) return bfail(NUMA_EINVAL, "numa_batch_get_config: NULL argument");
    numa_batch_config c{};
    for (int nq = 0; nq < 9; ++nq) {
        c.tile[nq] = nq >= 2 ? numa::elements_per_pass(nq) * b->tile_mult[nq] : 0;
        c.sweep[nq] = ((b->tc_mask >> nq) & 1u) ? NUMA_SWEEP_TENSOR_TF32 : NUMA_SWEEP_CUDA_CORES;
    }
    c.ctas_per_sm = b->ctas_per_sm;
    c.costliest_first = b->costliest_first ? 1 : 0;
    c.state_in_tmem = b->tmem_state ? 1 : 0;
    c.tuned_ms_per_step = b->tuned_ms;
    c.tuned_candidates = b->tuned_candidates;
    *out = c;
    return NUMA_OK;
}

int numa_batch_set_config(numa_batch *b, const numa_batch_config *c) {
    g_batch_error.clear();
    if (!b || !c) return bfail(NUMA_EINVAL, "numa_batch_set_config: NULL argument");
    const bool mixed = b->prec == NUMA_MIXED;
    if (c->ctas_per_sm < 0 || c->ctas_per_sm > numa::batch_max_ctas_per_sm(mixed))
        return bfail(NUMA_EINVAL, "numa_batch_set_config: ctas_per_sm out of range");
    unsigned mask = 0;
    int mult[9];
    for (int nq = 2; nq <= 8; ++nq) {
        const int epp = numa::elements_per_pass(nq);
        if (c->tile[nq] < epp || c->tile[nq] % epp != 0)
            return bfail(NUMA_EINVAL, "numa_batch_set_config: a tile is not a positive multiple "
                                      "of the elements per pass of its order");
        mult[nq] = c->tile[nq] / epp;
        if (c->sweep[nq] == NUMA_SWEEP_TENSOR_TF32) {
            if (!mixed)
                return bfail(NUMA_EUNSUPPORTED,
                             "numa_batch_set_config: the tensor-core sweep is for NUMA_MIXED batches");
            mask |= 1u << nq;
        } else if (c->sweep[nq] != NUMA_SWEEP_CUDA_CORES) {
            return bfail(NUMA_EINVAL, "numa_batch_set_config: a sweep is not CUDA_CORES or TENSOR_TF32");
        }
    }
    for (int nq = 2; nq <= 8; ++nq) b->tile_mult[nq] = mult[nq];
    b->tc_mask = mask;
    b->ctas_per_sm = c->ctas_per_sm;
    if (c->state_in_tmem && !mixed)
        return bfail(NUMA_EUNSUPPORTED, "numa_batch_set_config: state_in_tmem is for NUMA_MIXED batches");
    b->costliest_first = c->costliest_first != 0;
    b->tmem_state = c->state_in_tmem != 0;
    b->dirty = true;
    drop_graph(b);
    return NUMA_OK;
}

int numa_batch_set_sweep(numa_batch *b, numa_sweep sweep) {
    g_batch_error.clear();
    if (!b) return bfail(NUMA_EINVAL, "numa_batch_set_sweep: NULL batch");
    if (sweep != NUMA_SWEEP_CUDA_CORES && sweep != NUMA_SWEEP_TENSOR_TF32 &&
        sweep != NUMA_SWEEP_AUTO)
        return bfail(NUMA_EINVAL, "numa_batch_set_sweep: unknown sweep");
    if (sweep != NUMA_SWEEP_CUDA_CORES && b->prec != NUMA_MIXED)
        return bfail(NUMA_EUNSUPPORTED,
                     "numa_batch_set_sweep: the tensor-core sweep is for NUMA_MIXED batches");
    const unsigned mask = sweep == NUMA_SWEEP_TENSOR_TF32 ? numa::kTcAllOrders
                          : sweep == NUMA_SWEEP_AUTO      ? b->tc_mask
                                                          : 0u;
    b->sweep = sweep;
    if (mask != b->tc_mask) {
        b->tc_mask = mask;
        drop_graph(b);   // the next advance captures the other kernel
    }
    return NUMA_OK;
}

int numa_batch_sweep(const numa_batch *b) { return b ? (int)b->sweep : -1; }

int numa_batch_sweep_of(const numa_batch *b, int nq) {
    if (!b || nq < 2 || nq > 8) return -1;
    return ((b->tc_mask >> nq) & 1u) ? NUMA_SWEEP_TENSOR_TF32 : NUMA_SWEEP_CUDA_CORES;
}

int numa_batch_status(numa_batch *b, void *stream) {
    g_batch_error.clear();
    if (!b) return bfail(NUMA_EINVAL, "numa_batch_status: NULL batch");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int word = 0;
    cudaError_t e = cudaMemcpyAsync(&word, b->d_counter + 1, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && word != 0) e = cudaMemsetAsync(b->d_counter + 1, 0, sizeof(int), s);
    if (e == cudaSuccess && word != 0) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return bfail_cuda(e, "numa_batch_status");
    if (word & 1)
        return bfail(NUMA_ETIMEOUT, "numa_batch_status: a wait for the tensor core ran out");
    return NUMA_OK;
}

int numa_batch_tile(const numa_batch *b, int nq) {
    if (!b || nq < 2 || nq > 8) return 0;
    return numa::elements_per_pass(nq) * b->tile_mult[nq];
}

void numa_batch_destroy(numa_batch *b) {
    if (!b) return;
    cudaDeviceSynchronize();
    drop_graph(b);
    if (b->launched) cudaEventDestroy(b->launched);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    cudaFree(b->d_inst);
    cudaFree(b->d_items);
    cudaFree(b->d_counter);
    delete b;
}

}  // extern "C"
