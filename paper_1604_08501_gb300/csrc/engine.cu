// Serving engine: continuous batching of ensemble-member requests over the
// batched low-storage Runge-Kutta integrator.  See include/numa_vol.h.
//
// A request names a resident mesh (a numa_vol handle the caller created), an
// initial state and a number of RK steps.  The engine keeps members' states
// in an arena it reserves once (the HBM budget), and the work tables of its
// launches in buffers reserved at create time, so no round allocates memory.
// Each call of numa_engine_progress is one round, enqueued without waiting for
// the GPU:
//   1. report members whose final state has reached host memory and free
//      their arena blocks;
//   2. retire cancelled members (their blocks are freed once the last launch
//      that used them has finished);
//   3. admit queued requests in arrival order while a member slot is free and
//      the arena has room (first fit); the head of the queue waits if it does
//      not fit yet, so later requests cannot starve it.  Their states upload
//      on a copy stream; the round's launch waits for them on the device;
//   4. advance every resident member by s steps, all in one persistent launch
//      (members of different dt in one launch each) on the compute stream:
//      s = 1 by default, or up to a set limit but never past the next member's
//      completion; or, under the per-member policy, each member by its own
//      min(limit, remaining);
//   5. members that finish with this round copy their states out on a second
//      copy stream once its launch has run; they are reported (step 1) by
//      this or a later call, when the copy has completed.
// So the uploads of newly admitted members and the downloads of finished ones
// overlap the launches, and requests that arrive while a round runs join the
// next round, whose launch is queued behind it: the continuous batching.  At
// most two launches are in flight (their work tables are double-buffered);
// a call waits only for a free table buffer, for the last launch of a
// cancelled member, or, when it has nothing to enqueue, for the oldest copy
// still in flight.  Elements evolve independently in the volume term, so a
// member's result is bitwise the same whichever members share its rounds.
//
// Checkpoint and resume: a step of the 2N-storage scheme starts from the state
// alone (its register restarts at zero), so the state after a member's last
// completed step and the number of steps done are a complete checkpoint;
// submitting the state with the remaining steps resumes it, bit for bit.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "numa_internal.h"
#include "numa_vol.h"

namespace {

thread_local std::string g_engine_error;

int efail(int code, const std::string &msg) {
    g_engine_error = msg;
    return code;
}

int efail_cuda(cudaError_t e, const char *where) {
    // Reset the runtime's last-error state: a non-sticky error (an allocation
    // refused) is reported here, not again by the next unrelated launch check.
    cudaGetLastError();
    int code = (e == cudaErrorMemoryAllocation) ? NUMA_ENOMEM : NUMA_ECUDA;
    return efail(code, std::string(where) + ": " + cudaGetErrorName(e) + " (" +
                           cudaGetErrorString(e) + ")");
}

const numa::LsrkCoef kCoef = {
    {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
     -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0},
    {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
     1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
     2277821191437.0 / 14882151754819.0}};

constexpr size_t kAlign = 256;

// First-fit allocator over the arena, with coalescing of free neighbours.
struct Arena {
    char *base = nullptr;
    size_t size = 0;
    std::map<size_t, size_t> free_blocks;   // offset -> length
    size_t used = 0;

    void reset(char *b, size_t n) {
        base = b;
        size = n;
        free_blocks.clear();
        if (n) free_blocks[0] = n;
        used = 0;
    }
    // Returns an offset, or SIZE_MAX when no free block is large enough.
    size_t alloc(size_t n) {
        n = (n + kAlign - 1) / kAlign * kAlign;
        for (auto it = free_blocks.begin(); it != free_blocks.end(); ++it) {
            if (it->second < n) continue;
            const size_t off = it->first, len = it->second;
            free_blocks.erase(it);
            if (len > n) free_blocks[off + n] = len - n;
            used += n;
            return off;
        }
        return SIZE_MAX;
    }
    void release(size_t off, size_t n) {
        n = (n + kAlign - 1) / kAlign * kAlign;
        used -= n;
        auto it = free_blocks.emplace(off, n).first;
        auto next = std::next(it);
        if (next != free_blocks.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_blocks.erase(next);
        }
        if (it != free_blocks.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_blocks.erase(it);
            }
        }
    }
};

struct Request {
    int64_t id;
    const numa_vol *mesh;
    const void *q0;
    void *q_out;
    int nsteps, remaining;
    double dt;
    size_t bytes, off;
    int status;
};

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace

namespace {

// Work tables of one launch: device copies and their pinned host staging.
// `done` is recorded after the launch; the buffers are reused once it has
// completed.
struct LaunchSlot {
    numa::BatchInstance *d_inst = nullptr, *h_inst = nullptr;
    numa::BatchItem *d_items = nullptr, *h_items = nullptr;
    int *d_counter = nullptr;
    cudaEvent_t done = nullptr;
    bool used = false;
};

// A finished member whose state is being copied to its host buffer.
struct PendingResult {
    Request r;
    cudaEvent_t copied;
};

}  // namespace

struct numa_engine {
    numa_precision prec = NUMA_FP64;
    int device = 0, num_sms = 0, max_members = 0;
    size_t elem = 8;
    Arena arena;
    void *d_arena = nullptr;
    static constexpr int kSlots = 2;
    LaunchSlot slot[kSlots];
    int next_slot = 0;
    size_t items_cap = 0;
    cudaStream_t stream = nullptr;            // launches
    cudaStream_t h2d = nullptr, d2h = nullptr;   // admissions, results
    cudaEvent_t admitted = nullptr;           // after this call's admission uploads
    cudaEvent_t last_launch = nullptr;        // after the most recent launch
    bool launched_any = false;
    std::vector<PendingResult> pending;
    std::vector<cudaEvent_t> free_events;     // for PendingResult::copied
    int64_t next_id = 1;
    std::deque<Request> queue;
    std::vector<Request> resident;
    std::map<int64_t, numa_request_info> info;
    std::deque<int64_t> finished;          // ids of done or cancelled requests, oldest first
    size_t keep_finished = size_t(1) << 20;  // records of finished requests kept for query
    int64_t completed = 0, rounds = 0;
    double point_stages = 0.0;
    int tile_mult = 4;
    int max_round_steps = 1;   // steps per round: up to this, and never past a completion
    int round_policy = NUMA_ROUND_LOCKSTEP;
};

namespace {

size_t state_bytes(const numa_engine *e, const numa_vol *h) {
    return e->elem * (size_t)h->nf * (size_t)h->M;
}

void set_status(numa_engine *e, int64_t id, int status, bool stamp_done = false) {
    auto &inf = e->info[id];
    inf.status = status;
    if (stamp_done) inf.done_s = now_s();
    if (status == NUMA_REQ_DONE || status == NUMA_REQ_CANCELLED) {
        // a long-running engine keeps the records of its most recent finished
        // requests only
        e->finished.push_back(id);
        while (e->finished.size() > e->keep_finished) {
            e->info.erase(e->finished.front());
            e->finished.pop_front();
        }
    }
}

}  // namespace

extern "C" {

const char *numa_engine_last_error(void) { return g_engine_error.c_str(); }

int numa_engine_create(numa_precision prec, size_t budget_bytes, int max_members,
                       numa_engine **out) {
    g_engine_error.clear();
    if (!out) return efail(NUMA_EINVAL, "numa_engine_create: out is NULL");
    *out = nullptr;
    if (prec != NUMA_FP64 && prec != NUMA_MIXED)
        return efail(NUMA_EUNSUPPORTED, "numa_engine_create: NUMA_FP64 or NUMA_MIXED only");
    if (max_members < 1 || budget_bytes < kAlign)
        return efail(NUMA_EINVAL, "numa_engine_create: need max_members >= 1 and a budget");
    numa_engine *e = new (std::nothrow) numa_engine();
    if (!e) return efail(NUMA_ENOMEM, "numa_engine_create: host allocation failed");
    e->prec = prec;
    e->elem = prec == NUMA_MIXED ? sizeof(float) : sizeof(double);
    e->max_members = max_members;
    // The most work items one launch can have: every point the budget holds,
    // in items of the fewest points (tile_mult passes of one element at
    // Nq = 7: 4 x 343 points), plus one partial item per member.
    {
        size_t min_item_points = SIZE_MAX;
        for (int nq = 2; nq <= 8; ++nq)
            min_item_points = std::min(min_item_points, (size_t)numa::elements_per_pass(nq) *
                                                            e->tile_mult * nq * nq * nq);
        e->items_cap = budget_bytes / (e->elem * numa::kFields) / min_item_points +
                       (size_t)max_members + 1;
    }
    cudaError_t err = cudaGetDevice(&e->device);
    if (err == cudaSuccess)
        err = cudaDeviceGetAttribute(&e->num_sms, cudaDevAttrMultiProcessorCount, e->device);
    if (err == cudaSuccess) err = numa::prepare_batch_lsrk();
    if (err == cudaSuccess) err = cudaMalloc(&e->d_arena, budget_bytes);
    for (auto &sl : e->slot) {
        if (err == cudaSuccess)
            err = cudaMalloc(&sl.d_inst, sizeof(numa::BatchInstance) * max_members);
        if (err == cudaSuccess)
            err = cudaMallocHost(&sl.h_inst, sizeof(numa::BatchInstance) * max_members);
        if (err == cudaSuccess) err = cudaMalloc(&sl.d_items, sizeof(numa::BatchItem) * e->items_cap);
        if (err == cudaSuccess)
            err = cudaMallocHost(&sl.h_items, sizeof(numa::BatchItem) * e->items_cap);
        if (err == cudaSuccess) err = cudaMalloc(&sl.d_counter, 256);
        if (err == cudaSuccess) err = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    }
    if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&e->h2d, cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&e->d2h, cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&e->admitted, cudaEventDisableTiming);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&e->last_launch, cudaEventDisableTiming);
    for (int k = 0; k < max_members && err == cudaSuccess; ++k) {
        cudaEvent_t ev = nullptr;
        err = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (err == cudaSuccess) e->free_events.push_back(ev);
    }
    if (err != cudaSuccess) {
        numa_engine_destroy(e);
        cudaGetLastError();
        return efail_cuda(err, "numa_engine_create: reserving device memory");
    }
    e->arena.reset(static_cast<char *>(e->d_arena), budget_bytes);
    *out = e;
    return NUMA_OK;
}

int numa_engine_submit(numa_engine *e, const numa_vol *mesh, const void *q0_host, void *q_out_host,
                       int nsteps, double dt, int64_t *id) {
    g_engine_error.clear();
    if (id) *id = 0;
    if (!e) return efail(NUMA_EINVAL, "numa_engine_submit: NULL engine");
    if (!mesh || !q0_host || !q_out_host)
        return efail(NUMA_EINVAL, "numa_engine_submit: NULL mesh or buffer");
    if (nsteps < 1 || !(dt > 0.0))
        return efail(NUMA_EINVAL, "numa_engine_submit: need nsteps >= 1 and dt > 0");
    const bool mixed = e->prec == NUMA_MIXED;
    if (mesh->N > NUMA_MAX_N)
        return efail(NUMA_EUNSUPPORTED, "numa_engine_submit: the engine takes orders N <= 7");
    if (mixed ? mesh->kernel != numa::Kernel::Mixed : mesh->kernel != numa::Kernel::Native)
        return efail(NUMA_EINVAL, "numa_engine_submit: mesh handle precision differs from the engine's");
    if (mesh->device != e->device)
        return efail(NUMA_EINVAL, "numa_engine_submit: mesh handle lives on another device");
    const size_t bytes = state_bytes(e, mesh);
    if (bytes > e->arena.size)
        return efail(NUMA_ELIMIT, "numa_engine_submit: the member's state exceeds the whole HBM budget");
    Request r{e->next_id++, mesh, q0_host, q_out_host, nsteps, nsteps, dt, bytes, SIZE_MAX,
              NUMA_REQ_QUEUED};
    numa_request_info inf{};
    inf.id = r.id;
    inf.status = NUMA_REQ_QUEUED;
    inf.submit_s = now_s();
    e->info[r.id] = inf;
    e->queue.push_back(r);
    if (id) *id = r.id;
    return NUMA_OK;
}

int numa_engine_cancel(numa_engine *e, int64_t id) {
    if (!e) return efail(NUMA_EINVAL, "numa_engine_cancel: NULL engine");
    for (auto it = e->queue.begin(); it != e->queue.end(); ++it)
        if (it->id == id) {
            e->queue.erase(it);
            set_status(e, id, NUMA_REQ_CANCELLED, true);
            return NUMA_OK;
        }
    for (auto &r : e->resident)
        if (r.id == id) {
            r.status = NUMA_REQ_CANCELLED;   // retired at the start of the next round
            return NUMA_OK;
        }
    // (a member whose result is being copied out has finished: not cancellable)
    return efail(NUMA_EINVAL, "numa_engine_cancel: no queued or running request with this id");
}

namespace {

// Step 1 of a round: members whose result copy has completed (all of them
// with wait_all; with wait_oldest the oldest one is waited for first).
cudaError_t collect_results(numa_engine *e, bool wait_all, bool wait_oldest,
                            std::vector<int64_t> *done) {
    cudaError_t err = cudaSuccess;
    if (wait_oldest && !e->pending.empty()) err = cudaEventSynchronize(e->pending.front().copied);
    if (err != cudaSuccess) return err;
    for (size_t k = 0; k < e->pending.size();) {
        PendingResult &p = e->pending[k];
        cudaError_t q = wait_all ? cudaEventSynchronize(p.copied) : cudaEventQuery(p.copied);
        if (q == cudaErrorNotReady) {
            ++k;
            continue;
        }
        if (q != cudaSuccess) return q;
        e->arena.release(p.r.off, p.r.bytes);
        set_status(e, p.r.id, NUMA_REQ_DONE, true);
        ++e->completed;
        done->push_back(p.r.id);
        e->free_events.push_back(p.copied);
        e->pending.erase(e->pending.begin() + k);
    }
    return cudaSuccess;
}

int report(const std::vector<int64_t> &done, int64_t *done_ids, int max_done, int *num_done) {
    int n = 0;
    for (int64_t id : done) {
        if (done_ids && n < max_done) done_ids[n] = id;
        ++n;
    }
    if (num_done) *num_done = std::min(n, std::max(max_done, 0));
    return NUMA_OK;
}

}  // namespace

int numa_engine_progress(numa_engine *e, int64_t *done_ids, int max_done, int *num_done) {
    g_engine_error.clear();
    if (num_done) *num_done = 0;
    if (!e) return efail(NUMA_EINVAL, "numa_engine_progress: NULL engine");
    std::vector<int64_t> done;
    // 1. results that have reached host memory
    cudaError_t err = collect_results(e, false, false, &done);
    if (err != cudaSuccess) return efail_cuda(err, "numa_engine_progress: result copy");
    // 2. retire cancelled members, once the last launch that used them is over
    bool cancelled = false;
    for (const auto &r : e->resident) cancelled = cancelled || r.status == NUMA_REQ_CANCELLED;
    if (cancelled && e->launched_any) {
        err = cudaEventSynchronize(e->last_launch);
        if (err != cudaSuccess) return efail_cuda(err, "numa_engine_progress: retiring");
    }
    for (size_t k = 0; k < e->resident.size();) {
        Request &r = e->resident[k];
        if (r.status == NUMA_REQ_CANCELLED) {
            e->arena.release(r.off, r.bytes);
            set_status(e, r.id, NUMA_REQ_CANCELLED, true);
            e->resident.erase(e->resident.begin() + k);
        } else {
            ++k;
        }
    }
    // 3. admit in arrival order; members whose results are still being copied
    //    out hold their slots and blocks
    bool admitted = false;
    while (!e->queue.empty() &&
           (int)(e->resident.size() + e->pending.size()) < e->max_members) {
        Request r = e->queue.front();
        const size_t off = e->arena.alloc(r.bytes);
        if (off == SIZE_MAX) break;   // the head waits for room
        e->queue.pop_front();
        r.off = off;
        r.status = NUMA_REQ_RUNNING;
        err = cudaMemcpyAsync(e->arena.base + off, r.q0, r.bytes, cudaMemcpyHostToDevice, e->h2d);
        if (err != cudaSuccess) return efail_cuda(err, "numa_engine_progress: state upload");
        e->info[r.id].status = NUMA_REQ_RUNNING;
        e->info[r.id].admit_s = now_s();
        e->resident.push_back(r);
        admitted = true;
    }
    if (admitted) {
        err = cudaEventRecord(e->admitted, e->h2d);
        if (err == cudaSuccess) err = cudaStreamWaitEvent(e->stream, e->admitted, 0);
        if (err != cudaSuccess) return efail_cuda(err, "numa_engine_progress: state upload");
    }
    if (e->resident.empty()) {
        // nothing to launch: wait for the oldest result still in flight
        // rather than return at once to a caller that polls
        if (done.empty() && !e->pending.empty()) {
            err = collect_results(e, false, true, &done);
            if (err != cudaSuccess) return efail_cuda(err, "numa_engine_progress: result copy");
        }
        return report(done, done_ids, max_done, num_done);
    }
    // 4. advance the residents, one launch per distinct dt.  Lockstep: every
    //    member by s, the smallest remaining step count up to max_round_steps,
    //    so every member that finishes does so in the round it would with
    //    single steps.  Per member: each by min(max_round_steps, remaining).
    int steps = e->max_round_steps;
    for (const auto &r : e->resident) steps = std::min(steps, r.remaining);
    const bool per_member = e->round_policy == NUMA_ROUND_PER_MEMBER;
    auto steps_of = [&](const Request &r) {
        return per_member ? std::min(e->max_round_steps, r.remaining) : steps;
    };
    std::vector<double> dts;
    for (const auto &r : e->resident)
        if (std::find(dts.begin(), dts.end(), r.dt) == dts.end()) dts.push_back(r.dt);
    for (double dt : dts) {
        std::vector<numa::BatchInstance> inst;
        int launch_steps = 1;
        bool tracers = false;   // some member has tracers: the tiles' tracer forms
        for (const auto &r : e->resident) {
            if (r.dt != dt) continue;
            numa::BatchInstance I{};
            I.N = r.mesh->N;
            I.nq = r.mesh->Nq;
            I.nf = r.mesh->nf;
            tracers = tracers || r.mesh->nf > numa::kFields;
            I.M = r.mesh->M;
            I.q = e->arena.base + r.off;
            I.geo = r.mesh->geo;
            I.np = r.mesh->nparams;
            I.mgeo = r.mesh->mgeo;
            I.mp = r.mesh->mparams;
            I.nsteps = steps_of(r);
            launch_steps = std::max(launch_steps, I.nsteps);
            inst.push_back(I);
            e->point_stages += 5.0 * I.nsteps * (double)r.mesh->M;
        }
        int mult[9];
        std::fill(mult, mult + 9, e->tile_mult);
        std::vector<numa::BatchItem> items = numa::build_items(inst, mult);
        if (per_member) {
            // costliest items first (points x steps), so that the long ones
            // do not start last and set the launch's tail
            auto cost = [&](const numa::BatchItem &it) {
                return (double)it.count * it.nq * it.nq * it.nq * inst[it.instance].nsteps;
            };
            std::stable_sort(items.begin(), items.end(),
                             [&](const numa::BatchItem &a, const numa::BatchItem &b) {
                                 return cost(a) > cost(b);
                             });
        }
        if (items.size() > e->items_cap || inst.size() > (size_t)e->max_members)
            return efail(NUMA_ECUDA, "numa_engine_progress: work list beyond the reserved tables");
        // the table buffers of the launch two back are free once it has run
        LaunchSlot &sl = e->slot[e->next_slot];
        e->next_slot = (e->next_slot + 1) % numa_engine::kSlots;
        if (sl.used) {
            err = cudaEventSynchronize(sl.done);
            if (err != cudaSuccess) return efail_cuda(err, "numa_engine_progress: step");
        }
        std::memcpy(sl.h_inst, inst.data(), sizeof(numa::BatchInstance) * inst.size());
        std::memcpy(sl.h_items, items.data(), sizeof(numa::BatchItem) * items.size());
        err = cudaMemcpyAsync(sl.d_inst, sl.h_inst, sizeof(numa::BatchInstance) * inst.size(),
                              cudaMemcpyHostToDevice, e->stream);
        if (err == cudaSuccess)
            err = cudaMemcpyAsync(sl.d_items, sl.h_items, sizeof(numa::BatchItem) * items.size(),
                                  cudaMemcpyHostToDevice, e->stream);
        if (err == cudaSuccess) err = cudaMemsetAsync(sl.d_counter, 0, sizeof(int), e->stream);
        if (err == cudaSuccess)
            err = numa::launch_batch_lsrk(e->prec == NUMA_MIXED, sl.d_inst, sl.d_items,
                                          (int)items.size(), sl.d_counter, kCoef, launch_steps,
                                          dt, e->num_sms, e->stream, 0u, 0,
                                          e->prec == NUMA_MIXED, tracers);
        if (err == cudaSuccess) err = cudaEventRecord(sl.done, e->stream);
        if (err == cudaSuccess) err = cudaEventRecord(e->last_launch, e->stream);
        if (err != cudaSuccess) return efail_cuda(err, "numa_engine_progress: step");
        sl.used = true;
        e->launched_any = true;
    }
    ++e->rounds;
    // 5. members that finish with this round: their states go to their host
    //    buffers on the result stream once the round has run
    bool any_done = false;
    for (size_t k = 0; k < e->resident.size();) {
        Request &r = e->resident[k];
        r.remaining -= steps_of(r);
        if (r.remaining == 0) {
            if (!any_done) {
                err = cudaStreamWaitEvent(e->d2h, e->last_launch, 0);
                if (err != cudaSuccess) return efail_cuda(err, "numa_engine_progress: result copy");
                any_done = true;
            }
            if (e->free_events.empty())
                return efail(NUMA_ECUDA, "numa_engine_progress: no event left for a result copy");
            PendingResult p{r, e->free_events.back()};
            e->free_events.pop_back();
            err = cudaMemcpyAsync(r.q_out, e->arena.base + r.off, r.bytes, cudaMemcpyDeviceToHost,
                                  e->d2h);
            if (err == cudaSuccess) err = cudaEventRecord(p.copied, e->d2h);
            if (err != cudaSuccess) return efail_cuda(err, "numa_engine_progress: result copy");
            e->pending.push_back(p);
            e->resident.erase(e->resident.begin() + k);
        } else {
            ++k;
        }
    }
    err = collect_results(e, false, false, &done);
    if (err != cudaSuccess) return efail_cuda(err, "numa_engine_progress: result copy");
    return report(done, done_ids, max_done, num_done);
}

int numa_engine_drain(numa_engine *e, int64_t *done_ids, int max_done, int *num_done) {
    g_engine_error.clear();
    if (num_done) *num_done = 0;
    if (!e) return efail(NUMA_EINVAL, "numa_engine_drain: NULL engine");
    cudaError_t err = cudaStreamSynchronize(e->stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(e->h2d);
    if (err == cudaSuccess) err = cudaStreamSynchronize(e->d2h);
    std::vector<int64_t> done;
    if (err == cudaSuccess) err = collect_results(e, true, false, &done);
    if (err != cudaSuccess) return efail_cuda(err, "numa_engine_drain");
    return report(done, done_ids, max_done, num_done);
}

int numa_engine_set_round_steps(numa_engine *e, int max_steps) {
    if (!e || max_steps < 1) return efail(NUMA_EINVAL, "numa_engine_set_round_steps: need max_steps >= 1");
    e->max_round_steps = max_steps;
    return NUMA_OK;
}

int numa_engine_set_round_policy(numa_engine *e, int policy) {
    if (!e || (policy != NUMA_ROUND_LOCKSTEP && policy != NUMA_ROUND_PER_MEMBER))
        return efail(NUMA_EINVAL, "numa_engine_set_round_policy: NULL engine or unknown policy");
    e->round_policy = policy;
    return NUMA_OK;
}

int numa_engine_checkpoint(numa_engine *e, int64_t id, void *state_host, int *steps_done) {
    g_engine_error.clear();
    if (steps_done) *steps_done = 0;
    if (!e || !state_host) return efail(NUMA_EINVAL, "numa_engine_checkpoint: NULL argument");
    for (const auto &r : e->queue)
        if (r.id == id) {   // not admitted yet: its state is the initial state
            std::memcpy(state_host, r.q0, r.bytes);
            return NUMA_OK;
        }
    for (const auto &r : e->resident)
        if (r.id == id && r.status == NUMA_REQ_RUNNING) {
            // after the launches already enqueued, the arena holds the state
            // after the member's last enqueued step
            cudaError_t err = cudaStreamSynchronize(e->stream);
            if (err == cudaSuccess)
                err = cudaMemcpyAsync(state_host, e->arena.base + r.off, r.bytes,
                                      cudaMemcpyDeviceToHost, e->stream);
            if (err == cudaSuccess) err = cudaStreamSynchronize(e->stream);
            if (err != cudaSuccess) return efail_cuda(err, "numa_engine_checkpoint");
            if (steps_done) *steps_done = r.nsteps - r.remaining;
            return NUMA_OK;
        }
    for (const auto &p : e->pending)
        if (p.r.id == id) {   // finished, its result still being copied out
            cudaError_t err = cudaEventSynchronize(p.copied);
            if (err == cudaSuccess) std::memcpy(state_host, p.r.q_out, p.r.bytes);
            if (err != cudaSuccess) return efail_cuda(err, "numa_engine_checkpoint");
            if (steps_done) *steps_done = p.r.nsteps;
            return NUMA_OK;
        }
    return efail(NUMA_EINVAL, "numa_engine_checkpoint: no queued or running request with this id");
}

int numa_engine_query(const numa_engine *e, int64_t id, numa_request_info *out) {
    if (!e || !out) return efail(NUMA_EINVAL, "numa_engine_query: NULL argument");
    auto it = e->info.find(id);
    if (it == e->info.end()) return efail(NUMA_EINVAL, "numa_engine_query: unknown request id");
    *out = it->second;
    return NUMA_OK;
}

int numa_engine_stats(const numa_engine *e, numa_engine_counters *out) {
    if (!e || !out) return efail(NUMA_EINVAL, "numa_engine_stats: NULL argument");
    out->queued = (int)e->queue.size();
    out->resident = (int)(e->resident.size() + e->pending.size());
    out->bytes_used = e->arena.used;
    out->bytes_budget = e->arena.size;
    out->completed = e->completed;
    out->rounds = e->rounds;
    out->point_stages = e->point_stages;
    return NUMA_OK;
}

void numa_engine_destroy(numa_engine *e) {
    if (!e) return;
    for (cudaStream_t st : {e->stream, e->h2d, e->d2h})
        if (st) {
            cudaStreamSynchronize(st);
            cudaStreamDestroy(st);
        }
    for (auto &sl : e->slot) {
        cudaFree(sl.d_inst);
        cudaFreeHost(sl.h_inst);
        cudaFree(sl.d_items);
        cudaFreeHost(sl.h_items);
        cudaFree(sl.d_counter);
        if (sl.done) cudaEventDestroy(sl.done);
    }
    for (auto &p : e->pending) e->free_events.push_back(p.copied);
    for (cudaEvent_t ev : e->free_events) cudaEventDestroy(ev);
    if (e->admitted) cudaEventDestroy(e->admitted);
    if (e->last_launch) cudaEventDestroy(e->last_launch);
    cudaFree(e->d_arena);
    delete e;
}

}  // extern "C"
