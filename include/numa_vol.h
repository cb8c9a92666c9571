/*
 * numa_vol.h - C ABI of the GB300 (sm_103a) element volume term of a
 * NUMA-style dry compressible Euler model on hexahedral GLL spectral
 * elements (Kloeckner, Wilcox, Warburton, "Array Program Transformation with
 * Loo.py by Example: High-Order Finite Elements", ARRAY'16).
 *
 * The operation (Sec. 2, Eq. (2), with the sign of the paper's r- and s-flux
 * subroutines in Sec. 3, which subtract Jinv * D * flux from rhsq).  For
 * every element e, point (i, j, k) and field b of q = (rho, U1, U2, U3, Theta):
 *
 *   rhs_b(e,i,j,k) = -Jinv(e,i,j,k) * [ sum_n D[i][n] F_r[b](e,n,j,k)
 *                                     + sum_n D[j][n] F_s[b](e,i,n,k)
 *                                     + sum_n D[k][n] F_t[b](e,i,j,n) ]
 *                    - delta_{b,U3} * (rho - rho_ref) * grav
 *
 * where, for reference direction d in {r, s, t} (Sec. 2, Eq. (1), flux column
 * f_a, contracted with the metric terms as in the paper's subroutines):
 *
 *   u_d      = (g_{1d} U1 + g_{2d} U2 + g_{3d} U3) / rho
 *   F_d[rho] = rho u_d,  F_d[U_a] = U_a u_d + g_{ad} p',  F_d[Theta] = Theta u_d
 *   p'       = p(Theta) - p(Theta_ref),  p(Theta) = p0 (R Theta / p0)^gamma,
 *   gamma    = cp / (cp - R)            (equation of state, Sec. 2)
 *
 * and D is the (N+1) x (N+1) GLL differentiation matrix, D[i][n] = l_n'(xi_i).
 * The reference-state pressure subtraction and the gravity source extend the
 * paper's gravity-free form. Theta_ref = rho_ref = grav = 0 gives the
 * paper's form exactly.
 *
 * Layout (all per-point arrays): element-major, then k, j, i with i fastest,
 * i.e. index ((e*Nq + k)*Nq + j)*Nq + i with Nq = N + 1.  M = Ne * Nq^3.
 * State and rhs: five planes of M values each, contiguous, in the order
 * (rho, U1, U2, U3, Theta), then one plane per tracer (meshes with
 * num_tracers > 0; the tracers follow Theta: flux Q u_d, no source, the
 * paper's 8-field form of Eq. (1)); plane b starts at element offset b*M.
 *
 * Errors: every int-returning call returns NUMA_OK (0) or a negative code;
 * numa_vol_last_error() then returns a message for the calling thread.  No
 * call aborts the process, and invalid arguments are rejected on the host
 * before anything is launched.
 *
 * Threading: a handle must not be used from two threads at once.  Distinct
 * handles are independent.
 */
#ifndef NUMA_VOL_H
#define NUMA_VOL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NUMA_OK 0
#define NUMA_EINVAL (-1)        /* null pointer, N out of range, bad size or misalignment */
#define NUMA_ENOMEM (-2)        /* device allocation failed                               */
#define NUMA_ECUDA (-3)         /* a CUDA call or kernel launch failed                    */
#define NUMA_EUNSUPPORTED (-4)  /* a valid request the library does not implement          */
#define NUMA_ETIMEOUT (-5)      /* a kernel's bounded device-side wait ran out              */
#define NUMA_ELIMIT (-6)        /* a count exceeds a fixed maximum of the call            */

#define NUMA_MAX_N 7            /* orders N = 1 .. 7 (Nq = 2 .. 8): every mode, the batch
                                   and the engine                                         */
#define NUMA_MAX_N_FP64 15      /* NUMA_FP64 and NUMA_MIXED evaluations also take
                                   N = 8 .. 15 (Nq up to 16)                              */

/* Physical constants: EOS reference pressure p0, gas constant R, specific heat
 * at constant pressure cp (gamma = cp / (cp - R), Sec. 2), gravity grav. */
typedef struct {
    double p0, R, cp, grav;
} numa_constants;

/* Mesh size: num_elements hexahedra of order N (Nq = N + 1 points per axis),
 * and num_tracers passive tracers (0 .. NUMA_MAX_TRACERS; every precision,
 * tracers FP64 in NUMA_FP64 and NUMA_DF64, FP32 values as they are in
 * NUMA_MIXED; in the batch, its no-allocation advance and the engine): the
 * state and rhs then hold 5 + num_tracers planes, the tracers Q1.. after
 * Theta, each advected like Theta (flux Q u_d, no source; the paper's 8-field
 * form, Sec. 2).  Zero-initialise the struct so that num_tracers defaults to 0. */
#define NUMA_MAX_TRACERS 3
typedef struct {
    int64_t num_elements;
    int N;
    int num_tracers;
} numa_mesh;

/* Per-point geometry and reference state, FP64, M values each, in the layout
 * above.  Host or device pointers (the library copies them).
 *   g[3*d + a] = g_{a+1,d+1} = J * d(xi_d)/d(x_a) for reference direction d
 *                (0 = r, 1 = s, 2 = t) and physical axis a (0 = x, 1 = y,
 *                2 = z): the paper's geometric-factor slots 1-3 (r) and 4-6
 *                (s), a fastest, extended by slots 7-9 for t.
 *   Jinv       = 1 / J (the paper's slot 10).
 *   rho_ref, rhotheta_ref = reference density and reference Theta. */
typedef struct {
    const double *g[9];
    const double *Jinv;
    const double *rho_ref;
    const double *rhotheta_ref;
} numa_geometry;

typedef enum {
    NUMA_FP64 = 0,   /* FP64 state and rhs, every operation on the FP64 pipe           */
    NUMA_MIXED = 1,  /* FP32 perturbation state (rho', U1, U2, U3, Theta'), FP32 rhs,
                        FP32 geometry and arithmetic                                    */
    NUMA_DF64 = 2    /* FP64 state and rhs, double-float arithmetic (hi + lo FP32 pairs,
                        about 48 significant bits) on the FP32 pipes; N = 1..7        */
} numa_precision;

typedef struct numa_vol numa_vol;

/*
 * Create a handle for one mesh on the current CUDA device.
 *
 * Copies the geometry and reference arrays into device memory owned by the
 * handle (the caller's arrays may be freed afterwards).  It builds the GLL
 * differentiation matrix for N and evaluates, once per point on the device,
 * 1/Theta_ref and p(Theta_ref)/Theta_ref.  p' is exactly zero wherever
 * Theta == Theta_ref.  Synchronous.
 *
 * mesh->N in [1, NUMA_MAX_N_FP64] for NUMA_FP64 and NUMA_MIXED, and in
 * [1, NUMA_MAX_N] for NUMA_DF64; mesh->num_elements >= 0; every pointer of
 * geo non-null;
 * c->cp > c->R > 0 and c->p0 > 0.  On success *out receives the handle
 * (release with numa_vol_destroy).  Errors: NUMA_EINVAL, NUMA_ENOMEM,
 * NUMA_ECUDA, NUMA_EUNSUPPORTED (NUMA_DF64 with N > 7).
 * Handles of N > 7 evaluate one element per CTA of 3 or 4 (N+1)^2 threads,
 * the fields in groups (vol_rhs_high_kernel); the batch, the engine and
 * numa_batch_advance_noalloc take handles of N <= 7.
 *
 * NUMA_MIXED takes the state as FP32 perturbations from the reference state:
 * plane 0 holds rho - rho_ref, plane 4 holds Theta - Theta_ref, planes 1-3
 * hold U1..U3, and tracer planes (if any) hold the tracers as they are.  It
 * writes the (same) rhs in FP32.  The geometry is rounded to
 * FP32 once.  p' is evaluated from Theta - Theta_ref without cancellation
 * (series in x, or expm1(gamma log1p(x))).  Error against the FP64 volume term
 * of the full state: about 1e-7 times the sweep condition number, normwise.
 *
 * NUMA_FP64 and NUMA_DF64 compute the same operation.  Both evaluate
 * p(Theta) - p(Theta_ref) as p_ref ((1 + x)^gamma - 1) in x =
 * (Theta - Theta_ref)/Theta_ref: NUMA_FP64 by its binomial series (|x| <= 1/8)
 * or expm1(gamma log1p(x)), the form chosen per warp of 32 points;
 * NUMA_DF64 by the series where |x| <= 1/64 and by pow elsewhere.  The error
 * of NUMA_FP64 against an exact evaluation is a few units of 2^-53 times the
 * condition number of the D sweeps (the ratio of
 * sum |Jinv D F| to |rhs|).  The factor for NUMA_DF64 is about 2^-48, so
 * NUMA_DF64 suits states with well-conditioned sweeps, such as the benchmark's
 * per-point random velocities.  Smooth fields with a large mean (a uniform wind)
 * need NUMA_FP64.  NUMA_DF64 falls back to native FP64: for the whole handle
 * when a geometry array (after values below 2^-50 of the array's largest
 * magnitude are set to zero) holds a magnitude outside [2^-40, 2^41); and for
 * one element when its state holds such a value or its double-float result
 * overflows.  N > 7 with NUMA_DF64 gives NUMA_EUNSUPPORTED.
 */
int numa_vol_create(const numa_mesh *mesh, const numa_geometry *geo,
                    const numa_constants *c, numa_precision prec, numa_vol **out);

/*
 * Enqueue one evaluation of the volume term on a CUDA stream.
 *
 * q:   device pointer, 5 (+ num_tracers) planes of M values (read only):
 *      doubles for NUMA_FP64 and NUMA_DF64, floats (perturbation form) for
 *      NUMA_MIXED.
 * rhs: device pointer, as many planes of the same type (overwritten; the
 *      paper's kernel accumulates into rhsq, this call stores the volume term).
 * Both must be 16-byte aligned and must not overlap.  stream is a
 * cudaStream_t (NULL = the legacy default stream).  The call returns once
 * the kernel is enqueued; rhs is complete when the stream reaches that
 * point.  Errors: NUMA_EINVAL (null handle/pointer, misalignment,
 * overlap), NUMA_ECUDA (launch failure).  Ne = 0 enqueues nothing.  The call
 * may be made while `stream` is being captured into a CUDA graph (after one
 * call outside capture on the device); a replay evaluates the captured q into
 * the captured rhs.
 */
int numa_vol_rhs(numa_vol *h, const void *q, void *rhs, void *stream);

/*
 * Evaluate the volume term from HOST memory: copies q to the device, runs the
 * kernel, copies rhs back and waits for completion.  The mesh is processed in
 * up to 64 chunks of elements (NUMA_FP64; 16 for NUMA_DF64 and NUMA_MIXED) on four
 * internal streams, so the copy-in of one
 * chunk, the kernel on the previous one and the copy-out of the one before
 * overlap; each chunk moves with one 2D copy per direction over all planes.  Device staging buffers
 * (2 x (5 + num_tracers) x M values) are allocated on the first call and
 * owned by the handle.  q and rhs are host pointers to 5 (+ num_tracers)
 * planes of M values of the
 * handle's state type (pinned memory gives full copy bandwidth).  Errors:
 * NUMA_EINVAL, NUMA_ENOMEM, NUMA_ECUDA.
 */
int numa_vol_rhs_host(numa_vol *h, const void *q, void *rhs);

/*
 * Status of the kernels enqueued so far on a handle.  Reads and clears the
 * handle's device status word on `stream` and waits for the stream.  Returns
 * NUMA_ETIMEOUT if a kernel of the handle gave up a bounded device-side wait
 * (every wait in the library's kernels has a time limit far above its normal
 * duration; the evaluation kernels themselves do not wait, and the self-test
 * below makes one such wait run out).  Returns NUMA_OK otherwise.
 * numa_vol_rhs_host checks it itself.
 */
int numa_vol_status(numa_vol *h, void *stream);

/*
 * Failure-detection self-test: makes a bounded device-side wait run out.
 * Enqueues on `stream` one CTA that waits, with the library's bounded
 * mbarrier wait, on a barrier nothing completes; after limit_us
 * microseconds (1 .. 1,000,000) of GPU time the wait gives up and sets the
 * handle's status word, so that a following numa_vol_status on the same
 * stream returns NUMA_ETIMEOUT.  No copy or other asynchronous work is in
 * flight when it gives up: the context and the handle stay usable.  Returns
 * NUMA_EINVAL for a NULL handle or a limit out of range, NUMA_ECUDA if the
 * launch fails, NUMA_OK otherwise.
 */
int numa_vol_selftest_wait(numa_vol *h, uint32_t limit_us, void *stream);

/* Release a handle and its device memory.  NULL is a no-op.  Synchronises
 * the device before freeing. */
void numa_vol_destroy(numa_vol *h);

/* Name of the kernel numa_vol_rhs launches for this handle:
 * "vol_rhs_fp64_kernel<Nq>" (NUMA_FP64, or NUMA_DF64 after a geometry
 * fallback), "vol_rhs_df64_kernel" or "vol_rhs_mixed_kernel<Nq>".  Static
 * string; "" for a NULL handle. */
const char *numa_vol_kernel_name(const numa_vol *h);

/*
 * How the three D sums of the volume term (Sec. 2, Eq. (2)) are evaluated:
 *   NUMA_SWEEP_CUDA_CORES   FMAs on the CUDA cores (every mode's default; in
 *                           NUMA_MIXED FP32 with relative error about 2^-24
 *                           times the sums' condition number);
 *   NUMA_SWEEP_TENSOR_TF32  TF32 split products on the tensor cores (tcgen05)
 *                           with FP32 accumulation in tensor memory: each flux
 *                           and each entry of D is a TF32 head plus an FP32
 *                           tail, and the sums take head x head, head x tail
 *                           and tail x head (relative error about 2^-21 times
 *                           the condition number); NUMA_MIXED only;
 *   NUMA_SWEEP_AUTO         batches only (numa_batch_set_sweep).
 */
typedef enum {
    NUMA_SWEEP_CUDA_CORES = 0,
    NUMA_SWEEP_TENSOR_TF32 = 1,
    NUMA_SWEEP_AUTO = 2
} numa_sweep;

/* Choose the sweep of a handle: NUMA_SWEEP_TENSOR_TF32 takes NUMA_MIXED
 * handles of N = 7 without tracers (vol_rhs_mixed_tc_kernel: a persistent
 * grid, one element per CTA, one MMA round per element); NUMA_SWEEP_CUDA_CORES
 * any handle.  The first tensor-core choice on a device uploads the kernel's
 * tables (synchronous): make it before any stream capture.  A bounded wait of
 * that kernel that runs out is reported by numa_vol_status (NUMA_ETIMEOUT).
 * Errors: NUMA_EINVAL (NULL handle, NUMA_SWEEP_AUTO or unknown value),
 * NUMA_EUNSUPPORTED, NUMA_ECUDA. */
int numa_vol_set_sweep(numa_vol *h, numa_sweep sweep);

/* Message for the last error on the calling thread ("" if none).  The
 * pointer stays valid until the thread's next numa_vol call. */
const char *numa_vol_last_error(void);

/*
 * Host-only: write the (N+1) x (N+1) GLL differentiation matrix the kernels
 * apply, row-major, D[i*(N+1) + n] = l_n'(xi_i) (the paper's D(i,n)), into
 * D_out, for N in [1, NUMA_MAX_N_FP64].  Needs no GPU.  Errors: NUMA_EINVAL.
 */
int numa_vol_diff_matrix(int N, double *D_out);

/* ------------------------------------------------------------------------- */
/* Batched time integration                                                  */
/* ------------------------------------------------------------------------- */

/*
 * A batch advances many instances (handles of any order and size) of
 * dq/dt = v(q), with v the volume term above, by the five-stage fourth-order
 * low-storage Runge-Kutta scheme of Carpenter and Kennedy (NASA TM-109112,
 * 1994).  Per stage s = 0..4: dq <- A_s dq + dt v(q), q <- q + B_s dq, with
 * dq = 0 at the start of each call.  The paper (Sec. 2) frames the volume term
 * as the rate function of such an explicit solver.
 *
 * The volume term couples only the points of one element, so elements advance
 * independently: one persistent kernel takes tiles of elements of every
 * instance through all stages with q and dq on chip.  Each element's result
 * is the same whichever other instances share the launch (bitwise), because
 * its arithmetic does not depend on them.  The kernel, and the reset of its
 * work counter, are captured once in a CUDA graph per (nsteps, dt) and
 * replayed.
 */
typedef struct numa_batch numa_batch;

/* Create an empty batch on the current device.  prec: NUMA_FP64 (native FP64
 * handles, FP64 state) or NUMA_MIXED (mixed handles, FP32 perturbation state).
 * Errors: NUMA_EINVAL, NUMA_EUNSUPPORTED (other precisions), NUMA_ENOMEM,
 * NUMA_ECUDA. */
int numa_batch_create(numa_precision prec, numa_batch **out);

/* Add an instance: handle h (created with the batch's precision on the same
 * device; the batch neither copies nor frees it, and it must outlive its use
 * in the batch) and its state q, a device pointer to 5 (+ num_tracers) planes
 * of M values of the handle's state type, 16-byte aligned, that
 * numa_batch_advance updates in place.  *index (optional) receives the
 * instance's position.  A batch holding an instance with tracers runs the
 * shared-memory-state tiles' tracer forms for all its instances; its
 * tensor-core sweep and tensor-memory state settings then have no effect.
 * Errors: NUMA_EINVAL; NUMA_EUNSUPPORTED for a handle of order N > NUMA_MAX_N. */
int numa_batch_add(numa_batch *b, const numa_vol *h, void *q, int *index);

/* Remove every instance (the handles and states are untouched). */
int numa_batch_clear(numa_batch *b);

/* Number of instances. */
int numa_batch_size(const numa_batch *b);

/* Advance every instance by nsteps steps of size dt, as one graph launch on
 * `stream` (asynchronous).  The first call after the batch changed uploads
 * the work list (synchronous) and captures the graph.  Errors: NUMA_EINVAL,
 * NUMA_ENOMEM, NUMA_ECUDA. */
int numa_batch_advance(numa_batch *b, int nsteps, double dt, void *stream);

/* Choose the launch configuration (numa_batch_config below) by timing
 * launches of two steps on copies of the current states, best of three per
 * candidate (synchronous; states unchanged).  First each order alone over its
 * tiles (1, 2, 4, 8, 16 or 32 passes of 512 threads per work item), and under
 * NUMA_SWEEP_AUTO over both sweeps; then, in the launch the batch actually
 * runs (all orders together), one round of coordinate descent over each
 * order's candidates, the CTAs per SM of the persistent grid, the order of
 * the work items and (NUMA_MIXED) where the CUDA-core tiles keep the state,
 * keeping a change that saves at least 1 %. */
int numa_batch_autotune(numa_batch *b, void *stream);

/* Launch configuration of a batch.  Indices are Nq = N + 1 (2..8; 0 and 1
 * unused). */
typedef struct {
    int tile[9];               /* elements per work item: a positive multiple of
                                  512 / Nq^3 (the elements one pass of 512
                                  threads holds) */
    int sweep[9];              /* NUMA_SWEEP_CUDA_CORES or NUMA_SWEEP_TENSOR_TF32 */
    int ctas_per_sm;           /* CTAs per SM of the persistent grid: 1 .. 2
                                  (NUMA_MIXED) or 1 (NUMA_FP64); 0 = the most */
    int costliest_first;       /* nonzero: work items sorted by points, largest
                                  first (else instance by instance) */
    int state_in_tmem;         /* NUMA_MIXED, nonzero (the default): the
                                  CUDA-core tiles keep each point's q, dq,
                                  metric terms and J^-1 in tensor memory rather
                                  than shared memory */
    double tuned_ms_per_step;  /* read only: the last autotune's time for one
                                  step of the chosen configuration (0: none) */
    int tuned_candidates;      /* read only: launches the last autotune timed */
} numa_batch_config;

/* Read the current configuration.  Errors: NUMA_EINVAL. */
int numa_batch_get_config(const numa_batch *b, numa_batch_config *out);

/* Set tiles, sweeps, CTAs per SM and item order (the read-only fields are
 * ignored); applies from the next numa_batch_advance.  Errors: NUMA_EINVAL
 * (a field out of range), NUMA_EUNSUPPORTED (a tensor-core sweep in a
 * NUMA_FP64 batch). */
int numa_batch_set_config(numa_batch *b, const numa_batch_config *c);

/* Elements per work item the batch uses for order Nq (2..8). */
int numa_batch_tile(const numa_batch *b, int nq);

/*
 * How a NUMA_MIXED batch evaluates the three D sums of the volume term
 * (numa_sweep, declared with numa_vol_set_sweep above): NUMA_SWEEP_CUDA_CORES
 * (the default), NUMA_SWEEP_TENSOR_TF32 at every order, or NUMA_SWEEP_AUTO:
 * numa_batch_autotune times both for each order present and keeps the faster
 * (until it runs, the previous choice per order stands).  The choice applies
 * from the next numa_batch_advance.  NUMA_FP64 batches take
 * NUMA_SWEEP_CUDA_CORES only (tcgen05 has no FP64 kind).
 * Errors: NUMA_EINVAL (NULL batch or unknown value), NUMA_EUNSUPPORTED.
 */
int numa_batch_set_sweep(numa_batch *b, numa_sweep sweep);

/* The sweep mode last set (a numa_sweep value), or -1 for a NULL batch. */
int numa_batch_sweep(const numa_batch *b);

/* The sweep order Nq (2..8) uses now: NUMA_SWEEP_CUDA_CORES or
 * NUMA_SWEEP_TENSOR_TF32; -1 for a NULL batch or an Nq outside 2..8. */
int numa_batch_sweep_of(const numa_batch *b, int nq);

/*
 * Read and clear the batch's device status word, after the work on `stream`
 * has finished (synchronous).  NUMA_ETIMEOUT: a launch's bounded wait for the
 * tensor core ran out; that launch stopped early and the states it was
 * advancing are not valid.  NUMA_OK otherwise.  Errors: NUMA_EINVAL, NUMA_ECUDA.
 */
int numa_batch_status(numa_batch *b, void *stream);

/* Message for the last batch error on the calling thread. */
const char *numa_batch_last_error(void);

/* Release a batch (synchronises the device first).  NULL is a no-op. */
void numa_batch_destroy(numa_batch *b);

/* ------------------------------------------------------------------------- */
/* Serving engine: continuous batching of ensemble-member requests           */
/* ------------------------------------------------------------------------- */

/*
 * An engine serves requests, each an ensemble member to be advanced: a mesh
 * (a numa_vol handle the caller created and keeps alive), an initial state in
 * host memory, a number of low-storage RK steps and a step size.  The engine
 * reserves its HBM budget once, as an arena for members' states, and admits
 * requests in arrival order while a member slot is free and the arena has room.
 * Each numa_engine_progress call enqueues one round without waiting for the
 * GPU: upload newly admitted states (on a copy stream), advance every
 * resident member by one step (or several, numa_engine_set_round_steps) in one
 * persistent launch (one per distinct dt) queued behind the previous round,
 * and copy the states of members that finish with it to their host buffers
 * (on a second copy stream).  Uploads and downloads overlap the launches, and
 * requests submitted while a round runs join the next one.  A request is done
 * when its final state is in host memory; progress reports it then, in the
 * same or a later call.  Work tables are reserved at create time: no round
 * allocates memory.  A member's result is bitwise the same whichever members
 * share its rounds.  Engines are not thread-safe.
 */
typedef struct numa_engine numa_engine;

#define NUMA_REQ_QUEUED 0
#define NUMA_REQ_RUNNING 1
#define NUMA_REQ_DONE 2
#define NUMA_REQ_CANCELLED 3

typedef struct {
    int64_t id;
    int status;                        /* NUMA_REQ_*                                    */
    double submit_s, admit_s, done_s;  /* steady-clock seconds (0 where not reached)    */
} numa_request_info;

typedef struct {
    int queued, resident;
    size_t bytes_used, bytes_budget;   /* arena bytes held by members / reserved         */
    int64_t completed, rounds;
    double point_stages;               /* sum over launches of points x 5 RK stages      */
} numa_engine_counters;

/* Create an engine on the current device: prec NUMA_FP64 or NUMA_MIXED,
 * budget_bytes of device memory reserved now for members' states, at most
 * max_members resident.  Errors: NUMA_EINVAL, NUMA_EUNSUPPORTED, NUMA_ENOMEM
 * (the budget cannot be reserved), NUMA_ECUDA. */
int numa_engine_create(numa_precision prec, size_t budget_bytes, int max_members,
                       numa_engine **out);

/* Queue a request.  mesh: a handle of the engine's precision on its device.
 * q0_host: the initial state (5 + num_tracers planes of M values of the
 * handle's state type; a round holding a member with tracers runs the batch's
 * tracer tiles)
 * and q_out_host: where the final state goes; both host memory, read and
 * written during later progress calls, kept alive until the request is done or
 * cancelled.  nsteps >= 1, dt > 0.  *id receives the request id.
 * Errors: NUMA_EINVAL (malformed request; the engine is unchanged),
 * NUMA_ELIMIT (the state exceeds the whole budget: it can never be admitted),
 * NUMA_EUNSUPPORTED (a mesh of order N > NUMA_MAX_N). */
int numa_engine_submit(numa_engine *e, const numa_vol *mesh, const void *q0_host,
                       void *q_out_host, int nsteps, double dt, int64_t *id);

/* Cancel a queued request now, or a running one at the start of the next
 * round (its state is discarded).  Errors: NUMA_EINVAL (unknown or finished). */
int numa_engine_cancel(numa_engine *e, int64_t id);

/* One round, enqueued on the device (see above).  Up to max_done ids of
 * requests whose final state has reached host memory since the last call go
 * to done_ids, their count to *num_done.  The call waits only when two
 * launches are already in flight (for the older one), when a cancelled member's
 * last launch has to finish before its memory is freed, and, with no member
 * to advance, for the oldest result still being copied out.
 * Errors: NUMA_ECUDA. */
int numa_engine_progress(numa_engine *e, int64_t *done_ids, int max_done, int *num_done);

/* Wait for everything enqueued (launches and copies) and report the requests
 * that finished, like numa_engine_progress, without starting a round.
 * Errors: NUMA_EINVAL, NUMA_ECUDA. */
int numa_engine_drain(numa_engine *e, int64_t *done_ids, int max_done, int *num_done);

/* Status and timestamps of a request.  The engine keeps the records of its
 * 2^20 most recently finished (done or cancelled) requests; an older finished
 * id, like an unknown one, returns NUMA_EINVAL. */
int numa_engine_query(const numa_engine *e, int64_t id, numa_request_info *out);

/* Steps per round (default 1).  A round then advances every resident member
 * by s = min(max_steps, the smallest remaining step count of the residents)
 * steps in one launch, with each member's state kept on chip across them: no
 * member finishes later than with single steps, and results are bit for bit
 * the same, but requests arriving during a round wait up to s steps for
 * admission.  Errors: NUMA_EINVAL (NULL engine, max_steps < 1). */
int numa_engine_set_round_steps(numa_engine *e, int max_steps);

/* How a round with a step limit above 1 (numa_engine_set_round_steps) splits
 * its steps among the residents.
 *   NUMA_ROUND_LOCKSTEP (default): every member advances by the same s, the
 *     smallest remaining step count up to the limit (above).
 *   NUMA_ROUND_PER_MEMBER: each member advances by its own min(limit, its
 *     remaining steps) in the same launch (the persistent kernel takes the
 *     costliest work items first).  Long requests no longer advance at the
 *     pace of the shortest one, so they finish in fewer rounds; a short
 *     request now waits, within its round, for the longer members' steps.
 * Results are bit for bit the same under either policy.  Errors: NUMA_EINVAL
 * (NULL engine, unknown policy). */
#define NUMA_ROUND_LOCKSTEP 0
#define NUMA_ROUND_PER_MEMBER 1
int numa_engine_set_round_policy(numa_engine *e, int policy);

/* Checkpoint of a queued or running request: copies its state after its last
 * completed step (the initial state if not yet admitted) into state_host
 * (host memory of the mesh's state size) and stores the number of steps done
 * in *steps_done (optional).  A step of the scheme depends on the state alone,
 * so submitting that state with the remaining steps, to this or another
 * engine, resumes the request: the final state is bit for bit the one the
 * uninterrupted request produces.  Synchronous; call between progress calls.
 * Errors: NUMA_EINVAL (NULL argument; no queued or running request with this
 * id), NUMA_ECUDA. */
int numa_engine_checkpoint(numa_engine *e, int64_t id, void *state_host, int *steps_done);

/* Counters of the engine. */
int numa_engine_stats(const numa_engine *e, numa_engine_counters *out);

/* Message for the last engine error on the calling thread. */
const char *numa_engine_last_error(void);

/* Release an engine and its reserved memory (queued requests are dropped). */
void numa_engine_destroy(numa_engine *e);

/*
 * Advance instances like numa_batch_advance, without allocating any memory.
 * The paper has no counterpart.  It is for callers that cannot call
 * cudaMalloc once running.  An example is a serving process that has committed
 * all of its HBM budget to resident ensemble states; another is an
 * application whose allocator forbids growth after start-up.
 *
 * handles[k] (NUMA_FP64 or NUMA_MIXED handles, all of one kind, on the current
 * device) and states[k] (its state: a device pointer, 16-byte aligned, updated
 * in place), for k < count, with 1 <= count <= NUMA_NOALLOC_MAX_INSTANCES.
 * Each call advances every instance by nsteps steps of size dt, with the same
 * scheme, tiles (4 passes per work item) and per-element arithmetic as a
 * numa_batch of those handles without autotuning.
 *
 * Scratch: the work counter and the instance table live in one fixed __device__
 * array of the library (about 57 KB, held by every GPU that loads the library
 * until the process exits).  The first call on a device does a one-time
 * set-up there: it looks up the array's device address and sets the kernel's
 * shared-memory limit.  Every call overwrites the same array, so calls whose
 * kernels may overlap on the GPU (other streams, other host threads) race.
 * Serialise them on one stream.
 *
 * The call builds the table on its own stack, copies it into the array,
 * zeroes the counter and launches, all on `stream` (asynchronous).  The copy
 * reads the stack frame while the call runs, which holds only when the
 * stream is executing, not when it is being captured into a CUDA graph: a
 * stream under capture is refused with NUMA_EINVAL before anything is
 * enqueued (the capture itself stays valid).  It calls no allocator: no
 * cudaMalloc or cudaFree, no host heap, and it records no error message.
 * Returns NUMA_OK; NUMA_ELIMIT if count > NUMA_NOALLOC_MAX_INSTANCES (or the
 * total work exceeds 2^31 - 1 items); NUMA_EINVAL for a NULL or misaligned
 * pointer, count < 1, nsteps < 0, handles of mixed kinds or of another device,
 * a double-float handle, or a stream under capture; NUMA_EUNSUPPORTED for a
 * handle of order N > NUMA_MAX_N; NUMA_ECUDA if a CUDA call
 * fails.
 */
#define NUMA_NOALLOC_MAX_INSTANCES 64
int numa_batch_advance_noalloc(const numa_vol *const *handles, void *const *states, int count,
                               int nsteps, double dt, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* NUMA_VOL_H */
