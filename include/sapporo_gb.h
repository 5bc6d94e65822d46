/*
 * sapporo_gb.h -- C ABI of the GB300 (sm_103a) direct-summation gravity library.
 *
 * The library implements the hot path of the Sapporo2 method (Bedorf, Gaburov &
 * Portegies Zwart 2015): store j-particles (sources) in FP64, Taylor-predict
 * them to a common time, and sum over them, for a list of active i-particles
 * (sinks), the Plummer-softened acceleration, jerk, snap (6th order),
 * potential and nearest neighbour.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Units: G = 1.  Potential is negative.  Softening enters as r.r + eps2.
 *  - Vectors are n x 3 row-major FP64 arrays (x0 y0 z0 x1 y1 z1 ...).
 *  - ptr_kind = SP2_HOST: every array argument of the call is host memory; the
 *    call copies in, runs, copies out and returns when the results are in
 *    place (synchronous).  ptr_kind = SP2_DEVICE: every array argument is
 *    device memory of the context's GPU; the call only enqueues work on the
 *    context's stream and returns (asynchronous; sp2_sync waits).
 *  - Ownership: the caller owns every array it passes; the library never keeps
 *    a caller pointer after a call returns.  The library owns its device copy
 *    of the j-particles, the predicted records and its scratch space.
 *  - Errors: every call returns an sp2_status; no exception or signal crosses
 *    the ABI.  On error nothing is written to the outputs, and
 *    sp2_last_error() returns a message.  A CUDA error makes the context
 *    unusable (SP2_ERR_CUDA from every later call).
 *  - Threads: a context is used by one host thread at a time.
 *  - Self-interaction: the sink is itself a loaded j-particle (given by slot),
 *    and the pair with itself is skipped.  Particle ids must be unique; the
 *    nearest-neighbour output reports the neighbour's id.
 *  - Precision: SP2_FP64 computes everything in IEEE double.  SP2_MIXED
 *    predicts in FP64, stores positions as double-single (FP32 hi + lo) pairs,
 *    forms x_j - x_i in double-single, evaluates rsqrt and the force terms in
 *    FP32, and accumulates per-thread partial sums in FP32 that are flushed
 *    into FP64 every tile; partial results of different j-slices are combined
 *    in FP64.
 */
#ifndef SAPPORO_GB_H
#define SAPPORO_GB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sp2_ctx sp2_ctx;
typedef struct sp2_graph sp2_graph;
typedef struct sp2_batch_plan sp2_batch_plan;

typedef enum {
    SP2_OK = 0,
    SP2_ERR_ARG = -1,        /* null pointer, bad enum, negative size */
    SP2_ERR_RANGE = -2,      /* size or index outside the context's capacity / loaded set */
    SP2_ERR_NOMEM = -3,      /* device allocation failed */
    SP2_ERR_CUDA = -4,       /* a CUDA runtime call or kernel failed */
    SP2_ERR_STATE = -5,      /* call out of order (e.g. compute before predict) */
    SP2_ERR_TIMEOUT = -6,    /* a bounded device-side wait gave up */
    SP2_ERR_NONFINITE = -7,  /* the optional output scan found NaN or Inf */
    SP2_ERR_UNSUPPORTED = -8 /* option not available in this configuration */
} sp2_status;

enum { SP2_FP64 = 0, SP2_MIXED = 1 };
enum { SP2_HOST = 0, SP2_DEVICE = 1 };

/* Optional device allocator (e.g. a caching allocator of the host program).
 * alloc returns NULL on failure; free accepts what alloc returned. */
typedef void *(*sp2_alloc_fn)(size_t bytes, void *user);
typedef void (*sp2_free_fn)(void *ptr, void *user);

typedef struct {
    int order;            /* 4 (Hermite-4: acc, jerk, pot), 6 (adds snap), or 2        */
                          /* (leap-frog / GRAPE-5 of Sec. 1: acc and pot only; sources */
                          /* are used at their stored positions, not predicted)        */
    int precision;        /* SP2_FP64 or SP2_MIXED                                     */
    int64_t n_max;        /* capacity: number of j-particle slots                      */
    double eps2;          /* softening length squared, >= 0                            */
    int with_nn;          /* 1: compute the nearest neighbour (id, r^2); 0: skip it     */
    void *cuda_stream;    /* borrowed cudaStream_t, NULL: the library creates one      */
    sp2_alloc_fn alloc;   /* NULL: cudaMalloc                                          */
    sp2_free_fn free;     /* NULL: cudaFree                                            */
    void *alloc_user;     /* passed to alloc / free                                    */
    int profile;          /* 1: time each kernel with CUDA events (sp2_profile_read)   */
    int check_finite;     /* 1: scan outputs for NaN/Inf after each compute (syncs)    */
} sp2_config;

/* Launch shape of the force kernel (the autotuner's search space). */
typedef struct {
    int threads;       /* threads per CTA: 32, 64, 128 or 256                         */
    int i_per_thread;  /* sinks held by one thread: 1, 2 or 4                          */
    int j_lanes;       /* threads sharing one sink (the paper's 2D blocks): 1, 2, 4,
                          ..., threads.  Up to 32 they are lanes of one warp, each
                          taking every j_lanes-th source of a tile; above 32
                          (SP2_MIXED, i_per_thread 1) j_lanes / 32 warps share
                          the sink, each taking its own contiguous part of
                          every tile                                          */
    int j_tile;        /* sources staged in shared memory per pipeline stage          */
    int split_j;       /* source slices processed independently, combined by the
                          FP64 reduction kernel (1: no reduction pass)                */
    int ctas_per_sm;   /* persistent-grid residency, 0 = occupancy maximum           */
} sp2_launch;

/* Fill *cfg with defaults: order 4, SP2_MIXED, n_max 0, eps2 0, with_nn 1, no
 * borrowed stream, cudaMalloc, no profiling, no finite check. */
void sp2_config_default(sp2_config *cfg);

/* Create a context on the current CUDA device (Sec. 2.2: one particle store and
 * its kernels per device).  Allocates the j store for cfg->n_max particles.
 * Errors: SP2_ERR_ARG (order not 2/4/6, precision, n_max <= 0 or > 2^30,
 * eps2 < 0 or not finite, alloc without free), SP2_ERR_NOMEM, SP2_ERR_CUDA. */
sp2_status sp2_open(sp2_ctx **out, const sp2_config *cfg);

/* Release everything the context owns (not a borrowed stream).  NULL is a no-op. */
sp2_status sp2_close(sp2_ctx *ctx);

/* Copy kernel (Sec. 2.2.4, "copy kernel"): store n j-particles.
 *  slots == NULL: into slots first .. first+n-1 (first <= loaded count, so the
 *                 loaded slots stay contiguous; first + n <= n_max); the loaded
 *                 count becomes max(loaded, first + n).
 *  slots != NULL: particle k goes to slot slots[k] (int32, each < loaded count;
 *                 `first` is ignored); used to update the active particles of a
 *                 block step.
 * id[n] int32, m[n], x/v/a/jerk[n x 3], snap[n x 3] (order 6 only, else NULL),
 * t[n] (time at which x, v, a, jerk, snap are valid).  Order 2 needs only id,
 * m and x (v, a, jerk, t may be NULL: they are not used).  Marks the predicted
 * records stale.  Errors: SP2_ERR_ARG, SP2_ERR_RANGE. */
sp2_status sp2_set_j(sp2_ctx *ctx, int64_t first, int64_t n, const int32_t *slots,
                     const int32_t *id, const double *m, const double *x, const double *v,
                     const double *a, const double *jerk, const double *snap,
                     const double *t, int ptr_kind);

/* Predictor (Sec. 2.2.4 "predict" kernel; Hermite predictor of Makino & Aarseth
 * 1992 / Nitadori & Makino 2008): Taylor-expand every loaded j-particle from its
 * own t_j to t and write the predicted records used by sp2_compute (FP64
 * records, or double-single records in SP2_MIXED).  FP64: dt^k/k! is formed as
 * dt^k times the double nearest 1/k!, sums left to right.  SP2_MIXED evaluates
 * the polynomial in double-single arithmetic from a double-single copy of the
 * store, and defers the work: the next sp2_compute with few enough sinks
 * predicts its sources inside the force pass, any other consumer writes the
 * records first.  Results do not depend on which happens.  Order 2 (leap-frog)
 * takes the stored positions as they are.
 * Errors: SP2_ERR_STATE (nothing loaded), SP2_ERR_ARG (t not finite). */
sp2_status sp2_predict(sp2_ctx *ctx, double t);

/* Gravity kernel (Sec. 2.1 and 2.2.4): for each of the n_i sinks, given as
 * slots i_idx[n_i] (int32) of the loaded set, sum over the sources in slots
 * j_begin .. j_end-1 (sp2_compute: all loaded) except itself:
 *   acc[n_i x 3], jerk[n_i x 3] (order 4 and 6; NULL for order 2),
 *   snap[n_i x 3] (order 6; else pass NULL),
 *   pot[n_i], nn_id[n_i] (int32, -1 when there is no other source),
 *   nn_r2[n_i] (unsoftened squared distance, +inf when none).
 * Any output may be NULL (not computed / not written); nn_* need with_nn.
 * Sinks are the predicted j-particles at t.  The source range is split into
 * slices over the whole GPU when n_i is small (Sec. 2.1, the source-split
 * method), and the slices are combined by a deterministic FP64 reduction
 * (inside the force kernel, or a second kernel for large slice counts).
 * Errors: SP2_ERR_STATE (records stale: call sp2_predict),
 * SP2_ERR_RANGE (slot >= loaded count, bad range), SP2_ERR_ARG,
 * SP2_ERR_NONFINITE (check_finite). n_i == 0 is a successful no-op. */
sp2_status sp2_compute(sp2_ctx *ctx, int64_t n_i, const int32_t *i_idx,
                       double *acc, double *jerk, double *snap, double *pot,
                       int32_t *nn_id, double *nn_r2, int ptr_kind);
sp2_status sp2_compute_range(sp2_ctx *ctx, int64_t j_begin, int64_t j_end,
                             int64_t n_i, const int32_t *i_idx,
                             double *acc, double *jerk, double *snap, double *pot,
                             int32_t *nn_id, double *nn_r2, int ptr_kind);

/* Forces on explicit sinks (the GRAPE-style form of the call, in which the
 * integrator sends the i-particles' own predicted state; Sec. 2.2.4 names the
 * i-particle data sent to the device): sink k has position xi[k], velocity
 * vi[k] and, for order 6, acceleration ai[k] (each [n_i x 3] double; vi may be
 * NULL for order 2).  i_slot[k] names the loaded slot that is the sink itself
 * (its self pair is skipped), or is negative when the sink is not one of the
 * loaded particles; i_slot == NULL means no sink is.  The sources are the
 * predicted records as for sp2_compute; outputs and errors as sp2_compute.
 * The paper has no separate call for this (the GRAPE API it implements does). */
sp2_status sp2_compute_ext(sp2_ctx *ctx, int64_t n_i, const int32_t *i_slot,
                           const double *xi, const double *vi, const double *ai,
                           double *acc, double *jerk, double *snap, double *pot,
                           int32_t *nn_id, double *nn_r2, int ptr_kind);

/* sp2_compute plus neighbour lists (Sec. 1: the library can return, for each
 * particle, the list of all particles within a given radius; Sec. 3: the
 * perturber lists of NBODY4-style integrators).  For sink k (position k of
 * i_idx) the neighbours are the other loaded particles j with unsoftened
 * |x_j - x_k|^2 < h2[k] (strict; the particle itself is never listed), r^2
 * formed as in the force pass (exact FP64, or the FP32 double-single
 * difference in mixed precision).
 *   h2       [n_i] double, squared radius per sink (<= 0: no neighbours).
 *   nb_max   list capacity per sink, 1 .. 4096.
 *   nb_count [n_i] int32 out: number of neighbours found.  A value above
 *            nb_max means the list overflowed: nb_max of the neighbours are
 *            listed (which ones is not defined) and the caller may retry with
 *            a smaller radius or a larger capacity.
 *   nb_ids   [n_i x nb_max] int32 out: row k holds min(nb_count[k], nb_max)
 *            neighbour ids in ascending order; the rest of the row is
 *            unspecified.
 * Needs a context opened with with_nn = 1 (the lists ride on the nearest-
 * neighbour kernels; nn_id / nn_r2 may still be NULL).  Runs with one sink per
 * thread.  Other arguments, layouts and errors as sp2_compute. */
sp2_status sp2_compute_nb(sp2_ctx *ctx, int64_t n_i, const int32_t *i_idx,
                          double *acc, double *jerk, double *snap, double *pot,
                          int32_t *nn_id, double *nn_r2,
                          const double *h2, int32_t nb_max, int32_t *nb_count,
                          int32_t *nb_ids, int ptr_kind);

/* Many independent systems (the few-body / planetary regime of Sec. 2.1):
 * system s owns the loaded slots offsets[s] .. offsets[s+1]-1 (host int64
 * array of n_sys + 1 increasing entries, offsets[n_sys] <= loaded), every
 * particle of every system is a sink, and only particles of the same system
 * interact.  The plan orders the (system, 32-sink chunk) work items by cost for
 * the persistent kernel's device-side work queue; build it once per set of
 * system sizes.  Errors: SP2_ERR_ARG, SP2_ERR_RANGE (a system larger than
 * 4096 particles, or offsets outside the loaded set). */
sp2_status sp2_batch_plan_create(sp2_ctx *ctx, int64_t n_sys, const int64_t *offsets,
                                 sp2_batch_plan **plan);
sp2_status sp2_batch_plan_destroy(sp2_batch_plan *plan);
/* Run the plan on the predicted records: outputs are indexed by slot - offsets[0]
 * (length offsets[n_sys] - offsets[0]), layouts as sp2_compute. */
sp2_status sp2_compute_batched(sp2_ctx *ctx, const sp2_batch_plan *plan,
                               double *acc, double *jerk, double *snap, double *pot,
                               int32_t *nn_id, double *nn_r2, int ptr_kind);

/* All-pairs forces of n particles given directly (no store, no predictor): every
 * particle is a sink and a source; m[n], x/v[n x 3] FP64; acc/jerk[n x 3],
 * pot[n] (any output may be NULL).  Order-4 quantities.  This is the forward of
 * the differentiable force below.  Uses the context's scratch (n <= n_max). */
sp2_status sp2_forces(sp2_ctx *ctx, int64_t n, const double *m, const double *x,
                      const double *v, double *acc, double *jerk, double *pot, int ptr_kind);

/* Vector-Jacobian product of sp2_forces: given cotangents abar, jbar [n x 3] and
 * pbar [n] (NULL = zero) of acc, jerk, pot, write
 *   xbar = sum abar . dacc/dx + jbar . djerk/dx + pbar . dpot/dx   [n x 3]
 *   vbar (same for v) [n x 3],  mbar [n].
 * One pairwise pass in which each pair contributes through both of its ends.
 * accumulate = 1 adds into xbar/vbar/mbar instead of overwriting. */
sp2_status sp2_force_vjp(sp2_ctx *ctx, int64_t n, const double *m, const double *x,
                         const double *v, const double *abar, const double *jbar,
                         const double *pbar, double *xbar, double *vbar, double *mbar,
                         int accumulate, int ptr_kind);

/* Read back loaded particles first .. first+n-1 from the store (any output may
 * be NULL): x, v, a, jerk [n x 3] and t [n], as last set by sp2_set_j or
 * advanced by sp2_block_run.  The paper has no counterpart (the integrator
 * keeps its own copy of the particles).  Errors: SP2_ERR_RANGE. */
sp2_status sp2_get_j(sp2_ctx *ctx, int64_t first, int64_t n, double *x, double *v,
                     double *a, double *jerk, double *t, int ptr_kind);

/* Block time-steps (Sec. 3.7: individual power-of-two time-steps; the paper
 * leaves the integrator to the host, here it runs on the device around the
 * force pass).  Order-4 contexts (sp2_block_run) and order-6 contexts
 * (sp2_block_run_h6).
 * sp2_block_init: the loaded particles (x, v and m, with t = t0 for all) get
 *   their acceleration and jerk (order 6: and snap, from a second pass that
 *   uses the first pass's accelerations; crackles zero) at t0 from a full
 *   pass and initial steps eta_s |a| / |j|, each the largest power of two not
 *   above that, dt_max at most, dividing t0.
 * sp2_block_run: repeat until the next block time exceeds t_end: the block
 *   time t1 = min_i(t_i + dt_i), the active set {i : t_i + dt_i = t1}, the
 *   prediction of all particles to t1, the force pass on the active set, and
 *   the 4th-order Hermite corrector (Makino & Aarseth 1992) on it, followed by
 *   Aarseth's time-step criterion with parameter eta (from the Hermite
 *   interpolation of the step), quantised to a power of two at most twice
 *   the last step and dt_max, dividing t1.  Afterwards every particle is at
 *   its own t_i <= t_end (all at t_end when t_end is a multiple of dt_max).
 *   Statistics go to *stats (may be NULL).
 *   Execution: the block time, the active count and a stop flag stay on the
 *   device; blocks are queued 32 at a time (the first 32 as plain launches,
 *   the rest by replaying one captured CUDA graph of 32 blocks) and the host
 *   reads the state once per 32 blocks.  A block past t_end makes the rest of
 *   its batch do nothing.  The force pass takes its shape (lanes per sink,
 *   source split) from the active count on the device.  Runs on the context's
 *   stream and returns after synchronising it; a stream that cannot be
 *   captured gets plain launches throughout.
 * sp2_block_run_h6: the same loop with the 6th-order Hermite scheme
 *   (Nitadori & Makino 2008; Sec. 3.7 runs it): the predictor carries each
 *   particle's crackle from its last correction (x to dt^5, v to dt^4, a to
 *   dt^3; FP64 arithmetic in both precisions), the pass gives acc, jerk and
 *   snap, and the corrector
 *     v1 = v0 + h/2 (a0 + a1) - h^2/10 (j1 - j0) + h^3/120 (s0 + s1)
 *     x1 = x0 + h/2 (v0 + v1) - h^2/10 (a1 - a0) + h^3/120 (j0 + j1)
 *   is followed by the crackle, pop and 5th derivative at t1 of the quintic
 *   interpolant and the next step: the mean of Aarseth's criterion as the
 *   4th-order driver evaluates it (a, jerk at both ends, their cubic Hermite
 *   interpolant's 2nd and 3rd derivatives a2, a3 at t1),
 *   sqrt(eta4 (|a||a2| + |j|^2) / (|j||a3| + |a2|^2)), and its 6th-order
 *   generalisation eta6 ((|a||s| + |j|^2) / (|c||q| + |p|^2))^(1/6),
 *   quantised as above (Sec. 3.7 uses eta4 = 0.01, eta6 = 0.1).
 * A new step at the 2^-50 floor stops the run after that block with
 *   SP2_ERR_RANGE (the particles stay at their last times, *stats is filled):
 *   the criterion has collapsed.  Sec. 3.7 warns of this for the 6th-order
 *   criterion on double-single forces, whose noisy jerk and snap enter the
 *   interpolated higher derivatives amplified by h^-3 to h^-5.
 * Errors: SP2_ERR_UNSUPPORTED (order; sp2_block_run on an order-6 context or
 * sp2_block_run_h6 on an order-4 one), SP2_ERR_STATE (nothing loaded, or
 * block_run without block_init after the last sp2_set_j), SP2_ERR_ARG,
 * SP2_ERR_RANGE (step underflow). */
typedef struct {
    int64_t block_steps;   /* force passes taken                          */
    int64_t active_sum;    /* sum of N_active over the passes             */
    int64_t max_active;
    int64_t min_active;
    double t;              /* time of the last block (-1 if none)         */
} sp2_block_stats;
sp2_status sp2_block_init(sp2_ctx *ctx, double t0, double eta_s, double dt_max);
sp2_status sp2_block_run(sp2_ctx *ctx, double t_end, double eta, double dt_max,
                         sp2_block_stats *stats);
sp2_status sp2_block_run_h6(sp2_ctx *ctx, double t_end, double eta4, double eta6, double dt_max,
                            sp2_block_stats *stats);

/* One shared time-step of the 4th-order Hermite scheme (Makino & Aarseth 1992)
 * on device arrays, in place: predict (x, v) with (a, jerk), evaluate acc and
 * jerk there (sp2_forces), correct
 *   v1 = v + (a + a1) dt/2 + (jerk - jerk1) dt^2/12
 *   x1 = x + (v + v1) dt/2 + (a - a1) dt^2/12
 * and leave (x1, v1, a1, jerk1).  Device pointers only. */
sp2_status sp2_hermite4_step(sp2_ctx *ctx, int64_t n, double dt, const double *m,
                             double *x, double *v, double *a, double *jerk);

/* Reverse of sp2_hermite4_step.  x, v, a, jerk hold the step's INPUT state
 * (unchanged).  On entry gx, gv, ga, gj hold the cotangents of the step's
 * outputs; on return the cotangents of its inputs.  gm[n] is accumulated.
 * The predicted state is recomputed.  Device pointers only. */
sp2_status sp2_hermite4_step_vjp(sp2_ctx *ctx, int64_t n, double dt, const double *m,
                                 const double *x, const double *v, const double *a,
                                 const double *jerk, double *gx, double *gv, double *ga,
                                 double *gj, double *gm);

/* Launch-shape control.  sp2_autotune times candidate launch shapes for sink
 * counts n_i on the current predicted records (Sec. 3.1: the block / thread
 * configuration is tuned per GPU) and caches the best for the power-of-two
 * buckets of n_i and of the loaded source count; sp2_get_launch reports what
 * sp2_compute would use for n_i; sp2_set_launch overrides it for those
 * buckets (validated: SP2_ERR_ARG). */
sp2_status sp2_autotune(sp2_ctx *ctx, int64_t n_i, sp2_launch *best);
sp2_status sp2_get_launch(sp2_ctx *ctx, int64_t n_i, sp2_launch *out);
sp2_status sp2_set_launch(sp2_ctx *ctx, int64_t n_i, const sp2_launch *in);

/* CUDA-graph capture of a sequence of calls on the context's stream (device
 * pointers only inside the capture; host-pointer calls return SP2_ERR_STATE).
 * sp2_graph_launch replays the captured calls with the same pointers and
 * arguments. */
sp2_status sp2_graph_begin(sp2_ctx *ctx);
sp2_status sp2_graph_end(sp2_ctx *ctx, sp2_graph **graph);
sp2_status sp2_graph_launch(sp2_ctx *ctx, const sp2_graph *graph);
sp2_status sp2_graph_destroy(sp2_graph *graph);

/* Wait for all work of the context's stream. */
sp2_status sp2_sync(sp2_ctx *ctx);

/* With cfg.profile = 1 every kernel launch of the library is bracketed by CUDA
 * events on the context's stream.  sp2_profile_read waits for the stream and
 * returns, per stage (predict, force, reduce, batched, vjp, other; n_stages
 * entries at most), the number of launches and their summed milliseconds since
 * the last sp2_profile_reset (a stage keeps the last 4096 launches).  Events
 * are not recorded while a graph is being captured. */
sp2_status sp2_profile_reset(sp2_ctx *ctx);
sp2_status sp2_profile_read(sp2_ctx *ctx, int64_t *counts, double *total_ms, int n_stages);

/* Measured pipe rates of the current device (a measurement utility; the
 * paper has none): independent chains of one operation per thread, 8 CTAs of
 * 256 threads per SM, one warm-up and one timed launch each (10-50 ms), on a
 * stream of its own, synchronous.  The rates are operations per second at
 * whatever clock the GPU ran: FP32 FMA lane-operations issued as scalar FFMA
 * and as packed f32x2 FMA (two lane-operations per lane and instruction),
 * FP64 FMAs, and MUFU reciprocal square roots.  The force kernels' FMA-pipe
 * roofline is quoted against the larger FP32 rate.  Errors: SP2_ERR_ARG
 * (null), SP2_ERR_CUDA. */
typedef struct {
    double fp32_fma_lane_ops;
    double fp32x2_fma_lane_ops;
    double fp64_fma_ops;
    double rsqrt_ops;
} sp2_pipe_peaks;
sp2_status sp2_measure_pipe_peaks(sp2_pipe_peaks *out);

/* Number of kernels the library has launched on this context since it opened
 * (memset / memcpy nodes excluded). */
int64_t sp2_kernel_launches(const sp2_ctx *ctx);

/* Loaded j-particle count and capacity. */
sp2_status sp2_info(const sp2_ctx *ctx, int64_t *n_loaded, int64_t *n_max, int *sm_count);

/* Allocation-free block step: predictor + mixed-precision Hermite-4 force pass
 * (+ source-split reduction) on caller-owned device arrays, with no context.
 * The paper has no counterpart; this entry point exists for callers that
 * cannot allocate device memory where they need forces: hosts whose device
 * memory belongs to an allocator or a fixed budget they may not bypass (an
 * integrator embedded in a larger code that hands out all device memory
 * itself), and real-time or signal-driven loops that must not enter the CUDA
 * allocator, which may block or fail under memory pressure.  Its scratch
 * (predicted records, per-slice partial sums, the work-queue counter) is one
 * fixed 16 MiB array inside the library, which every GPU that loads the
 * library keeps until the process exits; the call itself allocates nothing.
 *
 * Inputs (device, n_j <= 65536 sources): id[n_j], m[n_j], x/v/a/jerk[n_j x 3],
 * t_j[n_j]; predicted to t as sp2_predict does in SP2_MIXED (order 4).
 * Sinks: i_idx[n_i] slots in [0, n_j) (n_i <= 65536; an entry outside that
 * range is skipped, and that sink's acc, jerk, pot and nn_r2 are set to NaN and
 * its nn_id to -1, so a bad index is visible without a host read-back).
 * Outputs (device): acc, jerk
 * [n_i x 3], pot[n_i] (required), nn_id[n_i], nn_r2[n_i] (both NULL or both
 * given).  Work is enqueued on cuda_stream (NULL: the legacy default stream);
 * the call returns without waiting.
 *
 * The first call on a device looks the array's address up for that device
 * (cudaGetSymbolAddress, with the device current); make that first call before
 * any stream capture.  Every call shares the array and it keeps the previous
 * call's contents (each call clears the counter and error word it needs): calls whose GPU work
 * overlaps -- on different streams or from different host threads -- race and
 * must be serialised.  Errors: SP2_ERR_RANGE (n_j or n_i above 65536, or the
 * partial sums would not fit), SP2_ERR_ARG (null input, t or eps2 not finite,
 * eps2 < 0), SP2_ERR_STATE (n_j == 0 with sinks), SP2_ERR_CUDA.  n_i == 0 is a
 * successful no-op. */
sp2_status sp2_step_static(int64_t n_j, const int32_t *id, const double *m, const double *x,
                           const double *v, const double *a, const double *jerk, const double *t_j,
                           double t, double eps2, int64_t n_i, const int32_t *i_idx, double *acc,
                           double *jerk_out, double *pot, int32_t *nn_id, double *nn_r2,
                           void *cuda_stream);

const char *sp2_strerror(sp2_status s);
/* Copy the context's last error message (NUL-terminated, truncated to len). */
sp2_status sp2_last_error(const sp2_ctx *ctx, char *buf, size_t len);

#ifdef __cplusplus
}
#endif
#endif /* SAPPORO_GB_H */
