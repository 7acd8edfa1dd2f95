/*
 * jacobi.h -- C ABI of the GB300 over-decomposed Jacobi library.
 *
 * The operation is the Jacobi relaxation of the paper's Jacobi3D proxy
 * application (section 4.3: a fixed number of Jacobi iterations on a 3D
 * domain decomposed into cuboids; every iteration packs the faces of each
 * cuboid, moves them to the neighbours, unpacks them into the halos and then
 * applies the update) with the over-decomposition of section 4.4 (more blocks
 * than processors).  The paper never writes the equation down; this library
 * solves the Poisson problem -Lap(u) = f with Dirichlet values g on a grid of
 * unit spacing with the 5-point (2D) or 7-point (3D) stencil, iterating
 *
 *     x'_p = (sum of the 2d neighbours of p + f_p) / (2d)
 *
 * with the fixed summation order ((W+S)+(E+N))+f in 2D and
 * (((W+D)+(E+U))+(S+N))+f in 3D (W/E, S/N, D/U = -/+ neighbour along x, y, z).
 * The residual is r = b - A x with A the grid negative Laplacian and b = f plus
 * the Dirichlet values of boundary neighbours; the relative residual is
 * ||r||_2 / ||b||_2 (||r||_2 when b = 0).
 *
 * Array conventions (all arguments):
 *   - Fields (x, f) are "interior-dense": nz*ny*nx doubles (2D: ny*nx), x
 *     fastest, no ghost points.
 *   - Boundary faces are ordered -x,+x,-y,+y,-z,+z.  A face lists its points
 *     with the two other axes in order, lowest axis fastest: an x face has
 *     ny*nz values (y fastest), a y face nx*nz (x fastest), a z face nx*ny.
 *     In 2D the x faces have ny values and the y faces nx values.
 *   - Host pointers are copied before the call returns; the caller keeps
 *     ownership.  Device pointers (on_device = 1) must be device memory of the
 *     current device, readable/writable on the library's stream.
 *   - All device state belongs to the library and is released by the destroy
 *     call.  Device memory comes from the allocator registered with
 *     jacobi_set_allocator (cudaMalloc when none).
 *
 * Errors: every call returns a jacobi_status; no C++ exception crosses this
 * boundary and nothing aborts.  jacobi_last_error(ctx) returns a message for
 * the last failure of ctx (or of the calling thread when ctx is NULL).  After
 * JACOBI_ERR_CUDA the context should be destroyed.
 *
 * Threads: one context must not be used by two threads at the same time.
 * Distinct contexts are independent.
 */
#ifndef JACOBI_GB300_H
#define JACOBI_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  JACOBI_OK = 0,
  JACOBI_ERR_INVALID = 1,        /* bad argument or option */
  JACOBI_ERR_OOM = 2,            /* device allocation failed */
  JACOBI_ERR_CUDA = 3,           /* a CUDA call failed */
  JACOBI_ERR_NOT_CONVERGED = 4,  /* solve stopped at max_sweeps above tol */
  JACOBI_ERR_DIVERGED = 5,       /* residual became NaN or infinite */
  JACOBI_ERR_TIMEOUT = 6,        /* a bounded device-side wait ran out */
  JACOBI_ERR_BUSY = 7            /* server: request pending or cannot be admitted */
} jacobi_status;

/* Arithmetic of the iteration (the paper fixes none; FP64 is the plain form).
 *   JACOBI_F64              plain FP64 Jacobi sweeps.
 *   JACOBI_F32_REFINE       iterative refinement: r = b - A x and x += e in
 *                           FP64, inner Jacobi sweeps of A e = r (zero
 *                           boundary, e starting at 0) in FP32.
 *   JACOBI_BF16_REFINE      as F32_REFINE with e stored as bfloat16 (RNE),
 *                           inner sweeps computed in FP32, r stored as FP32.
 *   JACOBI_BF16_REFINE_R16  as BF16_REFINE with r also stored as bfloat16. */
typedef enum {
  JACOBI_F64 = 0,
  JACOBI_F32_REFINE = 1,
  JACOBI_BF16_REFINE = 2,
  JACOBI_BF16_REFINE_R16 = 3
} jacobi_dtype;

typedef enum { JACOBI_BC_ZERO = 0, JACOBI_BC_CONST = 1, JACOBI_BC_FACES = 2 } jacobi_bc_kind;

/* Dirichlet boundary: zero, one constant `value`, or per-face host arrays
 * (faces[i] may be NULL for a zero face). */
typedef struct {
  int kind;               /* jacobi_bc_kind */
  double value;           /* JACOBI_BC_CONST */
  const double* faces[6]; /* JACOBI_BC_FACES, host memory */
} jacobi_boundary;

typedef struct jacobi_ctx* jacobi_t;

/* Allocator hooks: alloc(bytes, cuda_stream, user) returns device memory or
 * NULL; free(ptr, cuda_stream, user).  Pass NULLs to restore cudaMalloc.
 * Affects contexts created afterwards. */
void jacobi_set_allocator(void* (*alloc)(size_t, void*, void*), void (*free_fn)(void*, void*, void*), void* user);

/* Create a solver for one grid (section 4.3's decomposed domain).
 *   ndim      2 or 3.
 *   dims      interior points {nx, ny, nz} (nz ignored in 2D), each >= 1.
 *   block     block extent per axis (section 4.4's over-decomposition),
 *             1 <= block[a] <= dims[a]; blocks that do not divide a dimension
 *             leave a smaller remainder block at the high end.  block = dims
 *             gives the monolithic (single-block) solver.
 *   dtype     jacobi_dtype.
 *   bc        boundary (NULL: zero).
 *   source    host f, interior-dense (NULL: f = 0).
 *   x0        host initial iterate, interior-dense (NULL: 0).
 *   cuda_stream  cudaStream_t all work is issued on (NULL: the legacy default
 *             stream).
 * On success *out holds the context; on failure *out is NULL. */
jacobi_status jacobi_create(jacobi_t* out, int ndim, const int64_t dims[3], const int64_t block[3],
                            int dtype, const jacobi_boundary* bc, const double* source, const double* x0,
                            void* cuda_stream);

/* Run n Jacobi sweeps (section 4.3's fixed-iteration loop), halo exchange
 * included.  In the refinement dtypes: n inner sweeps in outer steps of
 * "refine_period" sweeps, each closed by x += e.  Asynchronous. */
jacobi_status jacobi_sweep(jacobi_t ctx, int64_t n);

/* FP64 residual of the current iterate: *rel = ||b - A x|| / ||b|| (or
 * ||b - A x|| if b = 0), *abs = ||b - A x||.  Either pointer may be NULL.
 * Synchronises the stream. */
jacobi_status jacobi_residual(jacobi_t ctx, double* rel, double* abs);

/* Sweep until the relative residual is <= tol, testing at sweep counts 0,
 * c, 2c, ... (c = option "check_every"; in refinement dtypes every outer step
 * of "refine_period" inner sweeps), at most max_sweeps sweeps.  Returns
 * JACOBI_OK, JACOBI_ERR_NOT_CONVERGED (the field is still valid) or
 * JACOBI_ERR_DIVERGED; for the last two jacobi_last_error(ctx) says after how
 * many sweeps and at which residual it stopped.  *sweeps_done / *final_rel
 * may be NULL. */
jacobi_status jacobi_solve(jacobi_t ctx, double tol, int64_t max_sweeps, int64_t* sweeps_done,
                           double* final_rel);

/* Copy the current iterate out (interior-dense) to host (on_device = 0) or
 * device memory.  Synchronises the stream for host output: the host buffer
 * holds the field when the call returns.  A page-locked host buffer (pinned
 * or registered) is written by the layout kernel directly; other host memory
 * goes through a device staging buffer. */
jacobi_status jacobi_get_field(jacobi_t ctx, double* out, int on_device);

/* Replace the current iterate (interior-dense, host or device memory).  A
 * host buffer may be reused as soon as the call returns (page-locked buffers
 * are read by the layout kernel directly, other host memory through a
 * staging copy). */
jacobi_status jacobi_set_field(jacobi_t ctx, const double* in, int on_device);

/* Replace the source term f (interior-dense, host or device memory). */
jacobi_status jacobi_set_source(jacobi_t ctx, const double* in, int on_device);

/* Integer options (none changes a result bit; they choose how the work runs):
 *   "check_every"    sweeps between residual tests in jacobi_solve (F64), >= 1 (default 50)
 *   "refine_period"  inner sweeps per outer refinement step, 1..4096 (default 20)
 *   "halo"           0 = halo exchange fused into the sweep (default),
 *                    1 = separate pack and unpack kernels after every sweep
 *                    (section 4.3's pack / transfer / unpack steps)
 *   "rows_f64"       lines per warp work item of the FP64 kernels (default 32)
 *   "rows_low"       lines per warp work item of the low-precision kernels; 0
 *                    (default) chooses 16 (float) or 8 (bfloat16) in 2D, 32 in 3D
 *   "schedule"       0 = one launch per sweep (default); 1 = persistent block
 *                    scheduler: one launch runs many sweeps, blocks wait for
 *                    their neighbours' previous sweep, never for a global
 *                    barrier (section 3.1.4's scheduler with section 3.1.2's
 *                    dependencies, on the device).  Needs "halo" = 0.
 *   "graph"          1: every solve step (inner sweeps + outer step, or a
 *                    checked chunk of FP64 sweeps) is captured once as a CUDA
 *                    graph and replayed (section 3.1.3's explicit task graph)
 *   "spin_limit"     iterations a persistent-scheduler wait may spin before it
 *                    gives up with JACOBI_ERR_TIMEOUT (default 2^22)
 *   "poison_wait"    test hook: 1 makes every persistent-scheduler wait run out
 *   "autotune"       1: before the first solve, time the candidate work-item
 *                    shapes and schedules and keep the fastest (cached in the
 *                    file named by the environment variable JACOBI_TUNE_CACHE)
 *   "profile"        1: time every kernel launch with CUDA events (see jacobi_profile)
 *   "march"          1: 2D FP64 sweeps that test no residual run one warp
 *                    over every 64-point segment of a range of lines in turn,
 *                    handing the edge pair of each line to the next segment
 *                    (one FP64 addition per line and segment fewer); the
 *                    ranges are sized so that all of them run in one wave;
 *                    2: the same with four points per lane (128-point
 *                    segments), the next line's loads issued into registers
 *                    before the current line's arithmetic; 3 (default): four
 *                    points per lane with the lines ahead staged in a ring
 *                    of shared-memory buffers by per-lane async copies, and
 *                    the 2D fused-residual sweep and refinement outer step
 *                    also run over march items (ranges of whole residual
 *                    groups); bit-identical to 0; 0: one warp per 64-point
 *                    segment
 *   "emu_adds"       0 (default), 2 or 3: FP64 additions per warp step of the
 *                    FP64 sweep moved to the integer pipe (bit-identical;
 *                    slower on GB300, kept for measurement)
 *   "tma"            1: inner sweeps after the first of a refinement step
 *                    stage the lines they read in shared memory by bulk async
 *                    copies (2D: the warp's line of e and r; 3D: its rows of
 *                    e with the rows above and below, and of r)
 *   "stage3"         1 (default): 3D inner sweeps after the first of a
 *                    refinement step stage the e and r values each lane
 *                    reads, three (float) or four (bfloat16) lines ahead, in
 *                    shared memory by 16-byte async copies that each lane
 *                    reads back itself; 0: one line ahead in registers
 *                    (bit-identical)
 *   "tb"             2: in 2D, with the fused halo and one launch per sweep,
 *                    the inner sweeps run two per launch (temporal blocking:
 *                    one CTA per tile of 32 x 128 points keeps the first
 *                    sweep's values in shared memory, e and r are read and e
 *                    written once per two sweeps); bit-identical to single
 *                    sweeps; 0: one sweep per launch; 1 (default): two per
 *                    launch for FP32 corrections, one for bfloat16 (measured)
 *   "l2pf"           2D FP64 march sweeps: lines brought into L2 by bulk
 *                    prefetches ahead of the loads (0, default: none; 1..64)
 *   "outer_split"    1 (default): in 3D the refinement's outer step runs as
 *                    x_new = x + e over the whole block layout, then the
 *                    residual pass on x_new (fewer FP64 operations per point
 *                    than forming x + e for every neighbour load); 0: one
 *                    fused pass */
jacobi_status jacobi_set_option(jacobi_t ctx, const char* key, int64_t value);
jacobi_status jacobi_get_option(jacobi_t ctx, const char* key, int64_t* value);

/* Kernel timing collected while option "profile" = 1: total milliseconds and
 * number of launches of the kernel class `kernel` ("sweep_f64", "sweep_low",
 * "refine_outer", "reduce", "halo").  Synchronises the stream.  reset = 1
 * clears the counters afterwards.  kernel = "all" reports, in *launches, every
 * kernel launch the context has issued since creation (profiling not needed)
 * and 0 in *total_ms; kernel = "graph" reports the CUDA graph replays. */
jacobi_status jacobi_profile(jacobi_t ctx, const char* kernel, double* total_ms, int64_t* launches, int reset);

/* Bytes of device memory held by the context. */
jacobi_status jacobi_device_bytes(jacobi_t ctx, int64_t* bytes);

/* NULL-safe. */
void jacobi_destroy(jacobi_t ctx);

/* Message of the last failure of ctx (thread-local message when ctx is NULL).
 * The string stays valid until the next call on the same context/thread. */
const char* jacobi_last_error(jacobi_t ctx);

/* Library version: major * 10000 + minor * 100 + patch. */
int jacobi_version(void);

/* ---- batches: many independent grids in every launch -------------------- */

/* One problem of a batch (host memory; see jacobi_create). */
typedef struct {
  int ndim;
  int64_t dims[3];
  int64_t block[3];
  jacobi_boundary bc;
  const double* source; /* NULL: f = 0 */
  const double* x0;     /* NULL: 0 */
} jacobi_problem;

/* Outcome of one problem. */
typedef struct {
  int32_t status;   /* JACOBI_OK, JACOBI_ERR_NOT_CONVERGED or JACOBI_ERR_DIVERGED (server: also
                       JACOBI_ERR_OOM, see jacobi_server_poll) */
  int32_t reserved;
  int64_t sweeps;   /* sweeps (inner sweeps for refinement) at the accepted iterate */
  double rel;       /* relative residual of the returned field */
  double seconds;   /* wall time from the start of the batch solve to this decision */
} jacobi_result;

/* Create one context holding n independent grids of the same ndim (section
 * 4.4's over-decomposition across problems: every block of every grid is a
 * work item of the same launches).  Each grid's arithmetic does not depend on
 * the others: its field and sweep count equal those of solving it alone.
 * Options, jacobi_sweep (all grids), jacobi_profile, jacobi_device_bytes,
 * jacobi_destroy and jacobi_last_error apply to batch contexts; the other
 * single-grid calls return JACOBI_ERR_INVALID on them. */
jacobi_status jacobi_batch_create(jacobi_t* out, int n, const jacobi_problem* probs, int dtype, void* cuda_stream);

/* Solve every grid to its relative residual <= tol (the rule of jacobi_solve,
 * all grids stepping together; a grid retires as soon as it passes).
 * results[i] (may be NULL) receives grid i's outcome.  Returns JACOBI_OK when
 * every grid converged, else the first non-OK status. */
jacobi_status jacobi_batch_solve(jacobi_t ctx, double tol, int64_t max_sweeps, jacobi_result* results);

/* Copy grid i's current iterate out (interior-dense, host or device memory). */
jacobi_status jacobi_batch_get_field(jacobi_t ctx, int i, double* out, int on_device);

/* ---- serving: continuous batching under an HBM budget -------------------- */

typedef struct jacobi_server* jacobi_server_t;

typedef struct {
  /* request counts; rejected: refused at submit, or completed with
   * JACOBI_ERR_OOM at admission */
  int64_t submitted, admitted, completed, rejected;
  int64_t active, queued;                           /* solves on the GPU / waiting now */
  int64_t bytes_in_use, budget_bytes;               /* device memory of the arena */
  int64_t steps;                                    /* refinement steps run */
  double lups;                                      /* lattice-point updates of completed solves */
  int64_t evictions, resumed;                       /* solves evicted to host memory / admitted again */
} jacobi_server_stats;

/* Start a server: one arena of hbm_budget_bytes of device memory (allocated
 * here, through the registered allocator; the paper's custom device pool of
 * section 4.1.2) and a driver thread that owns all GPU work (section 4.1.6's
 * dedicated per-device thread).  dtype is a refinement dtype (1..3);
 * max_slots bounds the solves resident at once per dimensionality.  All
 * solves run refinement steps of "refine_period" inner sweeps (option, set
 * before the first submit; default 20), one launch per sweep, each step
 * replayed from a CUDA graph (options "schedule" = 0, "graph" = 1: measured
 * 1.33x the step rate of the persistent scheduler on a stream of small
 * solves). */
jacobi_status jacobi_server_create(jacobi_server_t* out, int dtype, int64_t hbm_budget_bytes, int max_slots,
                                   void* cuda_stream);

/* Options "refine_period", "schedule", "graph", "halo", "rows_low", "rows_f64"
 * (meaning as for contexts), and eviction under HBM pressure (the paper's
 * memory monitor with offload, section 3.1.1):
 *   "evict"            1: when a queued request has waited "evict_wait_steps"
 *                      driver steps (default 2) for arena room or a slot (the
 *                      oldest such request first), the resident solve that has run longest
 *                      since its admission (at least "evict_min_steps" steps,
 *                      default 20; evicted fewer than "max_evictions" times,
 *                      default 2; at least twice the waiting request's points)
 *                      is moved out: its iterate is copied to host
 *                      memory, its device state freed, and it rejoins the back
 *                      of the queue.  On readmission it continues from that
 *                      iterate; its field and sweep count equal those of a
 *                      solve that was never evicted.  0 (default): off.
 * JACOBI_ERR_BUSY once any request was submitted (the first
 * jacobi_server_submit fixes them). */
jacobi_status jacobi_server_set_option(jacobi_server_t srv, const char* key, int64_t value);

/* Queue one solve to relative residual tol (inputs are copied; thread-safe).
 * The driver admits queued requests in arrival order while their device
 * memory fits in the arena, keeps their state resident, steps every active
 * solve together and retires each as soon as it passes (continuous batching).
 * A solve's result equals the single-grid jacobi_solve with the same
 * refine_period when max_sweeps is a multiple of refine_period.
 * JACOBI_ERR_BUSY: the request can never fit in the budget. */
jacobi_status jacobi_server_submit(jacobi_server_t srv, const jacobi_problem* p, double tol, int64_t max_sweeps,
                                   uint64_t* ticket);

/* JACOBI_OK and the result (and, if field_out is not NULL, the interior-dense
 * field in host memory) when the request is done -- the ticket is then
 * forgotten; JACOBI_ERR_BUSY while it is queued or running.  out->status is
 * the solve's outcome: JACOBI_OK, JACOBI_ERR_NOT_CONVERGED,
 * JACOBI_ERR_DIVERGED, or JACOBI_ERR_OOM when its state did not fit even in
 * the otherwise empty arena (nothing ran; field_out is left untouched; the
 * request counts as rejected in the statistics). */
jacobi_status jacobi_server_poll(jacobi_server_t srv, uint64_t ticket, jacobi_result* out, double* field_out);

/* Block until the ticket is done or timeout_s elapses (JACOBI_ERR_BUSY). */
jacobi_status jacobi_server_wait(jacobi_server_t srv, uint64_t ticket, double timeout_s);

jacobi_status jacobi_server_get_stats(jacobi_server_t srv, jacobi_server_stats* out);

/* Stops the driver thread and frees everything (pending requests are dropped). */
void jacobi_server_destroy(jacobi_server_t srv);

/* Measurement helper (not part of the method): the rate of the FP64 pipe.
 * The plain FP64 sweep is bound by its FP64 additions on GB300 (the FP64 pipe
 * is a small fraction of the FP32 rate), and every such addition is issued as
 * an FMA with multiplier 1.0.  This call times one instruction form:
 *   form 0  fma.rn.f64 with the immediate multiplier 1.0
 *   form 1  fma.rn.f64 with the multiplier 1.0 held in a register
 *   form 2  add.rn.f64
 *   form 3  mul.rn.f64 by a register
 *   form 4  fma.rn.f64 with the multiplier 1.0 read from constant memory
 *   form 5  form 1 with 2 independent 32-bit integer additions per FMA
 *   form 6  form 1 with 4 independent 32-bit integer additions per FMA
 *   (forms 5 and 6 count only the FMAs)
 * in `chains` (1, 2, 4 or 8) independent dependency chains per thread, with
 * ctas_per_sm (1..8) CTAs of 256 threads per SM, each thread issuing
 * 8 * chains * iters operations (iters in [1, 2^24]).  *lane_ops_per_s gets
 * the FP64 lane operations per second over the whole device.  With 8 chains
 * and a full SM it is the pipe's throughput for that form (the peak the FP64
 * sweep is reported against); with one chain it also reflects the
 * dependent-issue latency.  Synchronises the stream; allocates no device
 * memory.  Errors through jacobi_last_error(NULL). */
jacobi_status jacobi_probe_fp64_rate(int form, int chains, int ctas_per_sm, int64_t iters, double* lane_ops_per_s,
                                     void* cuda_stream);

/* Residual of an interior-dense field WITHOUT ANY DEVICE ALLOCATION.
 *
 * The paper has no counterpart to this call; it exists for callers that
 * cannot call cudaMalloc -- a process whose device memory is owned in full by
 * another runtime's pool, or a latency-bound loop that must never stall the
 * device, since cudaMalloc and cudaFree may synchronise it.  It computes
 * *rss_out = sum over the grid of r_p^2 with r = b - A x, the same fused
 * residual and deterministic reduction as jacobi_residual, and its value is
 * bit-identical to that of a monolithic context holding the same field.
 *
 *   ndim, dims  as in jacobi_create.
 *   x           device, interior-dense FP64 field (read).
 *   f           device, interior-dense FP64 source, or NULL for f = 0.
 *   faces       NULL, or 2*ndim device pointers (entries may be NULL for a zero
 *               face) laid out as in jacobi_boundary.
 *   rss_out     device pointer to one double (written).
 *   cuda_stream the stream the two kernels run on (NULL: legacy stream);
 *               the call returns without synchronising.
 *
 * Scratch: one fixed array in device global memory (a file-scope __device__
 * variable of about 8 MiB that every GPU which loads the library keeps until
 * the process exits).  The grid must satisfy ceil(nx / 64) * ceil(ny / 8)
 * <= 2^20 in 2D and ceil(nx / 64) * ny * ceil(nz / 8) <= 2^20 in 3D (16384^2
 * and 512^3 fit); larger grids return JACOBI_ERR_INVALID before any GPU work.
 * The array has one instance per CUDA context that loads the library: the
 * first call in a context (the device's primary context, a context made
 * current through the driver API, or the primary context created again after
 * a device reset) looks up its device address with that context current and
 * keeps it for the context's later calls; make that first call before any
 * stream capture.  Every call shares the array and it keeps the last call's
 * contents (the reduction ticket is cleared by each call before use), so
 * calls that overlap on the GPU (on different streams, or from different
 * threads) race: order them.
 * Errors are reported through jacobi_last_error(NULL). */
jacobi_status jacobi_residual_noalloc(int ndim, const int64_t dims[3], const double* x, const double* f,
                                      const double* const faces[6], double* rss_out, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* JACOBI_GB300_H */
