/*
 * burgers.h -- C ABI of libburgers, the B300 (sm_103a) implementation of the
 * 1D viscous Burgers solvers of arXiv 2601.12204:
 *
 *     u_t + u u_x = nu u_xx                                   (Eq. 1)
 *
 * advanced either by the explicit forward-Euler upwind/central step (Eq. 21,
 * upwind side chosen by the sign of u_i as in Sec. 2.2, time step from the CFL
 * limits of Eq. 7-8) or by the implicit BTCS step (Sec. 2.4, Eq. 23) with the
 * convecting velocity lagged from u^n (one Picard linearisation per step),
 * whose tridiagonal system is solved directly under Dirichlet BCs (Eq. 16-17)
 * and through Sherman-Morrison under periodic BCs (Eq. 18).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  * Device pointers are CUDA device addresses of the context's device; the
 *    caller owns them and the stream. Work is enqueued on `stream` (NULL = the
 *    legacy default stream) and the call returns without waiting unless its
 *    comment says "blocking".
 *  * A batch is a packed buffer of `count` independent rows. Row b occupies
 *    elements [inst[b].offset, inst[b].offset + inst[b].n) of the buffer, in
 *    the batch dtype (FP32 or FP64). Rows must not overlap. `inst` is a host
 *    array; it is read during the call only.
 *  * Grid: periodic rows have n distinct nodes (node n is node 0, Eq. 18), so
 *    dx = L/n; Dirichlet rows have n nodes including both ends, dx = L/(n-1),
 *    and u[0], u[n-1] carry the boundary values a, b, which stay fixed.
 *  * r = dt/dx and s = nu*dt/dx^2 are formed in FP64 on the host and rounded
 *    once to the batch dtype.
 *  * Errors: every function returns a status and never aborts or throws.
 *    BURGERS_EINVAL: n < 3, dx <= 0, nu < 0, dt <= 0, nsteps < 0, a NULL
 *    pointer, a bad enum, overlapping rows. BURGERS_ENOMEM: the context
 *    could not grow its workspace. BURGERS_ECUDA: a CUDA call failed (the
 *    message is in burgers_last_error()). The buffers are unchanged on
 *    EINVAL; after ECUDA their contents are unspecified.
 *  * A context owns its workspace, tuning table and graph cache; it is not
 *    thread-safe and its calls must be ordered on one stream at a time.
 */
#ifndef BURGERS_H
#define BURGERS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* burgers_stream; /* identical to cudaStream_t */

typedef enum {
  BURGERS_OK = 0,
  BURGERS_EINVAL = 1,
  BURGERS_ENOMEM = 2,
  BURGERS_ECUDA = 3,
  BURGERS_EAGAIN = 4,    /* serving: request still pending */
  BURGERS_ETIMEOUT = 5,  /* a bounded wait gave up */
  BURGERS_ECANCELED = 6, /* serving: request cancelled */
  BURGERS_ENOTFOUND = 7  /* serving: unknown ticket */
} burgers_status;

typedef enum { BURGERS_F32 = 0, BURGERS_F64 = 1 } burgers_dtype;
typedef enum { BURGERS_PERIODIC = 0, BURGERS_DIRICHLET = 1 } burgers_bc;
typedef enum {
  BURGERS_EXPLICIT = 0, /* forward Euler, Eq. 21 */
  BURGERS_BTCS = 1,     /* lagged upwind BTCS, Eq. 23 */
  BURGERS_RK4 = 2,      /* classical RK4, Eq. 22 */
  BURGERS_CN = 3,       /* Crank-Nicolson, lagged upwind coefficients */
  BURGERS_PICARD = 4,   /* implicit upwind, Picard-iterated */
  BURGERS_NEWTON = 5    /* Newton-Raphson on the residual of Eq. 11 */
} burgers_scheme;

/* One row of a batch (see the conventions above). */
typedef struct {
  int64_t offset; /* first element of the row in the packed buffer */
  int32_t n;      /* nodes, >= 3 */
  int32_t bc;     /* burgers_bc */
  double dx;      /* grid spacing, > 0 */
  double nu;      /* viscosity, >= 0 */
  double dt;      /* time step, > 0 */
  int64_t nsteps; /* steps to advance, >= 0 */
} burgers_instance;

typedef struct {
  int32_t dtype; /* burgers_dtype of the buffers */
  int32_t reserved;
  int64_t count;                /* number of rows */
  const burgers_instance* inst; /* host array of `count` rows */
} burgers_batch;

typedef struct burgers_ctx burgers_ctx;

/* ---- context ------------------------------------------------------------ */

/* Creates a context on CUDA device `device` (made current on the calling
 * thread). Queries the SM count and shared-memory limits used for launch
 * shapes. *out receives the context; destroy it with burgers_ctx_destroy. */
burgers_status burgers_ctx_create(int device, burgers_ctx** out);

/* Synchronises the context's device work and frees everything it owns. */
void burgers_ctx_destroy(burgers_ctx* ctx);

/* Message of the last failure on the calling thread ("" if none). The string
 * stays valid until the next call on this thread. */
const char* burgers_last_error(void);

/* Tunables (see burgers_option). Returns EINVAL for an unknown key or a value
 * out of range. */
typedef enum {
  BURGERS_OPT_GRAPHS = 0,        /* 1: replay multi-launch sequences as CUDA graphs (default 1) */
  BURGERS_OPT_PLAIN = 1,         /* 1: one launch per row per call, no batching (baseline) */
  BURGERS_OPT_STREAM_K = 2,      /* steps per HBM pass of the streaming explicit kernel, 1..64;
                                    0 (default) = the tuning table's entry, else FP32 64
                                    (128 where every streamed row has 262144 nodes or more;
                                    RK4 32), FP64 16 (RK4 4) */
  BURGERS_OPT_RESIDENT_MAX = 3,  /* rows longer than this use the streaming explicit kernel and
                                    the multi-level BTCS solver; 0 = device limit (default 0) */
  BURGERS_OPT_AUTOTUNE = 4,      /* 1: time candidate launch shapes on first use (default 0) */
  BURGERS_OPT_LAUNCH_COUNT = 5,  /* write-only reset of the launch counter (value ignored) */
  BURGERS_OPT_CLUSTER = 6        /* FP32 BTCS, Crank-Nicolson, Picard and Newton rows longer
                                    than one CTA but at most 65536 nodes stay resident in a
                                    thread-block cluster.
                                    1 (default): 128-thread CTAs in clusters of up to 16
                                    where the device can schedule them (non-portable size,
                                    checked with the occupancy API when the context is
                                    created), else up to 8, then 256-thread CTAs up to 8;
                                    2: portable cluster sizes only (<= 8 CTAs);
                                    0: the multi-level solver. Other values: EINVAL.
                                    Ignored while BURGERS_OPT_RESIDENT_MAX is set. */
} burgers_option;
burgers_status burgers_ctx_set(burgers_ctx* ctx, int32_t option, int64_t value);

/* Read-only facts of a context, for burgers_ctx_get. */
typedef enum {
  BURGERS_INFO_SM_COUNT = 100,          /* streaming multiprocessors of the context's device */
  BURGERS_INFO_CLUSTER_CTAS_MAX = 101   /* largest cluster of 128-thread BTCS CTAs the device
                                           schedules (8..16; 16 means rows up to 65536 nodes) */
} burgers_info;

/* Current value of a tunable (any burgers_option but LAUNCH_COUNT) or of a
 * burgers_info key, written to *value. Host only, no device work. EINVAL for
 * a NULL pointer or an unknown key (*value untouched). */
burgers_status burgers_ctx_get(const burgers_ctx* ctx, int32_t key, int64_t* value);

/* Number of kernel launches this context has issued (graph replays count the
 * kernels they contain). */
int64_t burgers_launch_count(const burgers_ctx* ctx);

/* Blocking (synchronises the context's device). The context's device error
 * word: bit 0 is set when a wait inside a kernel gave up (the single-step
 * streaming kernel waits on its bulk copies for at most about two seconds,
 * then stops that CTA's work, so a row's result is then incomplete). *bits
 * receives the word; clear != 0 resets it to 0 afterwards. No paper
 * counterpart: failure reporting of the GPU path. */
burgers_status burgers_device_error(burgers_ctx* ctx, int32_t* bits, int32_t clear);

/* Launch-shape autotuner. Blocking. For every capacity class of the rows of
 * `batch` (rows grouped by the smallest register capacity that holds them)
 * it times each registered kernel shape of that class on a private copy of up
 * to 512 of the caller's rows from u_dev (not modified), each row advanced
 * min(nsteps, probe_steps) steps, and records the fastest shape in the
 * context's table; for explicit rows longer than the resident limit it times
 * the streaming window shapes and steps-per-pass K. Later calls of the
 * advance functions use the table. *tuned (may be NULL) receives the number
 * of classes tuned. */
burgers_status burgers_autotune(burgers_ctx* ctx, int32_t scheme, const burgers_batch* batch,
                                const void* u_dev, int64_t probe_steps, int32_t* tuned,
                                burgers_stream stream);

/* Writes / reads the context's tuning table as text at `path`. Loading checks
 * that every entry names a registered kernel shape (else EINVAL, table
 * unchanged). */
burgers_status burgers_tune_save(const burgers_ctx* ctx, const char* path);
burgers_status burgers_tune_load(burgers_ctx* ctx, const char* path);

/* ---- time step (Eq. 7-8) ------------------------------------------------- */

/* Blocking. For every row b of `batch`, dt_host[b] = cfl * min(dx / max|u|,
 * dx^2 / (2 nu)), the max taken over all n nodes of the row in `u_dev` on the
 * device; the formula is evaluated in FP64 on the device. The rows' dt and
 * nsteps fields are ignored. A row with max|u| == 0 and nu == 0 has no finite
 * limit: dt_host[b] = -1 and the call returns EINVAL after filling the rest. */
burgers_status burgers_cfl_dt(burgers_ctx* ctx, const burgers_batch* batch, const void* u_dev,
                              double cfl, double* dt_host, burgers_stream stream);

/* ---- solvers ------------------------------------------------------------- */

/* Explicit forward-Euler upwind/central solve (Eq. 21, Sec. 2.2). In place:
 * u_dev holds u(0) of every row on entry and u(nsteps*dt) on exit. Each row
 * advances its own nsteps with its own dt. No CFL check is made. */
burgers_status burgers_explicit_advance(burgers_ctx* ctx, const burgers_batch* batch,
                                        void* u_dev, burgers_stream stream);

/* Lagged-coefficient upwind BTCS solve (Sec. 2.4, Eq. 23). In place, as
 * above. Step n solves A(u^n) u^{n+1} = u^n with
 *   l_i = -r a_i^+ - s,  d_i = 1 + r|a_i| + 2s,  c_i = r a_i^- - s,  a = u^n,
 * cyclically (periodic, Sherman-Morrison; the correction denominator in FP64,
 * or for FP32 as a pair of floats from error-free transformations) or with the
 * boundary nodes held (Dirichlet). */
burgers_status burgers_btcs_advance(burgers_ctx* ctx, const burgers_batch* batch,
                                    void* u_dev, burgers_stream stream);

/* Classical fourth-order Runge-Kutta solve (Eq. 22) on the spatial operator
 * of Eq. 21 (upwind side by the sign of u_i, Sec. 2.2): with Delta(w) the
 * forward-Euler increment of burgers_explicit_advance for the state w,
 *   K1 = Delta(u), K2 = Delta(u + K1/2), K3 = Delta(u + K2/2), K4 = Delta(u + K3),
 *   u' = u + (K1 + 2 K2 + 2 K3 + K4)/6.
 * Dirichlet end nodes are held in every stage. In place, layout, ownership and
 * errors as burgers_explicit_advance; no CFL check is made (RK4 is stable for
 * the same CFL-limited dt as forward Euler). */
burgers_status burgers_rk4_advance(burgers_ctx* ctx, const burgers_batch* batch,
                                   void* u_dev, burgers_stream stream);

/* Crank-Nicolson (named as an implicit option in Sec. 2.2) with the
 * convecting velocity lagged at u^n and the upwind side chosen by its sign:
 *   (I - dt/2 L(u^n)) u^{n+1} = (I + dt/2 L(u^n)) u^n,
 * L the upwind/central operator of Eq. 21 (so the rows are those of
 * burgers_btcs_advance with r/2 and s/2). Rows up to the resident capacity
 * (8192 nodes FP32, 4096 FP64) stay in one CTA; longer FP32 rows of up to
 * 65536 nodes stay in the shared memory of a thread-block cluster
 * (BURGERS_OPT_CLUSTER); other rows, of any length, go through the
 * multi-level partitioned solver of the long BTCS rows, with the same rows at
 * its first level. In place, layout, ownership and errors as
 * burgers_btcs_advance. */
burgers_status burgers_cn_advance(burgers_ctx* ctx, const burgers_batch* batch, void* u_dev,
                                  burgers_stream stream);

/* Fully implicit upwind step solved by `iters` Picard iterations per step,
 * A(w) w' = u^n from w = u^n, with A as in burgers_btcs_advance but its
 * coefficients taken from the latest iterate (iters = 1 is the lagged BTCS
 * step). iters in [1, 64], else EINVAL. Long rows as burgers_cn_advance
 * (each iteration one cluster or multi-level solve). */
burgers_status burgers_picard_advance(burgers_ctx* ctx, const burgers_batch* batch, void* u_dev,
                                      int32_t iters, burgers_stream stream);

/* Implicit step with central convection (Eq. 11) solved by `iters`
 * Newton-Raphson iterations per step (Eq. 10-14) from w = u^n:
 *   J(w) dw = -F(w), w += dw,
 *   F_i = w_i - u^n_i + r/2 w_i (w_{i+1} - w_{i-1}) - s (w_{i+1} - 2 w_i + w_{i-1}),
 *   J: sub -r/2 w_i - s, diag 1 + r/2 (w_{i+1} - w_{i-1}) + 2s, super r/2 w_i - s
 * (derived from Eq. 11; Eq. 15 prints only the sub-diagonal, with the sign of
 * its diffusive part garbled). Dirichlet ends held. No pivoting: the Jacobian
 * is strictly diagonally dominant while r max|w| < 1/2 (dt below half the
 * convective CFL limit dx/max|u|); beyond that it may not be, and the solve is
 * then not guaranteed. iters in [1, 64], else EINVAL. Long rows as
 * burgers_cn_advance (each iteration one cluster or multi-level solve). */
burgers_status burgers_newton_advance(burgers_ctx* ctx, const burgers_batch* batch, void* u_dev,
                                      int32_t iters, burgers_stream stream);

/* burgers_explicit_advance for one row, without allocating device memory.
 * The paper has no counterpart: this exists for callers that cannot allocate
 * device memory while they run (an arena that already owns the GPU's memory,
 * a service with a fixed footprint, code called under another allocator's
 * lock). The streaming kernel's working buffers sit in a 16 MiB file-scope
 * device array that every GPU loading this library holds until exit; the
 * caller passes the row. `inst` describes the row (its offset is applied to
 * u_dev); `dtype` is BURGERS_F32 or BURGERS_F64. Limits: 128 <= n <= 1048576
 * (EINVAL beyond, u untouched). Every call looks up the array's device
 * address on the current device; the first call on a device loads the
 * library's module there, so make it before any stream capture. Every call
 * shares the array and leaves its
 * contents behind (each call clears what must start at zero), so calls whose
 * work overlaps on the GPU race and must be serialised by the caller.
 * Asynchronous on `stream`; calls no cudaMalloc or cudaFree. */
burgers_status burgers_explicit_advance_noalloc(const burgers_instance* inst, int32_t dtype,
                                                void* u_dev, burgers_stream stream);

/* End-to-end variant through host memory: copies every row from u_host to a
 * context-owned device buffer, advances it with `scheme` (a burgers_scheme;
 * BURGERS_PICARD and BURGERS_NEWTON with one iteration per step), copies the
 * rows back into u_host. Batches of 64 rows or more are cut into eight chunks
 * of whole rows (in offset order) that are copied in, solved and copied out
 * as a pipeline on the context's copy streams, so transfers overlap the
 * solves. Rows are independent, so the result does not depend on the cut.
 * Blocking. u_host should be page-locked for full copy bandwidth and overlap. */
burgers_status burgers_solve_host(burgers_ctx* ctx, int32_t scheme, const burgers_batch* batch,
                                  void* u_host, burgers_stream stream);

/* ---- adjoints (reverse-mode differentiation, Sec. 2.7.1 / 2.7.3) ---------- */

/* Discrete adjoint of burgers_explicit_advance (scheme = BURGERS_EXPLICIT) or
 * burgers_btcs_advance (BURGERS_BTCS) for every row of `batch`: given
 * gT_dev = dJ/du(T) (batch dtype, row layout of the batch) it writes
 * gu0_dev = dJ/du(0) (same layout; may alias gT_dev) and gnu_dev[b] = dJ/dnu_b
 * (one FP64 device value per row, batch order), holding dt, dx and nsteps
 * fixed. u0_dev holds u(0) and is not modified. At u_i = 0 the derivative of
 * u+ is taken as 0 and that of u- as 1. The forward states are recomputed
 * from checkpoints every `ckpt_stride` steps (0 = ceil(sqrt(nsteps))), with
 * (w ceil(nsteps/stride) + stride + 1) * m values of context-owned workspace
 * per row: w = 2 for FP32 (state and compensation term), 1 for FP64, and m the
 * capacity of the kernel shape that holds the row (the smallest of 32, 128,
 * 512, 1024, 2048 and, FP32 only, 4096 nodes that is >= n). The nu gradient
 * is accumulated in FP64. Explicit rows longer than 4096 (FP32) or 2048 (FP64)
 * nodes take a path that advances one step per pass over tiles: checkpoints
 * every k steps (k = ckpt_stride, else ceil(sqrt(max nsteps)) over those rows)
 * and the k states of a segment in a second context-owned workspace of
 * (ceil(N/k) + k + 6) * span values for FP32 (plus one byte per node for the
 * checkpoints and two state buffers) and (ceil(N/k) + k + 4) * span for FP64,
 * span = the end of the last long row in the batch layout, N the largest
 * step count of those rows; their dJ/dnu is summed per tile in a fixed
 * order. BTCS rows longer than those limits: the forward states come from
 * the library's BTCS path one step per call (checkpoints as above, k + 1
 * states per segment, one more span for the transposed solution), and each
 * reverse step solves A(u^n)^T nu = lambda - A(u^n)^T lambda through the
 * multi-level solver. Asynchronous on `stream`, except that the long-row
 * path waits for its previous call's descriptor upload. */
burgers_status burgers_adjoint(burgers_ctx* ctx, int32_t scheme, const burgers_batch* batch,
                               const void* u0_dev, const void* gT_dev, void* gu0_dev,
                               double* gnu_dev, int64_t ckpt_stride, burgers_stream stream);

/* ---- time step on the device (Eq. 7-8), no host round trip ------------------ */

/* Asynchronous on `stream`: for every row b of `batch`, dt_dev[b] = cfl *
 * min(dx / max|u|, dx^2 / (2 nu)) from the row's current values in `u_dev`,
 * evaluated in FP64 on the device (as burgers_cfl_dt, without the copy to the
 * host and the synchronisation). dt_dev: caller-owned device memory of
 * batch->count doubles. A row with max|u| == 0 and nu == 0 has no finite
 * limit and gets dt_dev[b] = -1. The rows' dt and nsteps are ignored. The
 * reduction's descriptors are built once per batch layout (offsets, n, bc,
 * dx, nu) and kept by the context (at most 16 layouts). Errors as
 * burgers_cfl_dt, except that no row is rejected for its CFL limit. */
burgers_status burgers_cfl_dt_device(burgers_ctx* ctx, const burgers_batch* batch,
                                     const void* u_dev, double cfl, double* dt_dev,
                                     burgers_stream stream);

/* Asynchronous on `stream`: advances every row of `batch` by its nsteps steps
 * of `scheme` (as burgers_explicit_advance ... burgers_newton_advance; iters
 * for BURGERS_PICARD / BURGERS_NEWTON, ignored otherwise) with
 * dt_b = dt_factor * dt_dev[b], read on the device (typically written by
 * burgers_cfl_dt_device on the same stream), so a step sequence "CFL, then
 * advance" needs no host synchronisation. The rows' dt fields are ignored; a
 * row whose dt_dev[b] is not positive is left unchanged. Results are bitwise
 * those of the host-dt entry point with dt = dt_factor * dt_dev[b]. Plans are
 * cached as for the host-dt calls (keyed by the batch without its dt). Rows
 * that need the multi-level solver (FP32 BTCS, CN, Picard and Newton rows
 * longer than the cluster limit, FP64 rows of those schemes longer than the
 * resident capacity): EINVAL. dt_factor <= 0: EINVAL. */
burgers_status burgers_advance_dt_device(burgers_ctx* ctx, int32_t scheme,
                                         const burgers_batch* batch, void* u_dev,
                                         const double* dt_dev, double dt_factor, int32_t iters,
                                         burgers_stream stream);

/* ---- device peak (roofline denominator) ---------------------------------- */

/* Blocking. Measures the FMA issue rate the device sustains for `dtype`
 * (BURGERS_F32 or BURGERS_F64; anything else: EINVAL): every SM runs 2048
 * threads of eight independent register-resident FMA chains, and
 * *lane_fmas_per_s receives lane-FMAs per second at whatever SM clock the GPU
 * runs during the call (the clock is neither set nor locked). Two launches on
 * a stream of its own, the first a warm-up, a few ms each; a small workspace
 * is allocated and freed inside the call. The step kernels are bound by this
 * pipe, so this is the measured denominator of their roofline beside the one
 * derived from SMs x lanes x clock. */
burgers_status burgers_fma_peak(burgers_ctx* ctx, int32_t dtype, double* lane_fmas_per_s);

/* ---- norms (Nomenclature "L2", Sec. 2.7.4) ------------------------------- */

/* Blocking. out_host[b] = ||u_b - ref_b||_2 / ||ref_b||_2 over the n nodes of
 * row b, accumulated in FP64 in a fixed order (deterministic). `u_dev` has the
 * batch dtype, `ref_dev` has dtype `ref_dtype` and the same row offsets.
 * ||ref_b|| == 0 gives 0 if u_b == ref_b, else +inf. If rms_host is not NULL,
 * rms_host[b] = ||u_b - ref_b||_2 / sqrt(n). */
burgers_status burgers_rel_l2(burgers_ctx* ctx, const burgers_batch* batch, const void* u_dev,
                              const void* ref_dev, int32_t ref_dtype, double* out_host,
                              double* rms_host, burgers_stream stream);

/* ---- serving: continuous batching of mixed requests ----------------------- */

/* A server owns a device memory pool and a worker thread. Requests of mixed
 * scheme, BC, n and step count are admitted in arrival order as soon as their
 * state fits the pool (admission by free HBM), advance together in slices of
 * `slice_steps` steps per request (requests arriving meanwhile join at the
 * next slice boundary), and are copied back to the host when done, which
 * frees their slot for the next arrivals. Slice boundaries sit at fixed
 * multiples of slice_steps of each request, so a result does not depend on
 * the other requests in flight. */
typedef struct burgers_server burgers_server;

typedef struct {
  int32_t dtype;          /* burgers_dtype of every request's state */
  int32_t reserved;
  int64_t max_active;     /* cap on concurrently active requests (0 = none) */
  int64_t hbm_budget;     /* device bytes for pool + scratch (0 = half the free HBM) */
  int64_t slice_steps;    /* steps per request per slice (0 = 256) */
  double slice_timeout_s; /* deadline of one slice; exceeded: ETIMEOUT (0 = 60 s) */
} burgers_serve_cfg;

typedef struct {
  int32_t scheme; /* burgers_scheme */
  int32_t bc;     /* burgers_bc */
  int32_t n;      /* nodes, >= 3 */
  int32_t reserved;
  double dx, nu, dt;
  int64_t nsteps;
  const void* u0_host; /* n values of the server dtype, copied during submit */
} burgers_request;

typedef struct {
  double t_submit, t_admit, t_done; /* seconds on the server clock (CLOCK_MONOTONIC since create) */
  int64_t slices;                   /* slices the request took part in */
  int32_t status;                   /* burgers_status of the request */
  int32_t reserved;
} burgers_req_stats;

typedef struct {
  int64_t submitted, completed, slices, active_max, pool_used_max;
  double cell_updates; /* of completed requests */
  int64_t pending, active, pool_bytes, pool_used;
  double now_s;       /* server clock */
  double t_enqueue_s; /* worker time spent planning and enqueuing slices (host) */
  double t_slice_s;   /* worker time waiting for slices to finish on the device */
  double t_copy_s;    /* worker time in admission and result copies */
  double t_gpu_s;     /* device time inside the slices (first to last stamp of each on the
                         worker's stream, read as each slice retires) */
  double t_gpu_gap_s; /* device time between one slice's last stamp and the next one's
                         first: the device idle on the worker's stream */
} burgers_serve_stats;

/* Creates a server on ctx (cfg may be NULL for defaults). The pool is half
 * the budget; a quarter of it holds rows longer than the resident limit, and
 * the context reserves three times that quarter as long-row scratch. The
 * context must outlive the server and must not be used by other threads
 * while the server runs. */
burgers_status burgers_serve_create(burgers_ctx* ctx, const burgers_serve_cfg* cfg,
                                    burgers_server** out);

/* Queues a request; copies u0 before returning. *ticket identifies it.
 * EINVAL for bad fields, ENOMEM if its state can never fit the pool, the
 * server's fault status if the worker has failed. */
burgers_status burgers_serve_submit(burgers_server* sv, const burgers_request* rq,
                                    uint64_t* ticket);

/* Blocking: a client that replays a trace of `count` requests from the
 * calling thread (no interpreter between the requests and the server): request
 * i is submitted as burgers_serve_submit does, once t_arrive[i] seconds have
 * passed since the call began (at once if that time is already past), and
 * late_s[i] receives how late its submission returned against that time, so
 * a caller can measure latency from each request's scheduled arrival.
 * rqs, t_arrive, tickets and late_s are host arrays of `count` elements owned
 * by the caller (u0 of each request is copied during its submission).
 * Stops at the first submission that fails and returns its status; tickets
 * of requests not submitted are 0. count < 0 or a NULL array: EINVAL. */
burgers_status burgers_serve_submit_timed(burgers_server* sv, const burgers_request* rqs,
                                          const double* t_arrive, int64_t count,
                                          uint64_t* tickets, double* late_s);

/* Non-blocking: EAGAIN while the request is pending or running; otherwise
 * copies the result (n values) to out_host (may be NULL), fills *stats (may
 * be NULL), forgets the ticket and returns the request's status (OK,
 * ECANCELED, ETIMEOUT, ECUDA). ENOTFOUND for an unknown ticket. */
burgers_status burgers_serve_poll(burgers_server* sv, uint64_t ticket, void* out_host,
                                  burgers_req_stats* stats);

/* Blocking poll with a timeout in seconds: ETIMEOUT if still unfinished
 * (the request stays queued and can be waited for again). */
burgers_status burgers_serve_wait(burgers_server* sv, uint64_t ticket, double timeout_s,
                                  void* out_host, burgers_req_stats* stats);

/* Blocks until some request has finished (done, cancelled or failed) that
 * this call has not reported before and that poll/wait have not taken yet;
 * writes its ticket (then poll it to take the result). ETIMEOUT if none
 * finishes within timeout_s seconds. */
burgers_status burgers_serve_wait_any(burgers_server* sv, double timeout_s, uint64_t* ticket);

/* Cancels a request: removed from the queue, or from the device at the next
 * slice boundary; its poll then returns ECANCELED. */
burgers_status burgers_serve_cancel(burgers_server* sv, uint64_t ticket);

burgers_status burgers_serve_get_stats(burgers_server* sv, burgers_serve_stats* out);

/* Stops the worker (requests still queued are dropped), frees the pool. */
burgers_status burgers_serve_destroy(burgers_server* sv);

#ifdef __cplusplus
}
#endif
#endif /* BURGERS_H */
