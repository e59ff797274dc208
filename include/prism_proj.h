/*
 * prism_proj.h -- C ABI of libprism_proj, the batched QP projection of PRISM's
 * sampling-based MPC on one NVIDIA B300 (sm_103a).
 *
 * The operation (paper: Sec. III-A, Eqs. proj_cost, proj_bounds, proj_boundary;
 * Sec. III-D, Eqs. vel_bounds ... jerk_bounds, compact_qp, G_h_def, A_b_def):
 * every sampled joint-velocity sequence xi (one column = one sample n and one
 * joint j, an H-vector) is mapped to
 *
 *     argmin_x 1/2 ||x - xi||^2
 *     s.t.  v_min <= x_k <= v_max                                  k = 1..H
 *           q_min <= q0 + dt * sum_{i<=k} x_i <= q_max             k = 1..H
 *           a_min <= (x_k - x_{k-1}) / dt <= a_max,  x_0 := v0      k = 1..H
 *           j_min <= (x_k - 2 x_{k-1} + x_{k-2}) / dt^2 <= j_max    k = 2..H
 *           x_1 = v0
 *
 * by a fixed number of iterations of the paper's three-step splitting
 * (Eqs. admm_zeta, admm_primal, admm_KKT, admm_dual): a slack clip, a solve with
 * a pre-factorised KKT matrix that depends only on (H, dt, rho) (Sec. III-D
 * "Pre-computable factorization"), and a multiplier update.  The QP separates
 * across joints (Sec. III-D "Joint-wise separability"), so a batch of N samples
 * of J joints is N*J independent H-vector problems sharing one factorisation.
 *
 * Two iterations are offered (PRISM_MODE_*):
 *   ADMM  (default) the three steps with the multiplier kept in constraint
 *         space (one entry per two-sided bound row), so that the slack step sees
 *         it.  Converges to the projection.  The printed iteration does not.
 *   PAPER the iteration exactly as printed (primal-space multiplier lambda,
 *         step factor rho/2 in Eq. admm_dual).  Kept for fidelity comparisons.
 * Row scaling (PRISM_SCALE_*): ROWNORM divides each constraint row by its
 * Euclidean norm (same feasible set; needed for FP32 accuracy), NONE uses the
 * rows as printed.
 *
 * Conventions for every call:
 *   - Every function returns a prism_status and never aborts; on failure
 *     prism_last_error() returns a thread-local description.
 *   - "device" pointers are CUDA device (or managed) memory of the device that
 *     was current when the handle was created; that device must be current on
 *     every call.  The caller owns every buffer it passes in.
 *   - cuda_stream is a cudaStream_t (NULL = legacy default stream).  Solves are
 *     enqueued asynchronously; nothing in prism_proj_solve synchronises the
 *     host.  Outputs are valid once the stream reaches the enqueued work.
 *   - Layouts are the paper's stacking (Sec. III-D): time-major, joint-minor,
 *     row-major [N][H][J] for sequences, [J] for per-joint values, [N][J] for
 *     per-column values.
 *   - Residuals: primal_res[n][j] = max(|x_1 - v0|, max over bound rows r of
 *     max(0, c_r(x) - hi_r, lo_r - c_r(x)) / ||F_r||_2), the bound violation of
 *     the returned x normalised by the row norm of the unscaled operator
 *     (F = [I; dt L; D1/dt; D2/dt^2]); dual_res[n][j] = max_k |x^L_k - x^{L-1}_k|,
 *     the size of the last primal step (0 when iters = 0).
 *   - Initial iterate (the paper does not state one): x^0 = xi with x^0_1 := v0,
 *     multiplier 0.
 */
#ifndef PRISM_PROJ_H
#define PRISM_PROJ_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct prism_proj_s *prism_proj_t;   /* opaque; created and owned by the library */

typedef enum {
    PRISM_OK = 0,
    PRISM_ERR_INVALID_ARG = 1,      /* bad size, pointer, enum or bound ordering      */
    PRISM_ERR_NOT_FACTORED = 2,     /* solve before prism_proj_factor                 */
    PRISM_ERR_RHO_MISMATCH = 3,     /* solve's rho differs from the factored rho      */
    PRISM_ERR_INFEASIBLE_BOUNDS = 4,/* bounds that admit no trajectory                */
    PRISM_ERR_OOM = 5,              /* device or host allocation failed               */
    PRISM_ERR_CUDA = 6,             /* a CUDA runtime call failed (text in last_error) */
    PRISM_ERR_UNSUPPORTED = 7,      /* valid request this build does not implement    */
    PRISM_ERR_TIMEOUT = 8           /* a bounded device-side wait ran out: the results
                                       of that launch are invalid (see
                                       prism_proj_device_status)                      */
} prism_status;

enum { PRISM_MODE_ADMM = 0, PRISM_MODE_PAPER = 1 };
enum { PRISM_SCALE_ROWNORM = 0, PRISM_SCALE_NONE = 1 };
/* K-apply precision: FP32 on the FP32 pipe; TF32X3 on the tensor cores with
 * both operands split into a tf32 high part and a remainder (products of all
 * parts, FP32 accumulation: FP32-level accuracy); TF32 on the tensor cores with
 * the high parts only, except for the last polish_iters iterations
 * (prism_solve_opts), which use the split.  BF16X3 on the tensor cores in
 * bf16 (kind::f16 MMAs): both operands split exactly into three bf16 parts,
 * all products but the one of the two smallest parts, FP32 accumulation
 * (FP32-level accuracy), in either mode, on every solve entry point and in
 * plans (whose autotuner keeps such a group's K-apply). */
enum { PRISM_PREC_FP32 = 0, PRISM_PREC_BF16X3 = 1, PRISM_PREC_TF32 = 2, PRISM_PREC_TF32X3 = 3 };

#define PRISM_MAX_H 132   /* horizon limit of the on-chip solve kernel          */
#define PRISM_MAX_J 64    /* joints per sample handled by one thread block       */

/*
 * prism_proj_create -- a projector for J joints, horizon H, step dt.
 *   Bounds are host arrays of length J (Eqs. vel_bounds, pos_bounds,
 *   acc_bounds, jerk_bounds), copied at create: the caller may free them after
 *   the call.  Requirements: 1 <= J <= PRISM_MAX_J, 2 <= H <= PRISM_MAX_H,
 *   dt > 0 and finite, min <= max for every pair, and a_min <= 0 <= a_max (the
 *   first acceleration row equals (x_1 - v0)/dt = 0 under the equality x_1 = v0,
 *   so a bound excluding 0 makes the set empty: PRISM_ERR_INFEASIBLE_BOUNDS).
 *   On success *out holds a new handle; on failure *out is set to NULL.
 */
prism_status prism_proj_create(int J, int H, double dt,
                               const double *q_min, const double *q_max,
                               const double *v_min, const double *v_max,
                               const double *a_min, const double *a_max,
                               const double *j_min, const double *j_max,
                               prism_proj_t *out);

/*
 * prism_proj_factor -- the one-time per-shape factorisation (Sec. III-D
 * "Pre-computable factorization"; KKT matrix M of Eq. admm_primal).
 *   Builds B = I + c * rho * F^T W F in FP64 on the GPU (c = 1 for ADMM; c = 2
 *   for PAPER, where G^T G = 2 F^T F), Cholesky-factors the block acting on
 *   x_2..x_H, eliminates the equality x_1 = v0, and keeps K = [M^-1]_{1:H,1:H}
 *   and kb = [M^-1]_{1:H,H+1} on the device (FP64, plus an FP32 copy used by
 *   the solve).  rho > 0 is the paper's penalty delta.  prec selects the
 *   K-apply of prism_proj_solve: PRISM_PREC_FP32 (FP32 pipe, any H) or
 *   PRISM_PREC_TF32X3 / PRISM_PREC_TF32 / PRISM_PREC_BF16X3 (tensor cores,
 *   H <= 116; larger H returns PRISM_ERR_UNSUPPORTED).  Enqueued on
 *   cuda_stream; re-factoring a handle replaces its factor (the caller orders
 *   it after solves that still use the old one).
 */
prism_status prism_proj_factor(prism_proj_t h, double rho, int mode, int scale, int prec,
                               void *cuda_stream);

/*
 * prism_proj_solve -- project a batch (the hot path).
 *   batch  N >= 0 samples (N = 0 is a no-op)
 *   q0, v0 device float [J]: theta_init and thetadot_init (Eq. proj_boundary)
 *   samples device float [N][H][J]
 *   iters  >= 0 splitting iterations
 *   rho    must equal the factored rho (else PRISM_ERR_RHO_MISMATCH): the
 *          factorisation depends on it
 *   out    device float [N][H][J]; may alias samples exactly (in place)
 *   primal_res, dual_res device float [N][J], each may be NULL
 *   One persistent launch: each thread block keeps a tile of columns on chip
 *   for all iterations.  Boundary values outside the velocity bounds make the
 *   problem infeasible; they are not detected at enqueue time (they live in
 *   device memory) and show as primal_res >= their violation.
 *   "device" buffers are any memory the device can address: device memory, or
 *   page-locked host memory mapped into the device's address space (its device
 *   address; with unified addressing the host pointer itself).  samples and
 *   out are each read and written exactly once, tile by tile, in address
 *   order, so mapped host buffers stream over the bus while other tiles
 *   iterate (prism_proj_solve_host uses this).
 */
prism_status prism_proj_solve(prism_proj_t h, int batch, const float *q0, const float *v0,
                              const float *samples, int iters, double rho, float *out,
                              float *primal_res, float *dual_res, void *cuda_stream);

/*
 * prism_proj_solve_ex -- prism_proj_solve with a warm start and state export.
 *   opts may be NULL (then identical to prism_proj_solve).  Fields:
 *   x_init    device float [N][H][J] initial iterate, or NULL for x^0 = xi;
 *             x_1 is always reset to v0; must not alias out
 *   dual_init device float [N][D][J] initial multiplier, or NULL for 0
 *   dual_out  device float [N][D][J] multiplier after the last iteration, or NULL
 *   polish_iters  for PRISM_PREC_TF32: how many final iterations use the split
 *             (FP32-accurate) K-apply; ignored for other precisions
 *   init_layout  PRISM_INIT_SAMPLE_MAJOR (0, the layouts above) or
 *             PRISM_INIT_COLUMN_MAJOR (1): x_init [H][N*J] and dual_init
 *             [D][N*J], column n*J + j contiguous (what prism_ws_predict writes
 *             with coalesced stores); dual_out keeps [N][D][J]
 *   D = 4H-1 in ADMM mode: the multiplier of the row-normalised two-sided rows
 *   in the order velocity k=1..H, position k=1..H, acceleration k=1..H, jerk
 *   k=2..H (the scaled ADMM multiplier u of the oracle, same units under
 *   PRISM_SCALE_ROWNORM; under PRISM_SCALE_NONE the printed rows' units);
 *   D = H in PAPER mode: lambda of Eq. admm_dual.
 */
#define PRISM_INIT_SAMPLE_MAJOR 0
#define PRISM_INIT_COLUMN_MAJOR 1

typedef struct {
    const float *x_init;
    const float *dual_init;
    float *dual_out;
    int polish_iters;
    int init_layout;
} prism_solve_opts;

prism_status prism_proj_solve_ex(prism_proj_t h, int batch, const float *q0, const float *v0,
                                 const float *samples, int iters, double rho,
                                 const prism_solve_opts *opts, float *out, float *primal_res,
                                 float *dual_res, void *cuda_stream);

/*
 * prism_proj_sample_solve -- draw the batch on the device and project it: the
 * sampling step of Alg. 1 (xi ~ N(nu, diag(std^2))) fused into the solve, so
 * the samples never travel through HBM as an input.
 *   mean, std  device float [H][J]: nu and the per-entry standard deviation
 *   seed, stream_id  generator key and stream: xi[n][k][j] = mean[k][j] +
 *              std[k][j] * z_e with e = (n*H + k)*J + j; z_e is output e % 4 of
 *              Philox4x32-10 (Salmon et al., SC 2011) at counter (e/4 low, e/4
 *              high, stream_id low, stream_id high), key (seed low, seed high),
 *              through the Box-Muller transform on the word pairs (0,1), (2,3)
 *              with u = (w + 0.5) / 2^32.  Use a new stream_id per draw.
 *   samples_out  device float [N][H][J] receives the drawn xi, or NULL
 *   Other arguments and results as prism_proj_solve.
 */
prism_status prism_proj_sample_solve(prism_proj_t h, int batch, const float *q0, const float *v0,
                                     const float *mean, const float *std, unsigned long long seed,
                                     unsigned long long stream_id, int iters, double rho, float *out,
                                     float *samples_out, float *primal_res, float *dual_res,
                                     void *cuda_stream);

/*
 * prism_proj_solve_plain -- the same projection computed by the plain FP32
 * comparator: one thread per column, the iteration state in a device
 * workspace that the handle allocates on first use (and grows), the cached
 * inverse read from global memory.  Same arguments and results as
 * prism_proj_solve up to FP32 rounding order.  Not for production use.
 */
prism_status prism_proj_solve_plain(prism_proj_t h, int batch, const float *q0, const float *v0,
                                    const float *samples, int iters, double rho, float *out,
                                    float *primal_res, float *dual_res, void *cuda_stream);

/*
 * prism_proj_solve_host -- end-to-end call on HOST buffers (host float
 * arrays, layouts as above).  q0 and v0 are copied to a device staging buffer
 * owned by the handle.  When samples and out are both page-locked and mapped
 * into this device's address space (cudaHostAlloc, pinned torch tensors,
 * cudaHostRegister with cudaHostRegisterMapped), the batch is cut into chunks
 * of whole samples that flow through a pipeline: each chunk is copied in, solved
 * in place in the staging buffer and copied out, on streams of the handle
 * ordered by events, so that one chunk's copies overlap other chunks' solves
 * (prism_proj_set_host_chunks sets the number of chunks); with one chunk the
 * solve reads xi from and writes x into the mapped buffers directly.
 * samples == out is allowed.  Otherwise (pageable memory) samples are copied to
 * the staging buffer, solved in place there and x is copied back.  Each residual
 * array (when not NULL) is written directly if mapped, else copied back.
 * The work is ordered after what cuda_stream holds at the call; the call
 * synchronises cuda_stream before returning; a device-side wait that ran out
 * during the solve returns PRISM_ERR_TIMEOUT.  Host buffers must not be
 * freed or unpinned before the call returns.
 */
prism_status prism_proj_solve_host(prism_proj_t h, int batch, const float *q0_host,
                                   const float *v0_host, const float *samples_host, int iters,
                                   double rho, float *out_host, float *primal_res_host,
                                   float *dual_res_host, void *cuda_stream);

/*
 * prism_proj_shift_state -- receding-horizon shift of a warm start (in place).
 *   For every column, each block of the state moves `steps` entries earlier and
 *   the block's last entry fills the tail: x [N][H][J] (may be NULL) and the
 *   multiplier dual [N][D][J] of prism_proj_solve_ex (may be NULL; ADMM blocks:
 *   velocity H, position H, acceleration H, jerk H-1 rows; PAPER: one block of
 *   H).  The paper shifts its sampling distribution between MPC steps the same
 *   way (Sec. III-B); shifting the multiplier is this library's reading.
 *   steps >= 0; steps >= H leaves every block filled with its last entry.
 */
prism_status prism_proj_shift_state(prism_proj_t h, int batch, int steps, float *x, float *dual,
                                    void *cuda_stream);

/*
 * prism_proj_check_fp64 -- the final feasibility check in FP64 on the GPU:
 * primal_res_fp64[n][j] (device double [N][J]) as defined above, evaluated in
 * double precision from the FP32 trajectories x (device float [N][H][J]).
 */
prism_status prism_proj_check_fp64(prism_proj_t h, int batch, const float *q0, const float *v0,
                                   const float *x, double *primal_res_fp64, void *cuda_stream);

/*
 * prism_proj_get_factor -- copy the FP64 factor to host memory (synchronous):
 *   K_host [H][H] row-major = [M^-1]_{1:H,1:H}, kb_host [H] = [M^-1]_{1:H,H+1}.
 */
prism_status prism_proj_get_factor(prism_proj_t h, double *K_host, double *kb_host);

/*
 * prism_proj_query -- launch facts of the solve kernel for this handle:
 *   out[0] columns per tile, out[1] samples per tile (0: the tiles are runs
 *   of flattened columns n*J + j, as for the ADMM iteration on the tensor
 *   cores, not whole samples), out[2] thread blocks per
 *   SM, out[3] persistent grid size for batch, out[4] dynamic shared memory
 *   bytes per block, out[5] registers per thread, out[6] per-thread horizon
 *   chunk (the kernel variant), out[7] number of SMs.
 */
prism_status prism_proj_query(prism_proj_t h, int batch, long long out[8]);

/*
 * prism_proj_set_tiling -- tile shape of this handle's ADMM solves on the tensor
 * cores (PRISM_MODE_ADMM with PRISM_PREC_TF32X3 or PRISM_PREC_TF32; other
 * handles ignore it).  warps: 0 the library's default; 4 or 8 tiles of 32 or 64
 * columns, four threads per column; 16 tiles of 64 columns with eight threads
 * per column (eight time quarters, every cross-quarter term carried by the
 * MMA; 52 < H <= 104, else PRISM_ERR_UNSUPPORTED).  Results are those of the
 * same iteration up to FP32 rounding order.  Plans choose their own tiling.
 */
prism_status prism_proj_set_tiling(prism_proj_t h, int warps);

/*
 * prism_proj_set_host_chunks -- how prism_proj_solve_host moves page-locked,
 * mapped host buffers (the paper has no counterpart: a transfer schedule).
 *   chunks: 0 the library's choice (chunks of about 0.75 MB of samples, one
 *   chunk below 4 MB); 1 one solve that reads and writes the host buffers
 *   directly; 2..PRISM_HOST_MAX_CHUNKS that many chunks (fewer when the batch
 *   has fewer samples).  Results do not depend on it: every column is solved by
 *   the same kernel with the same arithmetic.  Else PRISM_ERR_INVALID_ARG.
 */
#define PRISM_HOST_MAX_CHUNKS 16
prism_status prism_proj_set_host_chunks(prism_proj_t h, int chunks);

/*
 * prism_proj_solve_plain_noalloc -- prism_proj_solve_plain for callers that
 * must not allocate device memory when they solve.
 *
 * The paper has no counterpart: this is a deployment variant.  Some callers
 * cannot call cudaMalloc at solve time: a real-time controller thread that
 * forbids allocation after start-up (an allocation may block in the driver
 * for an unbounded time), or a host whose device memory is owned by a pool
 * that this library cannot see.  prism_proj_solve_plain grows a per-handle
 * workspace with cudaMalloc on first use; this entry point instead keeps the
 * same workspace in one fixed, file-scope device array of
 * PRISM_NOALLOC_MAX_FLOATS floats (16 MiB) that every GPU which loads the
 * library holds until the process exits.  It calls no cudaMalloc, cudaFree
 * or allocating library routine.
 *
 *   Arguments, layouts and results are those of prism_proj_solve_plain; the
 *   handle must already be factored (create and factor allocate, so callers
 *   do them at start-up).  The workspace needs batch * J * 6 * H floats;
 *   larger requests return PRISM_ERR_INVALID_ARG before anything is enqueued.
 *   The first call on each device looks up the device address of the array
 *   (cudaGetSymbolAddress, with that device current) and caches it; make
 *   that first call before any stream capture begins.
 *   All calls share the one array and it keeps the last call's contents; the
 *   kernel writes every workspace entry it reads, so nothing has to be
 *   cleared, but calls whose work overlaps on the GPU (different streams or
 *   handles, no ordering between them) race on the array.  Order them on one
 *   stream or with events.
 */
#define PRISM_NOALLOC_MAX_FLOATS 4194304
prism_status prism_proj_solve_plain_noalloc(prism_proj_t h, int batch, const float *q0,
                                            const float *v0, const float *samples, int iters,
                                            double rho, float *out, float *primal_res,
                                            float *dual_res, void *cuda_stream);

/*
 * Batched plans -- many independent projection problems of differing
 * (J, H, N, dt, bounds) in one persistent launch per kernel variant.
 *
 * prism_problem describes one problem: a factored handle (its J, H, dt,
 * bounds, mode, rho and precision apply), N = batch samples and device
 * buffers laid out as for prism_proj_solve / prism_proj_solve_ex (residual
 * and warm-start pointers may be NULL).  The caller keeps every buffer alive
 * and in place while the plan exists: the plan stores the pointers.
 *
 * prism_plan_create groups the problems by kernel variant (horizon chunk,
 * mode, K-apply path) and uploads one descriptor table per group; a launch
 * runs one persistent kernel per group, each over every block slot of the
 * GPU, in sequence on the caller's stream.  flags:
 *   PRISM_PLAN_AUTOTUNE  time each group (this runs the solves, overwriting
 *                        the outputs) and, where all of a group's problems are
 *                        FP32-accurate, also the other K-apply path; keep the
 *                        faster path;
 *   PRISM_PLAN_GRAPH     capture the launches once in a CUDA graph;
 *                        prism_plan_launch then replays it.
 * prism_plan_launch enqueues one execution on cuda_stream (asynchronous).
 * prism_plan_query: group < 0 gives out[0] groups, out[1] graph (0/1),
 *   out[2] SMs; group g gives out[0] horizon chunk, out[1] tensor cores (0/1),
 *   out[2] problems, out[3] tiles, out[4] grid, out[5] blocks per SM, out[6]
 *   shared memory bytes, out[7] autotune time in microseconds (-1 if none).
 */
typedef struct {
    prism_proj_t h;
    int batch;
    const float *q0, *v0, *samples;
    float *out, *primal_res, *dual_res;
    const float *x_init, *dual_init;
    float *dual_out;
} prism_problem;

typedef struct prism_plan_s *prism_plan_t;
enum { PRISM_PLAN_AUTOTUNE = 1, PRISM_PLAN_GRAPH = 2 };

prism_status prism_plan_create(const prism_problem *probs, int nprob, int iters, int flags,
                               prism_plan_t *out);
prism_status prism_plan_launch(prism_plan_t plan, void *cuda_stream);
prism_status prism_plan_query(prism_plan_t plan, int group, long long out[8]);
prism_status prism_plan_destroy(prism_plan_t plan);

/*
 * prism_proj_describe -- shape of a handle: dims[0] J, dims[1] H, dims[2] D (multiplier
 * rows per column: 4H-1 ADMM, H PAPER), dims[3] mode, dims[4] precision, dims[5]
 * factored (0/1); *rho (may be NULL) the factored rho.
 */
prism_status prism_proj_describe(prism_proj_t h, int dims[6], double *rho);

/*
 * Serving loop -- continuous batching of projection requests from many MPC
 * controllers (no counterpart in the paper's code; its Sec. III-B MPC loop
 * calls the projection once per control step and warm-starts the next step).
 *
 * prism_server_create: a server on the current device with a device-memory
 *   budget (one arena of mem_budget_bytes, allocated here), at most
 *   max_inflight requests on the GPU at once (one CUDA stream each) and the
 *   control deadline used in the statistics.  A scheduler thread admits queued
 *   requests whenever a stream and arena memory for their buffers are free,
 *   so newly arrived requests start while others are running.
 * prism_server_add_controller: register a factored handle with its batch N and
 *   iteration count; warm_start != 0 keeps the controller's multiplier on the
 *   device between its requests (shifted one step along the horizon before
 *   each new solve).  Admission: the controller's resident state plus one
 *   request's buffers must fit in the remaining budget, else PRISM_ERR_OOM.
 *   Returns the controller id.  Handles must outlive the server.
 * prism_server_submit: queue one request (host arrays: q0, v0 [J], samples
 *   [N][H][J], out [N][H][J], primal [N][J] or NULL).  The host arrays must
 *   stay valid until the request finishes; pinned memory gives asynchronous
 *   copies.  One request per controller runs at a time, in submission order; a
 *   newer request replaces an older one that has not started (the older one is
 *   dropped).  Returns a ticket.
 * prism_server_wait: wait up to timeout_ms (< 0: forever) for a ticket;
 *   *state = 0 queued, 1 running, 2 done, 3 dropped, 4 failed; *latency_ms =
 *   submit-to-completion time (done) or -1.  A finished ticket is forgotten
 *   after it has been waited for.  A failed request returns PRISM_ERR_CUDA
 *   (an enqueue failed) or PRISM_ERR_TIMEOUT (a bounded device-side wait of
 *   its solve ran out, see prism_proj_device_status: its outputs are invalid).
 *   Each request reads and clears its handle's timeout flag on its own stream
 *   after the solve, without a host synchronisation; after a failed request
 *   the controller's next request starts cold (no warm-start multiplier).
 * prism_server_stats: out[0] completed, out[1] dropped, out[2] failed, out[3]
 *   p50 and out[4] p99 latency (ms), out[5] max latency, out[6] deadline misses
 *   (late or dropped), out[7] completed trajectories, out[8] trajectories/s
 *   between the first submission and the last completion, out[9] free arena
 *   bytes.  prism_server_reset_stats clears them.
 * prism_server_destroy: stop the scheduler (queued requests that have not started
 *   are abandoned), finish the work in flight and its completions, free the arena.
 */
typedef struct prism_server_s *prism_server_t;
prism_status prism_server_create(size_t mem_budget_bytes, int max_inflight, double deadline_ms,
                                 prism_server_t *out);
/*
 * prism_server_create_ex -- prism_server_create with flags:
 *   PRISM_SERVER_PLAIN  solve every request with the plain FP32 comparator
 *                       (prism_proj_solve_plain: cold start, no warm-start
 *                       multiplier, one thread per column), under the same
 *                       scheduling, admission and statistics; the comparison
 *                       arm of the serving benchmark.  The comparator's
 *                       per-handle workspace is allocated by a handle's first
 *                       request.
 */
enum { PRISM_SERVER_PLAIN = 1 };
prism_status prism_server_create_ex(size_t mem_budget_bytes, int max_inflight, double deadline_ms, int flags,
                                    prism_server_t *out);
prism_status prism_server_add_controller(prism_server_t s, prism_proj_t h, int batch, int iters,
                                         int warm_start, int *id);
prism_status prism_server_submit(prism_server_t s, int id, const float *q0_host, const float *v0_host,
                                 const float *samples_host, float *out_host, float *primal_host,
                                 unsigned long long *ticket);
prism_status prism_server_wait(prism_server_t s, unsigned long long ticket, double timeout_ms,
                               int *state, double *latency_ms);
prism_status prism_server_stats(prism_server_t s, double out[10]);
prism_status prism_server_reset_stats(prism_server_t s);
prism_status prism_server_destroy(prism_server_t s);

/*
 * Distribution update around the projection (paper Alg. 1, Eqs. weight_update,
 * mean_update_new, cov_update_new): from per-sample costs c [N] and projected
 * trajectories x [N][H][J] (device),
 *   w_n = exp(-c_n / temperature) / sum_m exp(-c_m / temperature)
 *   mean[k][j] = sum_n w_n x[n][k][j]
 *   var[k][j]  = sum_n w_n (x[n][k][j] - mean[k][j])^2 + eps
 * (the diagonal covariance).  mean and var are device [H][J]; weights (device
 * [N], may be NULL) receives w.  The caller passes a device workspace of at
 * least prism_mppi_workspace_bytes(N, H, J) bytes; nothing is allocated.
 * FP32 with a fixed reduction order (deterministic); enqueued on cuda_stream.
 */
size_t prism_mppi_workspace_bytes(int N, int H, int J);
prism_status prism_mppi_update(int N, int H, int J, const float *cost, double temperature, double eps,
                               const float *x, float *mean, float *var, float *weights, void *workspace,
                               size_t workspace_bytes, void *cuda_stream);

/*
 * prism_proj_device_status -- device-side errors of this handle's launches.
 * The tensor-core solve waits for its MMAs with a bounded poll (about a second
 * at most); when a bound runs out, the launch stops early, leaves its outputs
 * invalid and raises a flag in device memory.  This call synchronises
 * cuda_stream, reads and clears that flag and returns PRISM_ERR_TIMEOUT if any
 * launch of the handle since the previous call timed out, else PRISM_OK.  The
 * CUDA context stays usable after a timeout.
 */
prism_status prism_proj_device_status(prism_proj_t h, void *cuda_stream);

/*
 * prism_diag_wait_timeout -- self-test of the bounded device-side wait (the
 * paper has no counterpart).  One block waits on an mbarrier phase that
 * nothing completes, polling at most poll_limit times (1 .. 2^22) with the
 * same routine the tensor-core solve uses; *timed_out receives 1 when the
 * bound ran out (the expected outcome) and 0 if the phase completed.  Runs on
 * the current device's default stream and synchronises it; allocates (and
 * frees) one int of device memory.
 */
prism_status prism_diag_wait_timeout(unsigned int poll_limit, int *timed_out);

/*
 * prism_test_fail_allocs -- host-side fault injection for tests (the paper has
 * no counterpart).  After `skip` more device allocations made by this library,
 * the next `count` of them fail as if the device were out of memory: the call
 * that needed one returns PRISM_ERR_OOM, nothing is allocated for it and the
 * handle or server stays usable (a later call allocates afresh).  (0, 0)
 * switches it off.  Process-wide; not meant for use while other threads call
 * the library.  No device is touched, so no GPU fault is involved.
 */
void prism_test_fail_allocs(int skip, int count);

/*
 * prism_test_set_device_flag -- host-side fault injection for tests (the paper
 * has no counterpart): writes `value` (synchronously, cudaMemset) into the
 * handle's device-side timeout flag, exactly what a solve whose bounded wait
 * ran out leaves behind, so that the reporting paths (device_status,
 * solve_host, the serving loop, plans) can be tested without any device-side
 * fault.  The handle must be factored.
 */
prism_status prism_test_set_device_flag(prism_proj_t h, int value);

/* ------------------------------------------------------------------------
 * Learned warm start of the projection (the neural warm-starting of the
 * projection QP that the paper's conclusion lists as future work; it gives no
 * model, so the model is this library's reading).  Per column c = n*J + j a
 * network with a fixed first layer and a linear skip maps the d = H + 3
 * features
 *   f_k = xi[n][k][j] / vmax_j (k < H),  f_H = v0_j / vmax_j,
 *   f_{H+1} = (q0_j - (qmin_j + qmax_j)/2) / ((qmax_j - qmin_j)/2),  f_{H+2} = 1
 * (bounds of the handle) to phi = [max(0, W1 f + b1) | f] (K2 = hidden + d)
 * and y_hat = phi W2 = [u' | x]: the ADMM-mode multiplier in the units of
 * prism_proj_solve_ex's dual_init (D = 4H - 1 rows) and the trajectory, to be
 * passed as that call's dual_init and x_init.  W2 [K2][D + H] is fitted by
 * ridge regression on converged solves:
 *   (Phi^T Phi / n + lambda I) W2 = Phi^T Y / n   (FP64).
 * The calls on one model are not to run concurrently (accumulate may grow its
 * workspace); separate models are independent.
 * ------------------------------------------------------------------------ */
typedef struct prism_ws_s *prism_ws_t;

/*
 * prism_ws_create -- a warm-start model for a handle factored in ADMM mode
 * (else PRISM_ERR_NOT_FACTORED / PRISM_ERR_INVALID_ARG).  The handle must
 * outlive the model.
 *   hidden  width of the first layer: a multiple of 16 in [0, 128] (0: the
 *           linear model phi = f)
 *   W1_host, b1_host  host double [hidden][H+3] and [hidden], copied (the
 *           caller draws them; may be NULL when hidden = 0)
 *   On success *out holds the model; on failure *out is NULL.  Synchronous.
 */
prism_status prism_ws_create(prism_proj_t h, int hidden, const double *W1_host, const double *b1_host,
                             prism_ws_t *out);

/*
 * prism_ws_accumulate -- add a batch's columns to the fit's sums Phi^T Phi and
 * Phi^T Y (FP64, on the device).
 *   q0, v0    device float [J]; samples device float [N][H][J] (as prism_proj_solve)
 *   x_star    device float [N][H][J]: the converged trajectories of these samples
 *   dual_star device float [N][D][J]: their multiplier, as prism_proj_solve_ex
 *             exports it (dual_out)
 * Enqueued on cuda_stream; the model keeps a design-row workspace of up to
 * 65536 columns x (K2 + D + H) doubles.
 */
prism_status prism_ws_accumulate(prism_ws_t w, int batch, const float *q0, const float *v0, const float *samples,
                                 const float *x_star, const float *dual_star, void *cuda_stream);

/*
 * prism_ws_fit -- solve for W2 with ridge parameter lambda >= 0 (Cholesky in
 * FP64 on the device) and prepare the predictor's operands.  Synchronises
 * cuda_stream.  A matrix that is not positive definite (lambda = 0 with too few
 * or collinear columns) returns PRISM_ERR_INVALID_ARG and leaves no model.
 * The sums stay, so more batches can be added and the model refitted.
 */
prism_status prism_ws_fit(prism_ws_t w, double lambda, void *cuda_stream);

/*
 * prism_ws_predict -- the fitted model on a batch: x_init and dual_init for
 * prism_proj_solve_ex, in layout PRISM_INIT_SAMPLE_MAJOR (device float
 * [N][H][J] and [N][D][J]) or PRISM_INIT_COLUMN_MAJOR ([H][N*J] and [D][N*J],
 * whose stores are whole 128-byte lines; pass the same layout to the solve).
 * Runs on the tensor cores with bf16 operands and FP32 accumulation (the
 * prediction is a starting point, the solve sets the accuracy).  Enqueued on
 * cuda_stream; a bounded device-side wait that ran out raises the handle's
 * timeout flag (prism_proj_device_status).  Before a successful fit:
 * PRISM_ERR_NOT_FACTORED.
 */
prism_status prism_ws_predict(prism_ws_t w, int batch, const float *q0, const float *v0, const float *samples,
                              float *x_init, float *dual_init, int layout, void *cuda_stream);

/*
 * prism_ws_get -- synchronous copies for inspection: S = Phi^T Phi host double
 * [K2][K2], T = Phi^T Y host double [K2][D+H], W2 host double [K2][D+H] (after
 * a fit) and the number of accumulated columns; any pointer may be NULL.
 */
prism_status prism_ws_get(prism_ws_t w, double *S_host, double *T_host, double *W2_host, long long *n_out);

/* prism_ws_reset -- clear the sums (the fitted model stays until the next fit). */
prism_status prism_ws_reset(prism_ws_t w);

/* prism_ws_destroy -- free the model (synchronises the device). */
prism_status prism_ws_destroy(prism_ws_t w);

/* prism_proj_destroy -- free the handle and its device memory (synchronises the device). */
prism_status prism_proj_destroy(prism_proj_t h);

/* Static text of a status code. */
const char *prism_status_string(prism_status s);

/* Thread-local text of the last failure in this thread ("" if none). */
const char *prism_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PRISM_PROJ_H */
