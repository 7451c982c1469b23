/*
 * bsgd.h -- C ABI of the GB300 (sm_103a) BSGD hot path.
 *
 * Block stochastic gradient descent for tomographic reconstruction
 * (Gao, Biguri and Blumensath, arXiv:1903.11874): the on-the-fly Siddon
 * forward projection of a sampled row block, the matched back projection into a
 * sampled column block, the aggregated block gradient step, device-side block
 * sampling (uniform, sub-detector importance sampling, residual-weighted) and
 * the TV proximal step of BSGD-TV.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every call returns a bsgd_status; nothing throws across the ABI. After a
 *    failure bsgd_last_error() returns a message for the calling thread.
 *  - Pointers named "device" must be CUDA device (or managed) memory owned by
 *    the caller; the library never frees them. bsgd_solve() alone also accepts
 *    host pointers and copies them itself.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream). Calls are
 *    asynchronous on that stream unless their comment says they synchronise.
 *  - Kernels run on the calling thread's current CUDA device, which must be
 *    the device the geometry was created on (INVALID_ARG otherwise).
 *  - Volumes are stored [z][y][x] (x fastest), sinograms [view][v][u]
 *    (u fastest). Element types are given by bsgd_dtype.
 *  - The library owns the geometry tables and the solver state behind the
 *    opaque handles below; each has an explicit destroy call.
 *
 * Model (Sec. 1, Eqs. 1-2): y = A x + e, min_x 1/2 ||y - A x||^2, where A_ij >= 0
 * is the length of ray i inside voxel j (Siddon). A is never stored; every FP and
 * BP traces the rays on the fly. Rows are split into M row blocks I_i (whole
 * views), columns into N column blocks J_j (slabs of z planes for volumes, of y
 * rows for 2D images), Sec. 2, Eq. 3.
 */
#ifndef BSGD_H
#define BSGD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BSGD_OK = 0,
    BSGD_ERR_INVALID_ARG = 1, /* bad size, pointer, enum or combination       */
    BSGD_ERR_OOM = 2,         /* device or host allocation failed             */
    BSGD_ERR_CUDA = 3,        /* a CUDA call failed (message has the reason)  */
    BSGD_ERR_TIMEOUT = 4,     /* a bounded wait ran out                       */
    BSGD_ERR_BUDGET = 5,      /* request does not fit the memory budget       */
    BSGD_ERR_STATE = 6        /* call not valid in the object's current state */
} bsgd_status;

typedef enum { BSGD_F32 = 0, BSGD_BF16 = 1, BSGD_F16 = 2 } bsgd_dtype;

typedef enum {
    BSGD_PAR2D = 0,  /* parallel beam, one image slice (nz = nv = 1)          */
    BSGD_FAN2D = 1,  /* fan beam, one image slice (nz = nv = 1)               */
    BSGD_CONE3D = 2  /* circular cone beam                                    */
} bsgd_geom_kind;

/*
 * Scan geometry (the paper fixes none of these conventions; they are the ones
 * the library and its tests share):
 *  - voxel i along an axis with n voxels of size h spans
 *    [-n h / 2 + i h, -n h / 2 + (i + 1) h]; the rotation centre is the origin;
 *  - detector pixel k has centre (k - (n - 1) / 2) * size;
 *  - PAR2D view angle t: rays along (cos t, sin t, 0), detector axis
 *    (-sin t, cos t, 0);
 *  - FAN2D / CONE3D view angle b: source dso (cos b, sin b, 0), detector centre
 *    -(dsd - dso)(cos b, sin b, 0), axes u = (-sin b, cos b, 0), v = (0, 0, 1);
 *    one ray from the source to each pixel centre;
 *  - angles == NULL means a * pi / n_views (PAR2D) or a * 2 pi / n_views;
 *    an angle within 1e-9 rad of a multiple of pi / 2 is taken as that
 *    multiple exactly (axis-aligned directions);
 *  - a ray lying exactly in a voxel face belongs to the voxel on the + side.
 */
typedef struct {
    int kind;                   /* bsgd_geom_kind                                  */
    int nx, ny, nz;             /* voxels                                          */
    double dx, dy, dz;          /* voxel size (mm)                                 */
    int n_views;
    const double *angles;       /* host, n_views radians, or NULL (uniform)        */
    int nu, nv;                 /* detector pixels                                 */
    double du, dv;              /* detector pixel size (mm)                        */
    double dso, dsd;            /* source-origin, source-detector distance (mm)   */
    const int32_t *view_block;  /* host, n_views row-block ids in [0, M), or NULL
                                   for the interleaved partition I_i = {a : a mod M = i} */
} bsgd_geometry_desc;

typedef struct bsgd_geometry bsgd_geometry;
typedef struct bsgd_state bsgd_state;

typedef struct {
    int64_t n_rows;             /* r = n_views * nv * nu                           */
    int64_t n_cols;             /* c = nx * ny * nz                                */
    int M, N;
    int block_axis;             /* 1 (y strips, 2D) or 2 (z slabs, 3D)             */
    int max_views_per_block;
    int64_t max_block_cols;     /* voxels in the largest column block              */
    int64_t compact_rows;       /* rows of the compact per-block sinograms z^j and
                                   r~^j of a solver state: sum over (view, block)
                                   of the block's detector band (<= N * n_rows)    */
} bsgd_geometry_info;

const char *bsgd_last_error(void);
const char *bsgd_status_string(bsgd_status s);

/*
 * Build the ray and block tables of a geometry and upload them to the current
 * CUDA device (Sec. 2, Eq. 3: M row blocks of whole views, N column blocks).
 * Synchronous. *out receives a handle owned by the caller.
 * Errors: INVALID_ARG (sizes <= 0, nz/nv != 1 for 2D kinds, dsd <= dso or a
 * volume that reaches the source for divergent beams, M > n_views, N > planes
 * along the block axis, view_block ids out of range or a block without views),
 * OOM, CUDA.
 */
bsgd_status bsgd_geometry_create(const bsgd_geometry_desc *desc, int M, int N,
                                 bsgd_geometry **out);
bsgd_status bsgd_geometry_destroy(bsgd_geometry *g);
bsgd_status bsgd_geometry_get_info(const bsgd_geometry *g, bsgd_geometry_info *out);

/*
 * Rays the projector traces for the pair (row block i, column block j): the
 * detector band of J_j's shadow (with a one-pixel margin) summed over the views
 * of I_i. Rays outside the band cannot meet J_j (Sec. 2.1: a block projects
 * onto part of the detector only). Host-side; *out is a host int64.
 */
bsgd_status bsgd_geometry_pair_rays(const bsgd_geometry *g, int i, int j, int64_t *out);

/*
 * Forward projection y_S (= or +=) A_S^B x_B  (Sec. 1 after Eq. 2; the summand
 * A_I^J x_J of Sec. 2 and Algorithm 1's FP step).
 *  x: device, batch * n_cols elements of type xt (whole volumes; only the
 *     voxels of the selected column blocks are read).
 *  y: device, batch * n_rows elements of type yt. Rows of the selected row
 *     blocks are written (accumulate = 0) or added to (accumulate = 1); other
 *     rows are untouched.
 *  row_blocks / col_blocks: host arrays of block ids (n_rb / n_cb entries), or
 *     NULL to select every block. Ids must be distinct and in range.
 * Deterministic: each ray sums its segments in traversal order.
 * For volumes, the views whose rays run mostly along x gather from a y-fastest
 * copy of x that the call takes from the library's stream-ordered memory pool
 * (n_cols elements of type xt, returned when the call's work is done); if the
 * pool has no room the call reads x directly (same result, slower).
 * Errors: INVALID_ARG, CUDA (launch failure).
 */
bsgd_status bsgd_forward_project(const bsgd_geometry *g, const void *x, bsgd_dtype xt,
                                 void *y, bsgd_dtype yt,
                                 const int32_t *row_blocks, int n_rb,
                                 const int32_t *col_blocks, int n_cb,
                                 int accumulate, int batch, void *stream);

/*
 * Back projection x_B (= or +=) scale * (A_S^B)^T r_S, the exact transpose of
 * bsgd_forward_project (Algorithm 1's BP step).
 *  r: device, batch * n_rows elements of type rt; rows outside the selected
 *     row blocks are not read.
 *  x: device, batch * n_cols float32 (BSGD_F32 only: the scatter accumulates
 *     with float atomics). With accumulate = 0 the voxels of the selected
 *     column blocks are cleared first; other voxels are untouched.
 * Not bit-reproducible run to run (atomic order); results agree to float
 * rounding. For volumes, the views whose rays run mostly along x scatter into a
 * y-fastest float32 accumulator from the library's memory pool (n_cols floats),
 * added into x after each run of column blocks (x directly if the pool has no
 * room).
 */
bsgd_status bsgd_back_project(const bsgd_geometry *g, const void *r, bsgd_dtype rt,
                              void *x, bsgd_dtype xt,
                              const int32_t *row_blocks, int n_rb,
                              const int32_t *col_blocks, int n_cb,
                              float scale, int accumulate, int batch, void *stream);

/*
 * Number of voxel-ray updates of one FP (or one BP) over the selected blocks:
 * the (ray, voxel) pairs whose segment is longer than 1e-4 of the smallest
 * voxel edge (shorter pieces occur only where a ray passes, up to rounding,
 * through a voxel edge or corner, and vanish in exact arithmetic).
 * Synchronous; *out is a host int64.
 */
bsgd_status bsgd_count_updates(const bsgd_geometry *g,
                               const int32_t *row_blocks, int n_rb,
                               const int32_t *col_blocks, int n_cb,
                               int64_t *out, void *stream);

/*
 * bsgd_count_updates without any memory allocation. The paper has no
 * counterpart: this exists for callers that cannot let a library allocate
 * device memory (a process whose device memory is owned by a caching or
 * pre-reserving allocator, a serving loop that must not block on cudaMalloc /
 * cudaFree, which can synchronise the device). Its per-view counters live in a
 * fixed __device__ array of 16384 + 1 counters (about 128 KiB, held on every
 * GPU that loads the library until the process exits).
 *  - Same arguments, result and threshold as bsgd_count_updates; synchronous.
 *  - Geometries with more than 16384 views are rejected (INVALID_ARG).
 *  - Calls no cudaMalloc / cudaFree and no allocating library routine.
 *  - The first call on a device looks up the array's device address (once per
 *    device) and keeps it for the process's life (a cudaDeviceReset makes it
 *    stale: do not call this entry point again after one).
 *  - Synchronous (it reads the total back into *out): do not call it on a
 *    stream that is being captured into a CUDA graph.
 *  - Every call on a device shares the array (each call clears it first);
 *    calls that overlap on the GPU race and give wrong counts.
 *  - Host side it uses about 4 KiB of the calling thread's stack and no heap.
 *  - INVALID_ARG when the current device is not the geometry's device.
 */
bsgd_status bsgd_count_updates_noalloc(const bsgd_geometry *g,
                                       const int32_t *row_blocks, int n_rb,
                                       const int32_t *col_blocks, int n_cb,
                                       int64_t *out, void *stream);

/*
 * Step-size estimate lambda_J ~ ||A^J||_2^2 of column block j by power
 * iteration: v0 = 1 / sqrt|J| on J, v <- A^T A v / ||A^T A v|| (iters times),
 * lambda = ||A^J v||^2. Vector state, norms and lambda are FP64 on the device;
 * the projections read an FP32 copy of v. Synchronous; *lambda_out is host.
 * rows: every view (row_blocks == NULL) or the listed row blocks.
 */
bsgd_status bsgd_power_iteration(const bsgd_geometry *g, int col_block, int iters,
                                 const int32_t *row_blocks, int n_rb,
                                 double *lambda_out, void *stream);

/*
 * TV proximal step of BSGD-TV (Algorithm 4, Eqs. 9-10):
 *   x <- argmin_t ||t - x||^2 + 2 kappa TV(t),   kappa = mu * lambda,
 * with mu in this library's convention (gradient A^T r, twice the paper's mu):
 * the weight 2 mu lambda is ISTA's proximal step for the objective of
 * Eq. (TVequ), 4 mu lambda in the paper's mu (Algorithm 4 prints half that),
 * isotropic TV from backward differences (a missing neighbour gives 0), solved
 * by `iters` FGP iterations (Beck and Teboulle 2009) in FP32.
 *  x: device, n_cols elements of type xt, updated in place.
 * The library allocates (and frees before returning) its workspace: the image
 * and the primal iterate in FP32 and the dual field and its extrapolation as
 * four floats per voxel (10 * n_cols floats). Synchronises `stream`.
 */
bsgd_status bsgd_tv_prox(const bsgd_geometry *g, void *x, bsgd_dtype xt,
                         double kappa, int iters, void *stream);

/* ------------------------------------------------------------------------ */
/* Solver                                                                   */

typedef enum {
    BSGD_STEP_STRIP = 0, /* mu = rho / max_J ||A^J||^2 (power iteration)          */
    BSGD_STEP_BLOCK = 1, /* mu = rho / max_{i,J} ||A_{I_i}^J||^2                  */
    BSGD_STEP_FIXED = 2  /* mu given                                              */
} bsgd_step_rule;

typedef enum {
    BSGD_PAIRS_UNIFORM = 0,  /* alpha*M row and gamma*N column blocks, uniform   */
    BSGD_PAIRS_RESIDUAL = 1  /* one pair, p(i,j) ~ residual mass on J's band     */
} bsgd_pair_sampling;

typedef enum {
    BSGD_CELLS_NONE = 0,      /* whole views (Algorithm 1)                          */
    BSGD_CELLS_GEOMETRIC = 1, /* one sub-detector per view, p ~ footprint (Alg. 2) */
    BSGD_CELLS_UNIFORM = 2    /* one sub-detector per view, uniform (BSGD-RAN)     */
} bsgd_cell_sampling;

typedef struct {
    double alpha, gamma;     /* fractions of row / column blocks per iteration      */
    int epochs;              /* bsgd_solve: epochs of 1/(alpha*gamma) iterations    */
    int step_rule;           /* bsgd_step_rule                                      */
    double mu;               /* BSGD_STEP_FIXED: the step                            */
    double rho;              /* STRIP / BLOCK: fraction of the Lipschitz step        */
    int power_iters;         /* STRIP / BLOCK power iterations                      */
    int pair_sampling;       /* bsgd_pair_sampling                                  */
    int cells;               /* bsgd_cell_sampling                                  */
    int n_cells;             /* 2 (2D: detector halves) or 4 (3D: quadrants)        */
    double tv_lambda;        /* > 0: BSGD-TV prox every epoch (Algorithm 4), with   */
                             /* kappa = mu * tv_lambda (see bsgd_tv_prox)           */
    int tv_iters;            /* FGP iterations of the prox                          */
    int storage;             /* bsgd_dtype of y, x, z^j, r and snapshots             */
    uint64_t seed;           /* sampling stream (SplitMix64 counter spec)            */
    /* Algorithm 3 (automatic step length), Sec. 3.5: every auto_window epochs
     * (0: M epochs) the effective update direction of the window (the sum of
     * the directions g_J its updates applied) is compared with the previous
     * one, theta = cosine of the two; with the residual norms ||y - sum_j z^j||
     * at the last three window ends r0 (oldest), r1, r2:
     *   r2 < r1 < r0                                     -> mu *= 1 + auto_eps
     *   r2 > r1 > r0 and (theta < auto_t2 or
     *        |theta - previous theta| > auto_t1)          -> mu *= 1 - auto_delta
     * The test runs on the device (no host synchronisation); bsgd_state_query
     * reports the current mu. Not combined with tv_lambda > 0, nor in served
     * requests (INVALID_ARG). Memory: two FP64 images. */
    int auto_mu;             /* 1: on                                                */
    int auto_window;         /* epochs per test (0: M)                               */
    double auto_eps;         /* > 0 (the paper's epsilon)                            */
    double auto_delta;       /* in (0, 1) (the paper's delta; 0.4 in Sec. 5)          */
    double auto_t1, auto_t2; /* cosine thresholds t_1 > 0, t_2 (Algorithm 3)          */
    /* bsgd_solve: run the last final_uniform_epochs epochs without importance
     * sampling (uniform pairs, whole views), as suggested after Algorithm 2 to
     * remove the sampling's bias from the last iterations (0: off). */
    int final_uniform_epochs;
    /* bsgd_solve: 1 = start from x0 = 0 (Algorithm 1's start) whatever x holds
     * on entry, so x is not read (x is then output only); 0 = x holds x0. */
    int zero_start;
    /* BF16 / FP16 storage: 1 = keep the image in the storage type alone (round
     * to nearest at every update and after the TV prox: 2 bytes per voxel, but
     * a step below half an ulp of x is lost); 0 = compensated storage, a
     * low-order 16-bit term beside x (4 bytes per voxel). Ignored for FP32. */
    int image_plain;
} bsgd_solve_params;

typedef struct {
    double residual_norm;    /* ||y - sum_j z^j||_2 in FP64 (the paper's GAP)        */
    double mu;               /* step in the 1/2 ||.||^2 convention                   */
    int64_t iteration;       /* iterations done                                      */
    double epoch;            /* iteration * alpha * gamma                            */
    int64_t updates;         /* voxel-ray updates done (FP + BP)                     */
} bsgd_report;

/*
 * Create solver state for y (device, n_rows elements of type yt, copied into
 * the state's storage type). The state holds z^j and the residual snapshots
 * r~^j for the rows of each block's detector band only (compact_rows each in
 * all; a row outside block j's band has z^j = 0), r, the aggregated gradient g
 * (FP32), FP64 residual-norm
 * tables and the sampler's work list, all in library-owned device memory.
 * Initial state is Algorithm 1's: g = 0, z = 0, r = y, for the starting image
 * x0 = 0; the first bsgd_block_step takes the x it is given as x0 and, when
 * x0 is not zero, sets z^j = A^j x0_J and r = y - sum_j z^j first (see there).
 * Computes mu by power iteration for the STRIP / BLOCK rules; the largest
 * Lipschitz estimate is kept with the geometry (per rule and power_iters), so
 * later states on the same geometry take mu = rho / (that estimate) without
 * iterating again. Synchronous.
 * Memory: the state's arrays come from a stream-ordered pool per device, owned
 * by the library, that keeps up to 32 GiB of freed memory for reuse by later
 * states (so a state per call costs no page mapping once the pool is warm); the
 * update counts and cell weights are computed once per geometry and kept with
 * it (destroy a geometry only after its states).
 * Errors: INVALID_ARG (alpha, gamma outside (0, 1], residual pair sampling with
 * more than one pair per iteration, n_cells not 2 (2D) or 4 (3D) with cells),
 * OOM, CUDA.
 */
bsgd_status bsgd_state_create(const bsgd_geometry *g, const bsgd_solve_params *p,
                              const void *y, bsgd_dtype yt, void *stream,
                              bsgd_state **out);
bsgd_status bsgd_state_destroy(bsgd_state *s);

/*
 * n_iters iterations of BSGD (Algorithm 1; Algorithm 2 with cells; Algorithm 4
 * when tv_lambda > 0): device-side sampling, FP with fused residual update, BP
 * of the residual change into g_J, x_J += mu g_J.
 *  x: device, n_cols elements of the state's storage type, updated in place.
 *     With BF16 / FP16 storage the state also keeps the low-order part of x
 *     (compensated storage, so that steps below half an ulp of x accumulate);
 *     change x only through this call while the state lives.
 * Starting image: the first call on a state (iteration 0, n_iters > 0) takes x
 * as the starting image x0. Algorithm 1 starts from x0 = 0 with z = 0, r = y;
 * for x0 != 0 the call first sets z^j = A^j x0_J for every column block (one
 * FP of x0 over every view), r = y - sum_j z^j, and the residual-norm tables
 * from that r, with r~^j = 0 and g = 0, so that the memories describe x0. A
 * zero x0 is detected on the device and costs one read of x.
 * Asynchronous; no host synchronisation inside.
 */
bsgd_status bsgd_block_step(bsgd_state *s, void *x, int n_iters, void *stream);

/* Progress of the state. Synchronises `stream`. */
bsgd_status bsgd_state_query(bsgd_state *s, bsgd_report *out, void *stream);

/*
 * The state's residual r = y - sum_j z^j (Algorithm 1's r, as the last FP
 * epilogues left it): n_rows elements, [view][v][u], converted from the
 * storage type into out (device, n_rows elements of type ot). Asynchronous.
 */
bsgd_status bsgd_state_read_residual(bsgd_state *s, void *out, bsgd_dtype ot, void *stream);

/*
 * Owner-computes sharding across processes (Sec. 2 and Fig. 1: the nodes hold
 * the column blocks x_J and compute A_I^J x_J; the sums over J that form r_I
 * are collected in one place). Each process (one per GPU) creates a state of
 * the whole problem (same geometry, parameters and y) and marks the column
 * blocks it owns; it then computes the FP, BP and update only for those
 * blocks, keeping x_J, g_J, z^J and r~^J of its own blocks current, and a
 * replicated r. One iteration:
 *   bsgd_shard_begin  draw the pairs (uniform draws, the same on every
 *                     process), FP of the owned drawn pairs into z^J, and
 *                     this process's part sum_{J owned} z^J of the rows whose
 *                     z changed (the bounding box of the drawn blocks' bands
 *                     in every view of the drawn row blocks) into `exchange`;
 *   (caller)          sum `exchange` over all processes (one all-reduce of
 *                     *exchange_len floats, e.g. NCCL or gloo);
 *   bsgd_shard_end    r = y - (the summed buffer) on those rows, the residual
 *                     table, BP of r - r~^J into g_J and x_J += mu g_J for the
 *                     owned drawn blocks.
 * Blocks that no process owns are never updated; a block owned by two
 * processes would be counted twice. x: device, the state's storage type,
 * whole-image layout; only the owned blocks' voxels are read or written, and
 * every process's x must be zero at the start (x0 = 0: the first
 * bsgd_shard_begin checks it on the device, synchronises `stream` and returns
 * INVALID_ARG for a non-zero image). Supported: uniform pairs, whole views or
 * uniform cells; no TV prox, no automatic step, no replay (INVALID_ARG, also
 * from a later bsgd_state_set_sampling or bsgd_state_set_replay); call before
 * the first iteration (STATE otherwise).
 * The report's update count is the whole iteration's on every process.
 * bsgd_state_set_shard: owned_blocks host array of n_owned ids; sets
 *   *exchange_len (floats) for the caller's buffer (device, float32, layout
 *   [drawn row block][view of the block][v][u]). Synchronous.
 * bsgd_shard_begin / _end: asynchronous on `stream` (but for the first
 *   begin's check of x0); the same `exchange` buffer must hold the
 *   all-reduced sum when _end is called.
 */
bsgd_status bsgd_state_set_shard(bsgd_state *s, const int32_t *owned_blocks, int n_owned,
                                 int64_t *exchange_len);
bsgd_status bsgd_shard_begin(bsgd_state *s, void *x, float *exchange, void *stream);
bsgd_status bsgd_shard_end(bsgd_state *s, void *x, const float *exchange, void *stream);

/*
 * Sampling trace. Each iteration occupies bsgd_trace_stride() int32 entries:
 * [n_pairs, i_0, j_0, ..., i_{P-1}, j_{P-1}, then per pair the cell chosen for
 * each view of its row block (-1 when unused)], padded with -1.
 * bsgd_state_read_trace copies the trace of iterations [0, n) (n <= iterations
 * done, n * stride <= cap) to host memory; synchronises `stream`.
 * bsgd_state_set_replay uploads n_iters recorded iterations; the next n_iters
 * iterations consume them instead of sampling. Synchronous.
 */
int64_t bsgd_trace_stride(const bsgd_state *s);
bsgd_status bsgd_state_read_trace(bsgd_state *s, int32_t *host, int64_t cap,
                                  int64_t n_iters, void *stream);
bsgd_status bsgd_state_set_replay(bsgd_state *s, const int32_t *host, int64_t n_iters);

/*
 * Per-stage device timing of bsgd_block_step (tracing). While enabled, every
 * iteration records a CUDA event pair on the launching stream around each of
 * its stages; bsgd_state_read_profile synchronises `stream` and returns, per
 * stage, the number of kernel launches and their summed device time.
 * Enabling resets the counters.
 */
typedef enum {
    BSGD_STAGE_SAMPLE = 0,   /* block / cell sampling                         */
    BSGD_STAGE_FP = 1,       /* forward projection + fused residual update    */
    BSGD_STAGE_RESIDUAL = 2, /* residual recomputation (several J per row)    */
    BSGD_STAGE_BP = 3,       /* back projection of the residual change        */
    BSGD_STAGE_UPDATE = 4,   /* x_J += mu g_J                                 */
    BSGD_STAGE_TV = 5,       /* TV proximal step (BSGD-TV)                    */
    BSGD_STAGE_FPBP = 6,     /* FP, residual and BP in one kernel (1 to 4
                                column blocks per iteration)                  */
    BSGD_N_STAGES = 7
} bsgd_stage;

typedef struct {
    int64_t launches[BSGD_N_STAGES];
    double ms[BSGD_N_STAGES];
} bsgd_profile;

bsgd_status bsgd_state_profile(bsgd_state *s, int enable);
/*
 * Change how the next iterations draw their blocks (Algorithm 1 / 2): pair
 * sampling (bsgd_pair_sampling) and sub-detector cells (bsgd_cell_sampling,
 * n_cells as in bsgd_solve_params). The memory of every (block, cell) is kept,
 * so switching from BSGD-IM to whole views continues the same SAG estimate.
 * Iterations already launched are unaffected. May compute the geometry's
 * tables for the new cell count (synchronises `stream` then).
 * Errors: INVALID_ARG (residual pairs with more than one pair per iteration,
 * bad mode or cell count).
 */
bsgd_status bsgd_state_set_sampling(bsgd_state *s, int pair_sampling, int cells, int n_cells,
                                    void *stream);

/* split = 1: run FP, the residual (with several column blocks per iteration)
 * and BP as separate kernels (to time them apart); default 0: one fused kernel
 * when 1 to 4 column blocks are drawn per iteration (with 2 to 4: uniform
 * pair draws, not a replayed trace), separate kernels otherwise. */
bsgd_status bsgd_state_set_split(bsgd_state *s, int split);
bsgd_status bsgd_state_read_profile(bsgd_state *s, bsgd_profile *out, void *stream);

/*
 * Checkpoint / resume. The paper has no such facility; it follows from the
 * state being (z^j, r~^j, r, the FP64 residual table, g, mu, the iteration
 * counter, the update counter, the 16-bit image's low-order term, Algorithm 3's
 * window state and the sampling trace) and from every draw being a function of
 * (seed, iteration), so a resumed run takes the same draws as an
 * uninterrupted one.
 * bsgd_state_checkpoint_bytes: size of the checkpoint of s.
 * bsgd_state_save: copies it into host memory `host` of `cap` bytes
 *   (cap >= bsgd_state_checkpoint_bytes); synchronises `stream`. y and x are
 *   not part of it: the caller keeps x (as it was at the save) and y.
 * bsgd_state_restore: loads a checkpoint into s, a state created from the same
 *   geometry, parameters and y (a fresh one, or the same one to roll back);
 *   continue with bsgd_block_step and the x of the save. Restores the
 *   sampling mode the saved state ran with (bsgd_state_set_sampling).
 *   Synchronises `stream`. Errors: INVALID_ARG when the blob is not a
 *   checkpoint of a state of this geometry, block counts, pair counts and
 *   storage type, or is truncated.
 */
bsgd_status bsgd_state_checkpoint_bytes(const bsgd_state *s, int64_t *bytes);
bsgd_status bsgd_state_save(bsgd_state *s, void *host, int64_t cap, void *stream);
bsgd_status bsgd_state_restore(bsgd_state *s, const void *host, int64_t bytes, void *stream);

/*
 * One-call reconstruction: state_create, epochs * 1/(alpha*gamma) iterations,
 * query, destroy. y and x may be host or device pointers (host buffers are
 * copied in and out inside the call). x holds the starting image x0 (type xt;
 * zero for Algorithm 1's own start) on entry, unless p->zero_start = 1 (then
 * x0 = 0 and x is not read), and the reconstruction on return; see
 * bsgd_block_step for the start from x0 != 0. Synchronous.
 */
bsgd_status bsgd_solve(const bsgd_geometry *g, const bsgd_solve_params *p,
                       const void *y, bsgd_dtype yt, void *x, bsgd_dtype xt,
                       bsgd_report *out, void *stream);

/* ------------------------------------------------------------------------ */
/* Serving: continuous batching of many reconstructions on one GPU          */
/*
 * The paper's master node feeds sub-blocks to whichever GPU is free (Sec. 2,
 * Fig. 1); here one GPU runs many independent reconstructions at once. A server
 * admits requests of any geometry, size and storage type while their device
 * memory fits a byte budget, keeps each admitted request's state (x, z^j, r,
 * snapshots, sampling tables) resident, and advances all resident requests
 * together: one round = one BSGD iteration of every resident request, launched
 * as a captured CUDA graph of persistent kernels that share the GPU among the
 * requests' rays. Requests that arrive while others run are admitted as slots
 * and budget free up; finished requests leave without stopping the others.
 * Each request's result equals its result alone up to the order of float
 * atomics (its sampling depends only on its own seed and iteration count).
 * Requests may draw up to 4 column blocks per iteration (gamma N <= 4; with
 * more than one, uniform pairs), and use no TV prox and no automatic step;
 * others are rejected at submit.
 */
typedef struct bsgd_server bsgd_server;

/*
 * Round policy. SHARED: every resident request advances one iteration per
 * round (processor sharing). AGE: the resident request submitted first
 * advances every round and the others every second round, so the oldest
 * request gets twice the others' share of the GPU (shorter tail latency for
 * long requests that share the GPU with later, shorter ones). Results do not
 * depend on the policy (a request's draws depend only on its own seed and
 * iteration count).
 */
enum { BSGD_SERVE_SHARED = 0, BSGD_SERVE_AGE = 1 };

typedef struct {
    size_t budget_bytes;      /* device memory the resident requests may hold    */
    int max_slots;            /* resident requests at most (<= 64)               */
    int device;               /* CUDA device                                     */
    int priority;             /* BSGD_SERVE_SHARED or BSGD_SERVE_AGE             */
} bsgd_server_params;

typedef struct {
    int64_t submitted, admitted, completed, failed, queued, resident;
    int peak_resident;
    size_t bytes_resident, peak_bytes;
    double p50_ms, p99_ms, mean_ms, max_ms; /* submit -> result latency, completed requests */
    int64_t updates;          /* voxel-ray updates of completed requests         */
    double busy_s;            /* wall time with at least one request resident    */
    int64_t rounds;
} bsgd_server_stats;

/*
 * Device bytes a request holds while resident (its state, image, geometry
 * tables and the transient set-up buffers), as the admission test counts it.
 * Host-only; no GPU needed.
 */
bsgd_status bsgd_request_bytes(const bsgd_geometry_desc *desc, int M, int N,
                               const bsgd_solve_params *p, size_t *out);

/* Start a server (its scheduler threads, streams and round graph). */
bsgd_status bsgd_server_create(const bsgd_server_params *p, bsgd_server **out);
/* Stop: cancels queued requests, waits (bounded) for resident ones, frees all. */
bsgd_status bsgd_server_destroy(bsgd_server *s);

/*
 * Queue a reconstruction: y (host, n_rows elements of type yt) is copied before
 * the call returns; the result (n_cols float32 values) is written to x_out
 * (host, caller-owned, valid until the request completes or fails).
 * Errors: INVALID_ARG (bad geometry / params, gamma N > 4, TV), BUDGET (the
 * request alone exceeds the budget), STATE (server stopping).
 */
bsgd_status bsgd_server_submit(bsgd_server *s, const bsgd_geometry_desc *desc, int M, int N,
                               const bsgd_solve_params *p, const void *y, bsgd_dtype yt,
                               float *x_out, int64_t *id);
/*
 * Wait up to timeout_ms for request id; TIMEOUT if it is still running. The
 * report carries the iterations, the update count, the step mu the request
 * ran with and its residual norm ||y - sum_j z^j|| at the end (FP64).
 */
bsgd_status bsgd_server_wait(bsgd_server *s, int64_t id, int timeout_ms, bsgd_report *out);
/*
 * Sampling trace of a finished request: the pairs and cells its rounds drew
 * (Algorithm 1's selection step), in the layout of bsgd_state_read_trace with
 * *stride int32 entries per iteration (the first 65536 iterations are kept).
 * With host == NULL only *stride and *n_iters are set; otherwise copies
 * min(n_iters, cap / stride) iterations to host memory and sets *n_iters to
 * that. Lets a caller replay a served request elsewhere (an oracle, a plain
 * state through bsgd_state_set_replay). Errors: INVALID_ARG (unknown id),
 * STATE (the request has not finished, or failed).
 */
bsgd_status bsgd_server_read_trace(bsgd_server *s, int64_t id, int32_t *host, int64_t cap,
                                   int64_t *stride, int64_t *n_iters);
/* *done = 1 if request id finished (successfully or not). */
bsgd_status bsgd_server_poll(bsgd_server *s, int64_t id, int *done);
bsgd_status bsgd_server_get_stats(bsgd_server *s, bsgd_server_stats *out);

#ifdef __cplusplus
}
#endif
#endif /* BSGD_H */
