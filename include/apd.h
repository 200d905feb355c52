/*
 * apd.h -- C ABI of the GB300 (sm_103a) anisotropic power diagram library.
 *
 * An anisotropic power diagram (APD) of seeds x_i in R^D (D = 2 or 3) with
 * symmetric positive-definite anisotropy matrices A_i and weights w_i splits
 * the box Omega = [lo, hi] into cells
 *     L_i = { y : |y - x_i|^2_{A_i} - w_i <= |y - x_k|^2_{A_k} - w_k for all k }
 * (eq. (2.1) of Buze, Feydy, Roper, Sedighiani, Bourne, "Anisotropic power
 * diagrams for polycrystal modelling", arXiv 2403.03571).  The library works
 * on the regular pixel/voxel discretisation of Section 2.3 (eq. (2.6)):
 *     h_d = (hi_d - lo_d) / res_d,   pixel k has centre y_k = lo + (k + 1/2) h,
 *     linear pixel id j = k_0 + res_0 * (k_1 + res_1 * k_2)  (first axis fastest),
 *     J = prod_d res_d pixels of measure |P| = prod_d h_d.
 *
 * Conventions shared by every entry point
 *   - All array arguments are DEVICE pointers owned by the caller, contiguous,
 *     row-major, 8-byte aligned, seed ids 0-based.  The library never frees or
 *     retains them past the call (stream-ordered calls read them on the stream).
 *   - x: double [n][dim]; A: double [n][dim][dim] (symmetric positive definite;
 *     the scoring uses (A + A^T)/2); w: double [n]; v: double [n].
 *   - A workspace (apd_workspace_create) owns all scratch memory; the compute
 *     calls allocate nothing.  One workspace per concurrently used stream.
 *   - Calls marked "stream-ordered" enqueue work on `stream` and return; their
 *     return value covers argument validation and launch errors only.  Errors
 *     found on the device (non-finite input, an A that is not SPD, a wait that
 *     timed out) are latched in the workspace and returned by the next
 *     apd_workspace_status() or host-synchronous call.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).
 *   - Return values are the apd_status codes below.
 */
#ifndef APD_H
#define APD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *apd_stream_t; /* same type as cudaStream_t */

enum apd_status {
    APD_OK = 0,
    APD_NOT_CONVERGED = 1,       /* evaluation cap hit; outputs hold the best iterate */
    APD_WARN_TOL_INFEASIBLE = 2, /* |P| > eps min_i v_i / 2^D (eq. (2.10)); solve still ran */
    APD_ERR_ARG = -1,            /* null pointer, bad size, bad grid, bad volumes, non-finite input */
    APD_ERR_NOT_SPD = -2,        /* some (A_i + A_i^T)/2 is not positive definite */
    APD_ERR_CUDA = -3,           /* a CUDA runtime call or launch failed */
    APD_ERR_WORKSPACE = -4,      /* workspace too small for this call, or wrong dimension */
    APD_ERR_TIMEOUT = -5,        /* a bounded device-side wait ran out; kernel returned early */
    APD_ERR_UNSUPPORTED = -6     /* precision or option not available in this build */
};

/* Regular grid on the box [lo, hi] (eq. (2.6)); entries beyond dim are ignored. */
typedef struct {
    int32_t dim;     /* 2 or 3 */
    int32_t res[3];  /* pixels per axis, >= 1 each; J = prod res < 2^31 */
    double lo[3];
    double hi[3];    /* hi_d > lo_d, finite */
} apd_grid;

/* Generators (X, W, Lambda) of eq. (2.1): n seeds, device pointers. */
typedef struct {
    int32_t n;
    const double *x; /* [n][dim] */
    const double *A; /* [n][dim][dim] */
    const double *w; /* [n] */
} apd_seeds;

/* Arithmetic of the scoring stage (Algorithm 1).  Every precision returns the
 * same labels: a label is kept only when a rigorous rounding bound certifies
 * it, and every other pixel is rescored in FP64 with the reference arithmetic
 * of the cost matrix. */
typedef enum {
    APD_FP32 = 0,    /* CUDA-core FP32 scoring of the expanded quadratic */
    APD_TC_BF16 = 1, /* tcgen05 contraction of the features [y (x) y, y, 1] . phi_i, each FP32
                        feature split into two BF16 operands (hi + lo; three products summed,
                        K = 32), FP32 accumulate: ~1e-4 relative score error */
    APD_TC_TF32 = 2  /* the same with TF32 operands: ~3e-5 relative score error */
} apd_precision;
/* With APD_TC_BF16 / APD_TC_TF32, each seed preparation (the first pass of a
 * call, or of a weight solve) reads the seeds' conditioning back once (a
 * stream synchronisation): when max_i ||A_i||_F / min_i lambda_min(A_i) > 10
 * the certificate and the candidate bounds of the tensor-core form are too
 * loose to pay, and the pass scores with the FP32 kernel instead (same labels).
 * Grids wider than the workspace's tile scratch are scored by the FP32 kernel
 * too. */

typedef struct apd_workspace apd_workspace;

/* Moments layout: per seed K = 1 + dim + dim (dim + 1) / 2 int64 words:
 *   [0]            m_i  = #{ j : H_j = i }
 *   [1 .. dim]     S1_i = sum_{H_j = i} u_j      with u = 2k + 1 (odd pixel coordinates,
 *                                               y = lo + u h / 2)
 *   [dim+1 .. K-1] S2_i = sum_{H_j = i} u_j u_j^T, upper triangle row by row
 *                  (2D: 00 01 11; 3D: 00 01 02 11 12 22). */
#define APD_MOMENT_WIDTH(dim) (1 + (dim) + (dim) * ((dim) + 1) / 2)

/* Allocate device scratch for grids of up to max_j pixels and up to max_n
 * seeds of dimension dim, on the current CUDA device.  *ws receives the handle.
 * Errors: APD_ERR_ARG (null ws, dim not 2/3, max_n < 1, max_j < 1),
 * APD_ERR_CUDA (allocation failed; *ws is set to NULL). */
int apd_workspace_create(apd_workspace **ws, int32_t dim, int32_t max_n, int64_t max_j);

/* Free a workspace (NULL is ignored).  The caller makes sure no work that
 * uses it is still in flight. */
void apd_workspace_destroy(apd_workspace *ws);

/* Seed pruning of the scoring (default off: the dense sweep of Algorithm 1).
 * FP32: each warp skips every 32-seed group (Morton scan order) whose cost
 * lower bound over the warp's pixels,
 *     min lambda_min * dist(pixel box, seed box)^2 - (max w - w_ref),
 * exceeds the largest second-best cost among those pixels.  Tensor cores:
 * each 512-pixel tile scores only the seeds whose lower bound over the tile
 * lies below the fourth smallest upper bound lambda_max maxdist^2 - (w - w_ref);
 * the smallest bound of the seeds left out enters the certificate of every
 * label of the tile.  Either way labels and moments are the same as without
 * pruning.  Applies to every later scoring call on the workspace. */
int apd_workspace_set_pruning(apd_workspace *ws, int32_t enable);

/* Weight solves (Algorithm 2, and every solve inside the Lloyd, coarse-to-fine
 * and refining entry points) replay each evaluation after a solve's first from
 * a CUDA graph captured on first use: trial weights, scoring, rescoring,
 * moments, the dual of eqs. (2.7)-(2.8) and the read-back of its scalars, with
 * only the trial step changing between replays.  Results are the same with and
 * without graphs; a sharded workspace never uses them.  enable = 0 switches
 * them off for this workspace (default on).  Returns APD_ERR_ARG for a null
 * workspace. */
int apd_workspace_set_graphs(apd_workspace *ws, int32_t enable);

/* Incremental evaluations inside weight solves (tensor-core scorers with
 * pruning on, one rank; default on).  The weights enter every cost
 * C_ij = |y_j - x_i|_A^2 - w_i (eq. (2.1)) linearly: between weights w0 and w,
 * C_k - C_a changes by exactly -(D_k - D_a), D = w - w0.  A full pass at w0
 * records, per pixel, its label a, its runner-up b and certified bounds
 * gl <= C_b - C_a <= gu and g3 <= C_k - C_a for every other seed k.  A later
 * pass at w keeps a where min(gl, g3) > max D - min D; where g3 > max D - D_a
 * the label is a or b, decided by the sign of [gl, gu] - (D_b - D_a) (or by
 * the two costs in FP32 when that interval holds 0); the remaining pixels are
 * re-decided in FP32 over their tile's recorded candidate list, and in FP64
 * where that cannot decide.  The moments are the recorded ones plus the
 * changes.  The device chooses each pass's kind from the drift: it records
 * afresh when more than 8 % of the pixels have a recorded g3 within
 * max D - min D.  Labels and moments are the same as with full passes.
 * enable: 0 every pass a full one; 1 (default) incremental passes on grids of
 * at least 2^20 pixels (below that a full pass costs about as much as the
 * incremental pass's extra launches); 2 incremental passes on every grid.
 * Returns APD_ERR_ARG for a null workspace or another enable value. */
int apd_workspace_set_incremental(apd_workspace *ws, int32_t enable);

/* Poll limit of the bounded shared-memory barrier waits of the FP32 scoring
 * kernel on this workspace (each poll sleeps at most ~20 us; default 65536,
 * about 1.3 s).  polls >= 0 sets the limit, polls < 0 restores the default.
 * A wait that runs out latches APD_ERR_TIMEOUT: the kernel then waits, with
 * the default limit, for the copies it has in flight, writes no labels or
 * moments and returns; apd_workspace_status reports the status.  A limit of 0
 * gives up at the first wait: that is how the timeout path is tested without
 * a hung kernel.  Errors: APD_ERR_ARG (null ws, polls >= 2^32). */
int apd_workspace_set_wait_limit(apd_workspace *ws, int64_t polls);

/* ---- Slabs and sharded evaluation ------------------------------------------
 * The per-cell sums of eq. (2.7) are the only data that couple pixels: the
 * moments of disjoint sets of pixels add up to those of their union.  So one
 * APD can be split across ranks (processes, one GPU each) by contiguous slabs
 * of the grid's last (slowest) axis; every rank holds all n seeds, scores its
 * slab, and one sum-reduction of the n x APD_MOMENT_WIDTH(dim) int64 words per
 * evaluation gives every rank the full moments.  The dual, the gradient and
 * L-BFGS then run identically on every rank, and because the moments are
 * integers the result is bit-for-bit independent of the split and of the
 * order of the reduction. */

/* The slab of rank `rank` out of `world` along an axis of `res` pixels:
 * k_begin = floor(res rank / world), k_count = floor(res (rank + 1) / world) -
 * k_begin (empty slabs when world > res).  Host only, no device use.
 * Errors: APD_ERR_ARG (res < 1, world < 1, rank outside [0, world), null out). */
int apd_shard_range(int32_t res, int32_t rank, int32_t world, int32_t *k_begin, int32_t *k_count);

/* Algorithm 1 + moments over the slab of pixels whose last-axis index lies in
 * [k_begin, k_begin + k_count) of `grid` (2D: k_1, 3D: k_2).  moments: int64
 * device [n][APD_MOMENT_WIDTH(dim)], overwritten, in the full grid's
 * coordinates (u = 2k + 1 of the full-grid indices), so summing the slabs of
 * a partition of the axis gives apd_cell_moments of the whole grid exactly.
 * The workspace must hold the slab's pixels (max_j >= its pixel count).
 * Stream-ordered.  Errors as apd_cell_moments, plus APD_ERR_ARG for k_begin
 * < 0, k_count < 1 or k_begin + k_count > res of the last axis. */
int apd_cell_moments_slab(const apd_grid *grid, int32_t k_begin, int32_t k_count, const apd_seeds *seeds,
                          apd_precision precision, int64_t *moments, apd_workspace *ws, apd_stream_t stream);

/* Reduction hook of a sharded workspace.  Called on the host, once per
 * evaluation, after the moments of this rank's slab have been enqueued on
 * `stream` into `moments` (device, `words` int64 values) for the generators
 * `seeds` of that evaluation (device pointers: the positions, matrices and
 * trial weights it scored); it must leave in `moments`, ordered before any
 * later work on `stream`, the elementwise sum of every rank's moments (an
 * allreduce SUM of int64, e.g. NCCL's).  Return 0 on success; anything else
 * aborts the call with APD_ERR_CUDA. */
typedef int (*apd_reduce_fn)(void *ctx, int64_t *moments, int64_t words, const apd_seeds *seeds,
                             apd_stream_t stream);

/* Make every later scoring pass on this workspace cover only rank `rank`'s
 * slab (apd_shard_range of the grid's last axis, for each grid the call uses:
 * a coarse-to-fine solve shards both grids), followed by fn(ctx, ...) on the
 * moments.  All entry points that evaluate the dual or the moments (moments,
 * dual, weight solves, Lloyd steps, coarse-to-fine and warm-started solves)
 * then return the full-grid results on every rank, provided every rank makes
 * the same calls with the same arguments; apd_assign writes the labels of the
 * slab's pixels only; the masked calls return APD_ERR_UNSUPPORTED, and the
 * non-uniform (points) calls and batches are not sharded.  world == 1 (fn ignored) restores whole-grid passes.
 * Errors: APD_ERR_ARG (null ws, world < 1, rank outside [0, world), world > 1
 * with null fn). */
int apd_workspace_set_shard(apd_workspace *ws, int32_t rank, int32_t world, apd_reduce_fn fn, void *ctx);

/* Synchronise `stream`, return and clear the device-side status latched by the
 * stream-ordered calls (APD_OK, APD_ERR_ARG, APD_ERR_NOT_SPD, APD_ERR_TIMEOUT),
 * or APD_ERR_CUDA if the synchronisation itself failed. */
int apd_workspace_status(apd_workspace *ws, apd_stream_t stream);

/* Per-evaluation counters of the last scoring pass on this workspace
 * (host-synchronous: synchronises `stream`).  rescored_fp64 = pixels whose FP32
 * best/second-best gap was inside the rounding bound and were rescored in FP64. */
typedef struct {
    int64_t pixels;
    int64_t pairs;          /* pixels * n */
    int64_t rescored_fp64;
} apd_eval_stats;
int apd_last_stats(apd_workspace *ws, apd_eval_stats *out, apd_stream_t stream);

/* Algorithm 1 (pixel method): labels[j] = H_j = argmin_i C_ij with
 * C_ij = |y_j - x_i|^2_{A_i} - w_i; the lowest index wins exact ties.
 * labels: int32 device [J].
 * tie_gap: double device [J] or NULL.  When given, tie_gap[j] receives the
 *   relative gap between the two smallest costs at pixel j,
 *     (C_(2) - C_(1)) / (|q_(1)| + |q_(2)| + |w_(1)| + |w_(2)|),
 *   C_(1) <= C_(2) ordered by cost then seed index (an exact tie gives 0),
 *   q = |y_j - x|^2_A the quadratic part of each, +inf when n == 1.  Both
 *   costs are computed with the FP64 reference arithmetic (d = y - x; q summed
 *   a outer, b inner, each product (d_a A_ab) d_b rounded; C = q - w), so the
 *   gap is that of a full FP64 evaluation of Algorithm 1.  A label decided by
 *   rounding alone has gap ~1e-16; this is the band in which parity with
 *   another FP64 evaluation can differ.  Costs one more pass over the pixels.
 * Stream-ordered.
 * Errors: APD_ERR_ARG, APD_ERR_WORKSPACE, APD_ERR_UNSUPPORTED, APD_ERR_CUDA. */
int apd_assign(const apd_grid *grid, const apd_seeds *seeds, apd_precision precision,
               int32_t *labels, double *tie_gap, apd_workspace *ws, apd_stream_t stream);

/* Algorithm 1 fused with the per-cell reduction: moments int64 device
 * [n][APD_MOMENT_WIDTH(dim)] (layout above), exact integers, overwritten.
 * Stream-ordered.  Errors as apd_assign. */
int apd_cell_moments(const apd_grid *grid, const apd_seeds *seeds, apd_precision precision,
                     int64_t *moments, apd_workspace *ws, apd_stream_t stream);

/* Discrete dual of eq. (2.7) and its approximate gradient eq. (2.8):
 *   g~(W)   = sum_i ((v_i - m_i |P|) w_i + sum_{H_j=i} |P| |y_j - x_i|^2_{A_i})
 *   grad_i  = v_i - m_i |P|
 *   max_rel_err = max_i |grad_i| / v_i      (stop quantity of Algorithm 2)
 * g, max_rel_err: double device [1]; grad: double device [n] (may be NULL).
 * v: target volumes, v_i > 0.  Stream-ordered. */
int apd_dual_value_grad(const apd_grid *grid, const apd_seeds *seeds, const double *v,
                        apd_precision precision, double *g, double *grad, double *max_rel_err,
                        apd_workspace *ws, apd_stream_t stream);

/* Options of the weight solve (Algorithm 2) and the Lloyd loop (Algorithm 3). */
typedef struct {
    double eps;              /* relative volume tolerance, stop when max_i |v_i - m_i|P||/v_i < eps */
    int32_t max_evals;       /* cap on dual evaluations per solve */
    int32_t history;         /* L-BFGS memory (1..32) */
    apd_precision precision; /* scoring arithmetic */
    int32_t check_volumes;   /* nonzero: reject v unless v_i > 0 and |sum v - |Omega|| <= 1e-9 |Omega| */
} apd_solve_opts;

/* Fill *opts with the defaults: eps 0.01, max_evals 1000, history 10, APD_FP32, check_volumes 1. */
void apd_solve_opts_default(apd_solve_opts *opts);

typedef struct {
    int32_t status;        /* final status of the call */
    int32_t iterations;    /* accepted L-BFGS steps (summed over solves for apd_lloyd) */
    int32_t evaluations;   /* dual evaluations */
    int32_t solves;        /* Algorithm 2 runs */
    double max_rel_err;    /* at the returned weights */
    double g;              /* g~ at the returned weights */
    int64_t rescored_fp64; /* pixels rescored in FP64, summed over evaluations */
    double seconds;        /* wall time of the call */
    int32_t coarse_evaluations; /* evaluations on the coarse grid (coarse-to-fine solves; else 0) */
    int32_t pad;
} apd_solve_info;

/* Algorithm 2: maximise g~ by L-BFGS from W0 = seeds->w until
 * max_i |v_i - m_i |P|| / v_i < eps.  w_out: double device [n] (may alias
 * seeds->w).  info: host pointer (may be NULL).  Host-synchronous: returns
 * APD_OK, APD_NOT_CONVERGED (w_out = best iterate), APD_WARN_TOL_INFEASIBLE
 * (converged although eq. (2.10) fails for this grid) or an error. */
int apd_solve_weights(const apd_grid *grid, const apd_seeds *seeds, const double *v,
                      double *w_out, const apd_solve_opts *opts, apd_solve_info *info,
                      apd_workspace *ws, apd_stream_t stream);

/* One round of Algorithm 3: solve the weights from W0 = seeds->w at X = seeds->x,
 * then move every seed to the discrete centroid of its cell
 *   x_i <- sum_{H_j=i} |P| y_j / (m_i |P|)   (empty cells keep x_i),
 * writing x_out [n][dim] and w_out [n] (the solved weights, the warm start of
 * the next round).  x_out may alias seeds->x.  Host-synchronous; status as
 * apd_solve_weights. */
int apd_lloyd_step(const apd_grid *grid, const apd_seeds *seeds, const double *v,
                   double *x_out, double *w_out, const apd_solve_opts *opts,
                   apd_solve_info *info, apd_workspace *ws, apd_stream_t stream);

/* Algorithm 3 in full: `rounds` calls of apd_lloyd_step followed by a final
 * apd_solve_weights, from X0 = seeds->x and W0 = seeds->w.  Host-synchronous. */
int apd_lloyd(const apd_grid *grid, const apd_seeds *seeds, const double *v, int32_t rounds,
              double *x_out, double *w_out, const apd_solve_opts *opts, apd_solve_info *info,
              apd_workspace *ws, apd_stream_t stream);

/* Kernel timing for benchmarks: when enabled, the library records a CUDA event
 * pair on the caller's stream around every launch of the scoring kernel
 * (Algorithm 1 fused with the moments).  apd_profile_read synchronises those
 * events and returns (and resets) the summed kernel time in milliseconds, the
 * number of scoring launches, the pixel-seed pairs they scored, and the number
 * of kernels of any kind this workspace launched since the last read.
 * Host-synchronous. */
int apd_profile_enable(apd_workspace *ws, int32_t enable);
int apd_profile_read(apd_workspace *ws, double *assign_ms, int64_t *launches, int64_t *pairs,
                     int64_t *kernel_launches);

/* Pixel-seed pairs the FP32 scoring kernel actually evaluated since the last
 * call (counted on the device whether or not profiling is on; equal to the
 * padded N x J of each launch without pruning, fewer with it); resets the
 * count.  Host-synchronous. */
int apd_profile_read_scored(apd_workspace *ws, int64_t *pairs_scored);

/* apd_cell_moments without a workspace, for callers that cannot allocate device
 * memory (a device-memory budget fixed at start-up, a host framework whose
 * allocator owns all device memory, or a latency-critical loop that cannot take
 * the implicit synchronisation of cudaMalloc).  The paper has no counterpart:
 * this is a library convenience.
 *   - Same result as apd_cell_moments with APD_FP32: moments int64 device
 *     [n][APD_MOMENT_WIDTH(dim)], overwritten.
 *   - Scratch is one static device array per GPU (about 8.5 MiB, held by every
 *     GPU that loads the library until exit); the call allocates nothing.
 *   - Limits: n <= 4096 seeds and J <= 2,097,152 pixels; larger sizes return
 *     APD_ERR_WORKSPACE before any work is queued.
 *   - The first call on a device looks up the array's device address (with that
 *     device current); make that first call before any stream capture.
 *   - All calls share the array: calls that overlap on the GPU race on it.  Each
 *     call clears what must start at zero; the array keeps the last call's data.
 *   - Host-synchronous: synchronises `stream` and returns the device-side status
 *     (APD_OK, APD_ERR_ARG for non-finite input, APD_ERR_NOT_SPD, APD_ERR_TIMEOUT),
 *     or APD_ERR_ARG / APD_ERR_WORKSPACE / APD_ERR_CUDA. */
int apd_cell_moments_noalloc(const apd_grid *grid, const apd_seeds *seeds, int64_t *moments,
                             apd_stream_t stream);

/* Diagnostic of the tensor-core (tcgen05) plumbing: one 128 x 128 x 16 MMA on
 * integer-valued operands (exact in TF32 and BF16) from shared memory into
 * tensor memory, compared element by element with CUDA-core dot products.
 * kind: 0 = TF32, 1 = BF16; variant: 0 = the operand layout the library uses,
 * read back with tcgen05.ld; 2 = the same, read back with the min-reducing
 * tensor-memory load (sm_103), whose minimum over each 32-column slice is
 * compared as well (variant 1 is not accepted: APD_ERR_ARG).  Writes the
 * number of mismatching accumulator elements and the largest absolute error
 * (host pointers).  Host-synchronous; runs on the current device. */
int apd_tensor_core_check(int32_t kind, int32_t variant, int32_t *mismatches, float *max_err);

/* Diagnostic of the L-BFGS direction kernels of Algorithm 2's weight solve.  The
 * hist pairs (s_k, y_k) are pushed, oldest first, through the device push
 * kernel (which stores them with their Gram entries s_i.y_j, y_i.y_j), then the
 * direction p = -H g is formed as in the solve, with H0 = gamma I and
 * gamma = s.y / y.y of the newest pair, taken only if that pair passes the
 * curvature test s.y > 1e-12 |s| |y| (otherwise the direction uses the older
 * hist - 1 pairs and gamma = 1).
 *   fused = 0: every pair pushed alone, then the direction kernels (the path of
 *     a solve's first step and of a restart);
 *   fused = 1: the newest pair pushed by the kernel that also forms the
 *     direction's coefficients (the path after every accepted step).  That pair
 *     enters as the step from gradient g - y to gradient g, with g - y and
 *     then y = g - (g - y) rounded on the device.
 *   S, Y: host, [hist][n] row-major, row k = pair k (k = hist - 1 newest);
 *   g: host [n]; p: host [n], written; gp: host, written with <g, p>.
 * Returns APD_ERR_ARG for n < 1, hist outside [1, 31], fused outside {0, 1} or
 * a null pointer.  Host-synchronous; allocates and frees its own device
 * buffers on the current device. */
int apd_lbfgs_check(int32_t n, int32_t hist, const double *S, const double *Y, const double *g, int32_t fused,
                    double *p, double *gp);

/* ---- Batched weight solves (many independent problems at once) ------------
 * A batch holds `count` independent APD problems ("instances") of one
 * dimension, each with its own grid and seed count n_b.  Its seeds are rows
 * [off_b, off_b + n_b) of concatenated device arrays (off_b = n_0 + ... +
 * n_{b-1}, total N = sum n_b): x [N][dim], A [N][dim][dim], w [N], v [N], with
 * the conventions of the one-instance calls.  Each instance is the problem of
 * apd_solve_weights on its own grid (Algorithm 2); the batch evaluates all
 * unconverged instances per iteration with one persistent scoring launch over
 * a shared tile queue, runs the L-BFGS transitions on the device and replays
 * the iteration as a captured CUDA graph.  The paper solves one diagram at a
 * time; batching is a throughput layout of the same computation.  Scoring is
 * FP32 with exact rescoring, so labels and moments equal apd_cell_moments with
 * APD_FP32 per instance. */
typedef struct apd_batch apd_batch;

/* Create a batch for `count` instances (1 .. 50000): grids and n are HOST
 * arrays [count] (grids[b].dim == dim, n[b] >= 1).  tile = -1 picks the tile
 * shape of the scoring kernel on the first call by timing every compiled shape
 * on that call's inputs (autotune); 0 .. apd_batch_tile_info's n_variants - 1
 * fixes it.  Allocates all scratch (about 400 B per seed plus 4 B per pixel).
 * Errors: APD_ERR_ARG, APD_ERR_CUDA. */
int apd_batch_create(apd_batch **batch, int32_t dim, int32_t count, const apd_grid *grids,
                     const int32_t *n, int32_t tile);

/* Free a batch (NULL ignored); no work using it may be in flight. */
void apd_batch_destroy(apd_batch *batch);

/* Tile shape in use (-1 until autotuned), the number of compiled shapes, and
 * (each nullable, HOST arrays [n_variants]) the autotune time of one scoring
 * pass per shape in ms (-1 if not timed) and the shapes as (P, TY, TZ) triples:
 * a tile is P x TY x TZ pixels, P along the first axis. */
int apd_batch_tile_info(apd_batch *batch, int32_t *tile, int32_t *n_variants, double *ms,
                        int32_t *shape);

/* Seed-group pruning of the batch's FP32 scoring, as apd_workspace_set_pruning. */
int apd_batch_set_pruning(apd_batch *batch, int32_t enable);

/* Kernels this batch has launched (graph replays count their six kernels). */
int64_t apd_batch_kernel_launches(apd_batch *batch);

/* One evaluation of every instance at weights w: moments int64 device
 * [N][APD_MOMENT_WIDTH(dim)] (per instance, the layout of apd_cell_moments).
 * Host-synchronous; returns the device-side status (APD_OK, APD_ERR_ARG,
 * APD_ERR_NOT_SPD, APD_ERR_TIMEOUT) or APD_ERR_ARG / APD_ERR_CUDA. */
int apd_batch_cell_moments(apd_batch *batch, const double *x, const double *A, const double *w,
                           int64_t *moments, apd_stream_t stream);

/* Algorithm 2 for every instance from W0 = w0: w_out device [N] receives each
 * instance's converged weights (or its best iterate); info, if not NULL, is a
 * HOST array [count] with each instance's status, iterations, evaluations,
 * max_rel_err and g (seconds = wall time of the whole call).  opts: eps,
 * max_evals (per instance), history (clamped to 1..15), check_volumes;
 * precision must be APD_FP32 (else APD_ERR_UNSUPPORTED).  Host-synchronous.
 * Returns the first error of any instance, else APD_NOT_CONVERGED if any
 * instance hit its cap, else APD_WARN_TOL_INFEASIBLE if any instance's grid
 * fails eq. (2.10), else APD_OK. */
int apd_batch_solve_weights(apd_batch *batch, const double *x, const double *A, const double *w0,
                            const double *v, double *w_out, const apd_solve_opts *opts,
                            apd_solve_info *info, apd_stream_t stream);

/* Algorithm 2 for every instance, started from predicted weights and judged
 * against the plain start: each instance first evaluates g~ at w_pred and at
 * W = 0 and starts from the larger (ties: zero), so a poor prediction costs one
 * evaluation and never a worse start.  used_pred, if not NULL, is a HOST array
 * [count] set to 1 where the prediction was kept.  Otherwise as
 * apd_batch_solve_weights (the two first evaluations are counted). */
int apd_batch_solve_weights_judged(apd_batch *batch, const double *x, const double *A,
                                   const double *w_pred, const double *v, double *w_out,
                                   const apd_solve_opts *opts, apd_solve_info *info,
                                   int32_t *used_pred, apd_stream_t stream);

/* ---- Learned warm start ---------------------------------------------------
 * A per-seed network predicts initial weights for the weight solve from local
 * statistics of the generators.  The paper seeds its solves with W = 0 (and
 * motivates a heuristic initial guess); this predictor is an addition, always
 * judged against the zero start (apd_batch_solve_weights_judged,
 * apd_solve_weights_warm).
 *   Features of seed i of an instance with n seeds on the box [lo, hi] of
 *   measure |O|, s = n / |O|, lengths in units of s^(-1/D) (F = 28 in 2D, 32
 *   in 3D): [v_i s; upper triangle of (A_i + A_i^T)/2; distances to the 8
 *   nearest other seeds, ascending; target volumes of those seeds x s; distance
 *   to the nearer wall per axis; for r = 2, 4, 8: c_r / E_r and
 *   (V_r s - c_r) / E_r with c_r the number and V_r the summed target volume
 *   of the other seeds within distance r, E_r = (unit-ball volume) r^D].
 *   Missing neighbours (n <= 8) give distance 4 and volume 0.
 *   Network: F -> 64 -> 64 -> 64 -> 1, ReLU, FP32; inputs standardised by
 *   (f - mean) * inv_std.  Prediction w_i = y_i s^(-2/D).
 *   Parameters: one FP32 array of apd_warmstart_sizes' n_params values in the
 *   order W1 [64][F], b1 [64], W2 [64][64], b2, W3 [64][64], b3, W4 [64], b4 [1]
 *   (W row-major [out][in]); norm = mean [F] followed by inv_std [F].
 * Instances are described as for batches: offsets HOST int64 [count + 1]
 * (offsets[0] = 0, strictly increasing) into concatenated x / A / v, and
 * box HOST double [count][6] (lo[3] then hi[3] of each instance's domain;
 * entries beyond dim ignored). */
typedef struct apd_mlp apd_mlp;

/* Feature and parameter counts of the network for dim (2 or 3). */
int32_t apd_warmstart_sizes(int32_t dim, int32_t *n_features, int32_t *n_params);

/* Create a network on the current device from HOST params [n_params] and norm
 * [2F] (NULL: mean 0, inv_std 1).  Errors: APD_ERR_ARG, APD_ERR_CUDA. */
int apd_warmstart_create(apd_mlp **net, int32_t dim, const float *params, const float *norm);
void apd_warmstart_destroy(apd_mlp *net);

/* Copy the current parameters / norm to HOST arrays (each nullable). */
int apd_warmstart_get(apd_mlp *net, float *params, float *norm);

/* Features of every seed: features FP32 device [N][F]; knn (int32 device
 * [N][8], nullable) receives the global row of each of the 8 nearest other
 * seeds of the same instance (-1 where missing), in distance order.
 * Stream-ordered. */
int apd_warmstart_features(apd_mlp *net, int32_t count, const int64_t *offsets, const double *box,
                           const double *x, const double *A, const double *v, float *features,
                           int32_t *knn, apd_stream_t stream);

/* Set the network's norm to the mean and 1/std of `samples` feature rows
 * (device [samples][F]).  Stream-ordered. */
int apd_warmstart_fit_norm(apd_mlp *net, int64_t samples, const float *features, apd_stream_t stream);

/* Predicted weights w_out double device [N] from features.  Stream-ordered. */
int apd_warmstart_predict(apd_mlp *net, int32_t count, const int64_t *offsets, const double *box,
                          const float *features, double *w_out, apd_stream_t stream);

/* One training step on the samples idx[0 .. batch) (int32 device indices into
 * features [.][F] and targets FP32 device [.], targets in units of y):
 * loss = (1/batch) sum (y - target)^2, gradient by back-propagation, then an
 * Adam step (beta 0.9 / 0.999, eps 1e-8, step size lr; lr = 0 leaves the
 * parameters unchanged).  grad_out (FP32 device [n_params]) and loss_out (FP32
 * device [1], the SUM of squared residuals) are optional.  Stream-ordered. */
int apd_warmstart_train_step(apd_mlp *net, int32_t batch, const int32_t *idx, const float *features,
                             const float *targets, float lr, float *grad_out, float *loss_out,
                             apd_stream_t stream);

/* Training step on the neighbour-difference loss over the batch rows idx[0 ..
 * batch) and their neighbour lists knn [.][8] (every listed neighbour of a
 * batch row must itself be in the batch, e.g. the batch is whole instances):
 *   L = (1 / (8 batch)) sum_i sum_{j in knn(i)} ((y_i - y_j) - (t_i - t_j))^2
 *       + (mu / batch) sum_i (y_i - t_i)^2    (mu >= 0: a small anchor).
 * The dual's curvature couples neighbouring cells, so errors that differ from
 * cell to cell cost far more than slowly varying ones; this loss measures the
 * former and (for mu = 0) ignores the gauge constant.  y_buf, dy_buf: FP32
 * device scratch indexed like targets.  loss_out (FP32 device [1], nullable)
 * receives L.  Stream-ordered. */
int apd_warmstart_train_step_pairs(apd_mlp *net, int32_t batch, const int32_t *idx,
                                   const float *features, const float *targets, const int32_t *knn,
                                   float *y_buf, float *dy_buf, float mu, float lr, float *grad_out,
                                   float *loss_out, apd_stream_t stream);

/* apd_solve_weights started from the network's prediction for this instance,
 * judged against W = 0 as in apd_batch_solve_weights_judged (seeds->w is not
 * read).  used_pred (host, nullable) = 1 if the prediction was kept.
 * Host-synchronous; status as apd_solve_weights. */
int apd_solve_weights_warm(const apd_grid *grid, const apd_seeds *seeds, const double *v,
                           double *w_out, const apd_solve_opts *opts, apd_solve_info *info,
                           apd_workspace *ws, apd_mlp *net, int32_t *used_pred, apd_stream_t stream);

/* ---- Coarse-to-fine weight solve ------------------------------------------
 * The weights are per seed, not per pixel, so a solve on a coarser grid of the
 * same box gives a start for the fine grid directly.  The coarse solve fixes
 * the smooth, domain-scale part of W that is expensive for L-BFGS on the fine
 * grid; the fine solve then only corrects the discretisation difference.
 * This follows the refinement step that Algorithm 2 allows (raise M, reuse W,
 * continue) run in the opposite order: a cheap coarse solve first. */
typedef struct {
    int32_t factor;           /* coarse grid: ceil(res_d / factor) pixels per axis (>= 4); factor >= 2 */
    double coarse_eps;        /* stop rule of the coarse solve */
    int32_t coarse_max_evals; /* evaluation cap of the coarse solve (its best iterate is used) */
    int32_t carry_history;    /* apd_lloyd_multires: the coarse solves of successive rounds continue
                                 one L-BFGS history (pairs and scaling) instead of starting afresh;
                                 0 = off (default).  The history is kept in a second set of buffers
                                 the workspace allocates on first use. */
    int32_t min_cell_span;    /* the coarse solve runs only when the coarse grid has at least
                                 min_cell_span^dim pixels per seed (default 8: cells about 8 pixels
                                 across; coarser cells cannot reach coarse_eps and the coarse solve
                                 would only burn its evaluation cap); 0 = always */
    int32_t coarse_stall_evals; /* the coarse solve stops (its best iterate is used) after this many
                                   evaluations without a 2 % better max relative volume error: a coarse
                                   grid whose discretisation keeps it above coarse_eps has stalled
                                   (0 = off, the default: on the runtime tests' 2D points, 30 helped
                                   single-phase solves by up to 25 % and slowed multi-phase ones by up
                                   to 50 %, whose coarse stage keeps improving the smooth part of W
                                   while the largest error stands still) */
} apd_multires_opts;

/* Fill *mo with the defaults: factor 2, coarse_eps 0.05, coarse_max_evals 60. */
void apd_multires_opts_default(apd_multires_opts *mo);

/* Coarse solve from W0 = seeds->w (or, with net != NULL, from the network's
 * prediction judged against W = 0), then the fine solve (opts) from the coarse
 * weights.  info->evaluations counts fine evaluations, coarse_evaluations the
 * coarse ones.  used_pred as apd_solve_weights_warm (0 without a network).
 * Host-synchronous; status of the fine solve, as apd_solve_weights. */
int apd_solve_weights_multires(const apd_grid *grid, const apd_seeds *seeds, const double *v,
                               double *w_out, const apd_solve_opts *opts,
                               const apd_multires_opts *mo, apd_solve_info *info,
                               apd_workspace *ws, apd_mlp *net, int32_t *used_pred,
                               apd_stream_t stream);

/* Algorithm 3 with every weight solve coarse-to-fine: `rounds` Lloyd moves
 * and a final solve as apd_lloyd, each solve first on the coarse grid from the
 * previous weights (the first from seeds->w, or from the network's prediction
 * judged against W = 0 when net != NULL), then on the target grid.
 * info->evaluations / coarse_evaluations sum over all solves.  Host-synchronous;
 * status as apd_lloyd. */
int apd_lloyd_multires(const apd_grid *grid, const apd_seeds *seeds, const double *v, int32_t rounds,
                       double *x_out, double *w_out, const apd_solve_opts *opts,
                       const apd_multires_opts *mo, apd_solve_info *info, apd_workspace *ws,
                       apd_mlp *net, int32_t *used_pred, apd_stream_t stream);

/* The batched form: every instance solved on its coarse grid (a second batch
 * over the coarse grids, created on first use and kept), from w0, judged
 * against zero when judge != 0, then on its own grid from the coarse weights.
 * Arguments and status as apd_batch_solve_weights_judged. */
int apd_batch_solve_weights_multires(apd_batch *batch, const double *x, const double *A,
                                     const double *w0, const double *v, double *w_out,
                                     const apd_solve_opts *opts, const apd_multires_opts *mo,
                                     int32_t judge, apd_solve_info *info, int32_t *used_pred,
                                     apd_stream_t stream);

/* ---- Refining weight solve (Algorithm 2, step 4) -------------------------
 * When the weights cannot reach the tolerance on the grid (the solve stalls at
 * its evaluation cap, or the grid is coarser than eq. (2.10) asks for the
 * smallest target volume), the grid of the same box is refined and the solve
 * restarts from the weights found: they are per seed, so they carry over. */
typedef struct {
    double growth;          /* resolution factor per refinement, > 1 (default 1.5) */
    int32_t max_res[3];     /* largest resolution per axis; 0: bounded by the workspace's pixel capacity */
    int32_t max_rounds;     /* refinements at most (default 4) */
} apd_refine_opts;

void apd_refine_opts_default(apd_refine_opts *ro);

/* Solves on `grid` from seeds->w (as apd_solve_weights).  While the result is
 * APD_NOT_CONVERGED or APD_WARN_TOL_INFEASIBLE and rounds remain, every axis
 * grows by the same factor f = max(growth, (J_(2.10) / J)^(1/D)), J_(2.10) the
 * pixel count at which eq. (2.10) holds for the smallest v, each resolution
 * rounded up; the solve restarts from the weights found.  The round stops
 * early when the next grid exceeds max_res or the workspace's max_j.
 * grid_out (host, nullable) receives the grid of the last solve; info sums the
 * evaluations and iterations over the rounds (info->solves = rounds + 1) and
 * reports the last solve's error and status.  Arguments as apd_solve_weights;
 * ro null: defaults; growth <= 1, max_rounds < 0 or a max_res below the
 * grid's resolution on an axis: APD_ERR_ARG. */
int apd_solve_weights_refine(const apd_grid *grid, const apd_seeds *seeds, const double *v, double *w_out,
                             const apd_solve_opts *opts, const apd_refine_opts *ro, apd_solve_info *info,
                             apd_grid *grid_out, apd_workspace *ws, apd_stream_t stream);

/* The refinement rule of apd_solve_weights_refine, on the host: the grid of
 * the same box with every resolution scaled by f = max(growth, (J_(2.10) /
 * J)^(1/D)) and rounded up, J_(2.10) = |Omega| 2^D / (eps v_min).  Returns
 * APD_OK with *next written, 1 when it exceeds ro->max_res on an axis or
 * max_pixels (> 0), APD_ERR_ARG for invalid arguments (no device use). */
int apd_refine_next_grid(const apd_grid *grid, double v_min, double eps, const apd_refine_opts *ro,
                         int64_t max_pixels, apd_grid *next);

/* ---- Non-uniform discretisation (Section 2.3) -----------------------------
 * Elements P_j of any shape, given by a sample point y_j and a measure |P_j|
 * (the regular grid is the case y_j = pixel centre, |P_j| = |P|).  Labels as
 * Algorithm 1 (FP64 argmin, lowest index on ties, equal to a full FP64
 * evaluation); moments are the measure-weighted sums m_i = sum |P_j|,
 * S1_i = sum |P_j| y_j and S2_i = sum |P_j| y_j y_j^T (upper triangle, a <= b,
 * row-major), in FP64, accumulated with atomics (their last bits depend on the
 * order of the additions). */
typedef struct {
    int32_t dim;          /* 2 or 3 */
    int64_t count;        /* number of elements, >= 1 */
    const double *y;      /* [count][dim] sample points (device) */
    const double *mass;   /* [count] element measures |P_j| (device) */
} apd_points;

/* Labels (nullable, [count] int32) and FP64 moments [n][1 + D + D(D+1)/2]
 * (device, overwritten) of the elements.  Stream-ordered; argument errors are
 * returned (null pointers, count < 1, dim mismatch, n above the workspace's
 * max_n), device-side errors latch in the workspace. */
int apd_points_moments(const apd_points *pts, const apd_seeds *seeds, double *moments, int32_t *labels,
                       apd_workspace *ws, apd_stream_t stream);

/* Eqs. (2.7)-(2.8) on the elements: g~ = sum_i v_i w_i + sum_j |P_j| c_{H_j j}
 * into g_out[0], grad_i = v_i - m_i into grad [n], max_i |grad_i| / v_i into
 * max_rel_err[0] (all device).  Stream-ordered; errors as apd_points_moments. */
int apd_points_dual_value_grad(const apd_points *pts, const apd_seeds *seeds, const double *v, double *g_out,
                               double *grad, double *max_rel_err, apd_workspace *ws, apd_stream_t stream);

/* ---- Masked two-level discretisation (Section 4) ---------------------------
 * The paper's outlook: adaptable pixel sizes, with the pixels at the cell
 * boundaries found and refined by masking.  It gives no algorithm; this
 * library's reading, on a coarse grid G (the `coarse` argument) and an
 * integer factor r >= 1:
 *   1. Algorithm 1 on G gives the coarse labels H^G.
 *   2. A coarse pixel is a boundary pixel when a pixel of its 3^D
 *      neighbourhood (faces, edges and corners) inside the grid has another
 *      label, else an interior pixel.
 *   3. The fine grid F has r res[d] pixels per axis on the same box.  A fine
 *      pixel inside an interior coarse pixel takes that pixel's label; a fine
 *      pixel inside a boundary coarse pixel is labelled by Algorithm 1 on F
 *      (exact FP64 argmin, lowest index on ties).
 * The result is a labelling of F: its integer moments (count, sum u,
 * sum u u^T with u = 2k + 1 of the fine pixel indices k, the layout of
 * apd_cell_moments) feed eqs. (2.7)-(2.8) on F.  It equals the full
 * Algorithm 1 on F wherever no cell boundary passes through an interior
 * coarse pixel (always, for example, across the straight boundary of two
 * seeds with equal A away from the grid's outer layer).  Each fine pixel of a
 * boundary coarse pixel is scored against every seed (no pruning), so the
 * call only pays where few coarse pixels are boundary pixels.
 *
 * moments: device int64 [n][1 + D + D(D+1)/2], overwritten.
 * coarse_labels: device int32 [J_G], written with H^G.
 * refined: device int64 [1], nullable: the number of fine pixels of step 3
 *          labelled by Algorithm 1 (r^D times the boundary coarse pixels).
 * Stream-ordered.  APD_ERR_ARG: invalid grid or seeds, null moments or
 * coarse_labels, r < 1, or a fine grid of 2^31 pixels or more;
 * APD_ERR_WORKSPACE: the workspace does not hold the coarse grid and n
 * seeds.  Device-side errors latch in the workspace. */
int apd_masked_moments(const apd_grid *coarse, int32_t refine, const apd_seeds *seeds, int64_t *moments,
                       int32_t *coarse_labels, int64_t *refined, apd_workspace *ws, apd_stream_t stream);

/* Eqs. (2.7)-(2.8) on the fine grid F from the moments of apd_masked_moments
 * (held in the workspace): g~ into g_out[0], grad_i = v_i - |P_F| m_i into
 * grad [n] (nullable), max_i |grad_i| / v_i into max_rel_err[0] (all
 * device).  Arguments and errors as apd_masked_moments, plus null v, g_out
 * or max_rel_err: APD_ERR_ARG. */
int apd_masked_dual_value_grad(const apd_grid *coarse, int32_t refine, const apd_seeds *seeds, const double *v,
                               double *g_out, double *grad, double *max_rel_err, int32_t *coarse_labels,
                               apd_workspace *ws, apd_stream_t stream);

/* Eq. (2.10): smallest M with |Omega| / M^D <= eps v_min / 2^D (the non-strict
 * reading, which gives the paper's M = 200 for D = 3, N = 10^4, v = 1/N).
 * Returns M >= 1, or -1 for invalid arguments. */
int64_t apd_choose_resolution(int32_t dim, double v_min, double eps, double domain_measure);

/* Static text for a status code. */
const char *apd_status_string(int status);

/* Library version as an integer (major * 10000 + minor * 100 + patch). */
int32_t apd_version(void);

#ifdef __cplusplus
}
#endif
#endif /* APD_H */
