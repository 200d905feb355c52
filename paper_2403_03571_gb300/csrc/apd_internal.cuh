// Internal declarations shared by the CUDA translation units of libapd.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/apd.h"

namespace apd {

// ----------------------------------------------------------------------------
// device status bits (latched in DevScalars::status, mapped to apd_status)
// ----------------------------------------------------------------------------
enum : int {
    ST_NONFINITE = 1,   // non-finite x, A or w
    ST_NOT_SPD = 2,     // (A + A^T)/2 not positive definite
    ST_TIMEOUT = 4,     // a bounded mbarrier wait ran out
    ST_BAD_VOLUME = 8,  // v_i <= 0 or non-finite
    ST_BAD_LABEL = 16,  // internal: a label outside [0, n)
};

// Seed record streamed into shared memory by the scoring kernels: the FP64
// position and weight (recentred per tile in FP64, then rounded) and the FP32
// symmetric part of A (upper triangle: 2D 00 01 11, 3D 00 01 02 11 12 22).
struct __align__(16) SeedRec {
    double x[3];
    double w;
    float a[6];
    float pad[2];
};
static_assert(sizeof(SeedRec) == 64, "SeedRec must be 64 bytes");

// Seed record of the FP32 direct-form rescoring pass: x and w split into
// FP32 high and low parts (x = x_hi + x_lo to ~2^-48 relative), FP32 symmetric A,
// a lower bound of lambda_min and an upper bound of lambda_max of the FP64 A.
struct __align__(16) SeedRec32 {
    float xh[3], xl[3];
    float wh, wl;
    float a[6];
    float pad[2];  // [0] lambda_min lower bound, [1] lambda_max upper bound
};
static_assert(sizeof(SeedRec32) == 64, "SeedRec32 must be 64 bytes");

// Bounds of a group of 32 consecutive seeds (scan order) for pruning the
// scoring and the near-tie rescoring: FP32 box of the positions (rounded
// outwards), a lower bound of lambda_min over the group, the largest weight,
// and wref - wmax rounded down (wref = the largest weight of all seeds).
struct __align__(8) GroupBound {
    float lo[3], hi[3];
    float lam;
    float wgap;
    double wmax;
};
static_assert(sizeof(GroupBound) == 40, "GroupBound must be 40 bytes");

constexpr int kChunk = 256;         // seeds per shared-memory chunk (= scoring CTA size)
constexpr int kSortMax = 16384;     // largest padded seed count ordered on the device
constexpr int kGroup = 32;          // seeds per packed-index group (5 low mantissa bits)
constexpr int kWarmFeatMax = 32;    // warm-start features per seed (3D; 28 in 2D)
constexpr uint32_t kDefaultWaitPolls = 1u << 16;  // polls of a bounded mbarrier wait (~1.3 s)

// Small block of device scalars owned by the workspace.
struct DevScalars {
    int status;
    unsigned int flag_count;            // pixels queued for FP64 rescoring in the last pass
    unsigned long long wref_key;        // ordered-key max of w
    unsigned long long lam_abs_bits;    // max_i ||sym A_i||_F  (non-negative double bits)
    unsigned long long lam_min_bits;    // min_i lower bound of lambda_min(sym A_i)
    double g;                           // dual value
    double max_rel_err;
    double dot_gp;                      // <grad f, p> at the last evaluation
    double sum_v;
    double min_v;
    double sy, yy, ss;                  // L-BFGS curvature pair products
    double gp0;                         // <grad f, p> at the start of a line search
    unsigned int dual_done;             // block counter of the two-phase dual reduction
    int pair_ok;                        // the last pushed L-BFGS pair passed the curvature test
    long long rescored_total;
    unsigned int mask_count;            // boundary coarse pixels listed by the masked discretisation
    unsigned int lbfgs_done;            // block counter of the L-BFGS kernels' last-block reductions
    unsigned int band_count;            // pixels re-decided by the last incremental pass
    double drift_max, drift_min;        // max and min of w - w0 (incremental passes)
    float band_D;                       // drift_max - drift_min rounded up
    float band_shift;                   // w_ref - w_ref0 - drift_max rounded down
    float drift_hi;                     // drift_max rounded up to a float
    int inc_go;                         // this incremental pass re-decides from the record (else records)
    int inc_valid;                      // a record of this solve exists
};

// Partial sums per block row of the L-BFGS dot-product kernels: the push's
// 3 + 3 (cap - 1) Gram products and 2 + 2 (cap - 1) direction products, cap = 32.
constexpr int kLbfgsDots = 160;
constexpr int kPartStride = 6;  // doubles per block row of Workspace::part
// Bins of the incremental record's margin histogram: a positive float margin
// falls in bin (its bits >> 21), four bins per octave (bin 0: no margin).
constexpr int kIncBins = 1024;

// Coefficients of an L-BFGS direction p = -gamma g + sum_k (cy_k y_k + cs_k s_k)
// over the pairs in slot[0..hist) (device; written by the direction's first kernel).
struct LbfgsCoef {
    int hist;
    int slot[32];
    double gamma;
    double cy[32], cs[32];
};

// Bits of Workspace::attr_done: the dynamic shared-memory limit of these
// kernels is raised once per workspace (a workspace lives on one device).
constexpr unsigned kAttrFp32Score2 = 1u << 0, kAttrFp32Score3 = 1u << 1, kAttrMortonSort = 1u << 2;
constexpr unsigned kAttrTcScore = 1u << 3;     // + 1 bit per (dimension, operand kind): 4 bits
constexpr unsigned kAttrTcScoreRec = 1u << 7;  // the recording variant: 4 bits

// One evaluation of a weight solve (trial weights, scoring, rescoring, dual,
// read-back of the device scalars) captured as a CUDA graph and replayed with
// a new trial step t.  The key holds every argument the captured launches take.
struct EvalGraph {
    std::vector<unsigned char> key;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t begin = nullptr;  // the eval_begin kernel node (null: no trial step)
    int64_t launches = 0, pixels = 0, pairs = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;  // around the scoring stage (profiling)
    uint64_t used = 0;
    bool failed = false;  // capture refused: this key runs without a graph
    bool recorded = false;  // queued as an incremental pass (the device chooses its kind)
};

// Workspace (host struct; device pointers inside).
struct Workspace {
    int dim = 0;
    int max_n = 0;
    int64_t max_j = 0;
    int device = 0;
    int sms = 152;                      // the device's SM count, read when the workspace is made
    unsigned attr_done = 0;             // kAttr* bits: shared-memory attribute set on this device
    int rescore_bps[2] = {0, 0};        // resident rescoring blocks per SM (2-D, 3-D)
    int n_pad_max = 0;
    SeedRec *recs = nullptr;            // [n_pad_max]
    SeedRec32 *recs32 = nullptr;        // [n_pad_max]
    // Morton ordering of the seeds for the scoring scan (null: natural order)
    SeedRec *recs_tmp = nullptr;        // [n_pad_max] records in natural order
    uint32_t *codes = nullptr;          // [n_pad_max] Morton codes, natural order
    uint32_t *scodes = nullptr;         // [n_pad_max] sorted codes
    int32_t *perm = nullptr;            // [n_pad_max] scan position -> seed index
    SeedRec32 *recs32s = nullptr;       // [n_pad_max] SeedRec32 in scan order
    float *tc_centre = nullptr;         // [tc_tile_cap][6] tensor-core tile centres (FP32 hi, lo)
    int *tc_start = nullptr;            // [tc_tile_cap] Morton start chunk per tile (dense form)
    int4 *tc_meta = nullptr;            // [tc_tile_cap] first pixel per axis, candidate count
    float *tc_texcl = nullptr;          // [tc_tile_cap] cost lower bound of the seeds left out
    int *tc_list = nullptr;             // [tc_tile_cap][tc_list_cap()] candidates
    uint8_t *tc_bops = nullptr;         // [tc_tile_cap] x tc_bops_bytes_per_tile(): stored seed operands
    float4 *tc_axis = nullptr;          // [3 tc_tile_cap] per-axis tile centres and pixel boxes
    double tc_axis_key[12] = {};        // the grid and tiling tc_axis was computed for (all 0: none)
    double tc_cond = 0.0;               // max ||A||_F / min lambda_min of the last prepared seeds
    long long tc_tile_cap = 0;
    bool sorted = false;                // set by launch_seed_prep for the current pass
    bool prune = false;                 // FP32 scoring skips seed groups by their bounds
    uint32_t wait_limit = kDefaultWaitPolls;  // polls of the scoring kernels' chunk waits
    // sharded evaluation: every scoring pass covers this rank's slab of the last
    // axis only, and shard_fn sums the moments over the ranks before they are used
    int shard_rank = 0, shard_world = 1;
    apd_reduce_fn shard_fn = nullptr;
    void *shard_ctx = nullptr;
    unsigned long long *pairs_scored = nullptr;  // device counter: pairs the FP32 scoring evaluated
    unsigned long long *moments = nullptr;  // [max_n * K]
    uint32_t *flags = nullptr;          // [max_j]
    int32_t *flag_gi = nullptr;         // [max_j] FP32 best seed of each queued pixel (-1: none)
    GroupBound *groups = nullptr;       // [n_pad_max / 32] bounds of the scan-order seed groups
    DevScalars *sc = nullptr;           // device
    DevScalars *sc_host = nullptr;      // pinned host mirror
    double *part = nullptr;             // [part_rows][kPartStride] per-block partials (dual, trial weights)
    int part_rows = 0;
    double *grad = nullptr;             // [max_n] gradient of g~ of the last evaluation
    // L-BFGS / Lloyd state
    int hist_cap = 0;
    double *W = nullptr, *Wt = nullptr, *p = nullptr, *gf = nullptr, *gft = nullptr;
    double *Wbest = nullptr;
    double *S = nullptr, *Y = nullptr;  // [hist_cap][max_n]
    double *gram = nullptr;             // [2][hist_cap][hist_cap] s_i.y_j, y_i.y_j of the stored pairs
    double *lb_part = nullptr;          // [lb_rows][kLbfgsDots] per-block partial sums of the L-BFGS kernels
    int lb_rows = 0;
    LbfgsCoef *lb_coef = nullptr;       // the last direction's coefficients
    bool p_pending = false;             // lb_coef holds a direction that ws.p does not yet hold
    // incremental evaluation (weight solves with the pruned tensor-core scorer): a
    // full pass records each pixel's label, runner-up and certified cost margins,
    // the moments and the weights; a later pass at weights w re-decides only the
    // pixels whose margins the drift w - w0 can close.  Which of the two a pass
    // is, the trial-weights kernel decides on the device (sc->inc_go).
    int32_t *inc_labels = nullptr;      // [max_j] labels of the recorded pass
    float *inc_gap = nullptr;           // [max_j] certified gaps of the recorded pass
    float4 *inc_rec = nullptr;          // [max_j] runner-up and margins of the recorded pass
    unsigned *inc_hist = nullptr;       // [kIncBins] recorded pixels by their g3 margin (see kIncBins)
    float2 *inc_drift = nullptr;        // [max_n] w - w0 per seed as a float interval (lo, hi)
    int band_bps[2] = {0, 0};           // resident blocks per SM of the re-decision kernel (2D, 3D)
    bool inc_auto = false;              // set while an incremental pass is queued (kernels test sc->inc_go)
    unsigned long long *inc_mom0 = nullptr;  // [max_n * K] moments of the recorded pass
    double *inc_w0 = nullptr;           // [max_n] weights of the recorded pass
    unsigned long long *inc_aux = nullptr;  // [2] ordered key of the recorded pass's w_ref, spare
    float *rec_gap = nullptr;           // set while a recording pass is queued (the scorer's gap output)
    int incremental = 1;                // apd_workspace_set_incremental mode (0 off, 1 large grids, 2 all)
    bool inc_recorded = false;          // the last queued pass recorded its state
    double *rho = nullptr;              // [hist_cap]
    // a second L-BFGS history (pairs, Gram entries, 1 / s.y) continued by the coarse
    // solves of a Lloyd run (allocated on first use), and its host-side state
    double *S2 = nullptr, *Y2 = nullptr, *gram2 = nullptr, *rho2 = nullptr;
    int solve_stall = 0;                // the running solve's stall limit (coarse solves), 0: none
    bool carry_enabled = false;         // a Lloyd run with carry_history is in progress
    bool carry_on = false;              // the running solve starts from `carry` and leaves its history there
    struct {
        int hist = 0, newest = 0;
        double gamma = 1.0;
        bool valid = false;
    } carry;
    double *X = nullptr;                // [max_n * dim] seed positions for Lloyd
    double *vbuf = nullptr;             // [max_n]
    float *wfeat = nullptr;             // [max_n][kWarmFeatMax] warm-start features
    double *wpred = nullptr;            // [max_n] predicted weights
    int64_t last_pixels = 0, last_pairs = 0;
    // optional kernel timing (event pairs around scoring launches)
    bool profiling = false;
    std::vector<cudaEvent_t> ev;  // 2 per recorded launch
    size_t ev_used = 0;
    int64_t prof_pairs = 0;
    cudaEvent_t prof_e0 = nullptr;  // start event the next scoring kernel launch records
    double prof_ms_graph = 0.0;   // scoring-kernel time of replayed evaluation graphs
    int64_t prof_n_graph = 0;
    // evaluation graphs of the weight solve
    bool graphs = true;
    bool capturing = false;       // launches go into a stream capture
    cudaStream_t cap_stream = nullptr;
    cudaEvent_t cap_e0 = nullptr, cap_e1 = nullptr;
    std::vector<EvalGraph> graph_cache;
    uint64_t graph_clock = 0;
    int64_t kernel_launches = 0;  // every kernel launched with this workspace
};

// Grid description passed by value to kernels.  A scoring pass covers the
// pixels whose index along the last (slowest) axis lies in the window
// [kz0, kz1); kz1 == 0 means the whole axis.  Pixel ids, centres and the odd
// coordinates u of the moments are always those of the full grid, so the
// moments of disjoint windows add up to the full grid's.
struct GridDev {
    int dim;
    int res[3];
    double lo[3];
    double h[3];
    float h32[3];
    double cell;  // |P|
    long long J;  // pixels of the full grid
    int kz0, kz1;
};
// the last axis's resolution (a select, not a dynamic index: an indexed access
// to a kernel's by-value GridDev makes the compiler copy it to the stack)
__host__ __device__ inline int res_last(const GridDev &g) { return g.dim == 3 ? g.res[2] : g.res[1]; }
__host__ __device__ inline int win_lo(const GridDev &g) { return g.kz0; }
__host__ __device__ inline int win_hi(const GridDev &g) { return g.kz1 ? g.kz1 : res_last(g); }
// pixels of the window and the full-grid id of its first pixel
__host__ __device__ inline long long win_pixels(const GridDev &g) {
    return g.J / res_last(g) * (long long)(win_hi(g) - win_lo(g));
}
__host__ __device__ inline long long win_first(const GridDev &g) {
    return g.J / res_last(g) * (long long)win_lo(g);
}

// ----------------------------------------------------------------------------
// ordered keys for atomic max/min of doubles
// ----------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long dkey(double v) {
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double dkey_inv(unsigned long long k) {
    unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)b);
}

// ----------------------------------------------------------------------------
// Morton (Z-order) codes on the grid box, 10 bits per axis in 3D, 15 in 2D
// ----------------------------------------------------------------------------
__host__ __device__ inline uint32_t spread3_10(uint32_t v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}
__host__ __device__ inline uint32_t spread2_15(uint32_t v) {
    v &= 0x7fffu;
    v = (v | (v << 8)) & 0x00ff00ffu;
    v = (v | (v << 4)) & 0x0f0f0f0fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}
// frac: position in [0, 1) of the box per axis
__host__ __device__ inline uint32_t morton_code(int dim, const double *frac) {
    if (dim == 3) {
        uint32_t q[3];
        for (int a = 0; a < 3; ++a) {
            double f = frac[a] * 1024.0;
            q[a] = f <= 0.0 ? 0u : (f >= 1023.0 ? 1023u : (uint32_t)f);
        }
        return spread3_10(q[0]) | (spread3_10(q[1]) << 1) | (spread3_10(q[2]) << 2);
    }
    uint32_t q[2];
    for (int a = 0; a < 2; ++a) {
        double f = frac[a] * 32768.0;
        q[a] = f <= 0.0 ? 0u : (f >= 32767.0 ? 32767u : (uint32_t)f);
    }
    return spread2_15(q[0]) | (spread2_15(q[1]) << 1);
}

// ----------------------------------------------------------------------------
// mbarrier + bulk async copy (TMA, non-tensor form), all waits bounded
// ----------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
// 1-D bulk copy global -> shared, completion signalled on `bar` (16-byte aligned, size % 16 == 0).
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
// One poll of the phase; the thread may sleep up to kWaitHintNs while the phase
// is incomplete (it is woken when the phase completes).
constexpr uint32_t kWaitHintNs = 20000;
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "n"(kWaitHintNs)
        : "memory");
    return ok != 0;
}
// Bounded wait: returns false (and latches ST_TIMEOUT) after `limit` polls
// (at most limit x 20 us, about 1.3 s with the default).  A limit of 0 gives up
// without polling (used to exercise the timeout path on purpose).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int *status,
                                                  uint32_t limit = kDefaultWaitPolls) {
    for (uint32_t it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    atomicOr(status, ST_TIMEOUT);
    return false;
}

// ----------------------------------------------------------------------------
// host helpers (apd_capi.cu)
// ----------------------------------------------------------------------------
int map_bits(int bits);                              // ST_* bits -> apd_status
// contiguous slab [k_begin, k_begin + k_count) of `res` pixels for rank of world
void shard_range(int res, int rank, int world, int &k_begin, int &k_count);
int validate_grid(const apd_grid *gr, GridDev &g);  // apd_grid -> GridDev, APD_ERR_ARG if invalid
double domain_measure(const apd_grid *gr);          // |Omega|
int warmstart_dim(const apd_mlp *net);               // dimension of a warm-start network (apd_warmstart.cu)

// ----------------------------------------------------------------------------
// launchers (defined in the .cu files)
// ----------------------------------------------------------------------------
constexpr int moment_width(int dim) { return 1 + dim + dim * (dim + 1) / 2; }

// zero the per-evaluation counters and statistics in sc
cudaError_t launch_eval_reset(Workspace &ws, cudaStream_t st, bool keep_geometry = false);
// non-uniform discretisation (apd_points.cu, apd_kernels.cu): labels and FP64
// element-measure moments of `count` points; the dual from those moments
cudaError_t launch_points_assign(int dim, long long count, const double *y, const double *mass, int n,
                                 const double *x, const double *A, const double *w, double *mom,
                                 int32_t *labels, Workspace &ws, cudaStream_t st);
cudaError_t launch_points_dual(int dim, int n, const double *x, const double *A, const double *w, const double *v,
                               const double *mom_pts, Workspace &ws, double *g_out, double *grad_out,
                               double *err_out, cudaStream_t st);
// masked two-level discretisation (apd_masked.cu), after a coarse scoring pass
// that left its labels in `coarse_labels` and the seed records in ws: boundary
// mask, closed-form fine moments of the interior coarse pixels and the fine
// pixels of the boundary ones scored in FP64 (moments zeroed first; `refined`
// nullable)
cudaError_t launch_masked_refine(const GridDev &gc, const GridDev &gf, int r, int n, const double *x,
                                 const double *A, const double *w, const int32_t *coarse_labels,
                                 unsigned long long *mom, long long *refined, Workspace &ws, cudaStream_t st);
// start of an evaluation with the records of the last launch_seed_prep (same x,
// A, n): zeroed moments and counters, weights W0 + t pdir (into Wt; pdir null:
// W0 itself) in the records, wref and the group weight gaps
// form_p: pdir is first formed from the last direction coefficients (ws.lb_coef,
// gradient ws.gf) and <gf, p> goes to sc->gp0.
// w0 (nullable): the drift range max/min of w - w0 goes to sc->drift_max / drift_min.
// With w0 (incremental passes) also the drift range of w - w0 and the choice of
// the pass: re-decide from the record when one exists and at most full_max
// recorded pixels have a g3 margin within the drift (sc->inc_go), else record.
cudaError_t launch_eval_begin(int n, const double *W0, double t, const double *pdir, double *Wt,
                              unsigned long long *mom, Workspace &ws, cudaStream_t st, bool form_p = false,
                              const double *w0 = nullptr, unsigned full_max = 0u);
// seed records (FP64 x, w; FP32 symmetric A) + stats (max w, max ||A||_F, min lambda bound)
cudaError_t launch_seed_prep(const GridDev &g, int n, const double *x, const double *A,
                             const double *w, Workspace &ws, cudaStream_t st);
// FP32 scoring fused with the moments; queues near ties; labels optional.
cudaError_t launch_assign_fp32(const GridDev &g, int n, Workspace &ws, int32_t *labels,
                               unsigned long long *moments, cudaStream_t st);
// tcgen05 scoring fused with the moments (kind 0 = TF32, 1 = BF16; per-tile candidate
// lists when ws.prune); queues the pixels it cannot certify.
cudaError_t launch_assign_tc(const GridDev &g, int n, Workspace &ws, int32_t *labels,
                             unsigned long long *moments, int kind, cudaStream_t st);
// number of tensor-core tiles the grid's scoring window needs (the workspace holds
// tc_tile_cap), and the candidate seeds stored per tile
long long tc_tile_count(const GridDev &g);
int tc_list_cap();
size_t tc_bops_bytes_per_tile();
// bounds of the 32-seed groups of the scan-order records (ws.groups)
cudaError_t launch_group_bounds(int n, Workspace &ws, cudaStream_t st);
// FP64 rescoring of the queued pixels (labels optional, moments updated).
cudaError_t launch_rescore_fp64(const GridDev &g, int n, const double *x, const double *A,
                                const double *w, Workspace &ws, int32_t *labels,
                                unsigned long long *moments, cudaStream_t st,
                                const int32_t *old_labels = nullptr, const int *go = nullptr);
// relative gap of the two smallest FP64 costs of every pixel (after a scoring
// pass on the same seeds: uses its records, group bounds and w_ref)
cudaError_t launch_tie_gap(const GridDev &g, int n, const double *x, const double *A, const double *w,
                           Workspace &ws, double *gap, cudaStream_t st);
// dual value / gradient from the moments (outputs optional; scalars also into ws.sc)
cudaError_t launch_dual(const GridDev &g, int n, const double *x, const double *A, const double *w,
                        const double *v, const double *p_dir, const unsigned long long *moments,
                        Workspace &ws, double *g_out, double *grad_out, double *gf_out,
                        double *err_out, cudaStream_t st);
// discrete centroids from the moments (empty cells keep x)
cudaError_t launch_centroids(const GridDev &g, int n, const double *x,
                             const unsigned long long *moments, double *x_out, cudaStream_t st);
// L-BFGS helpers
cudaError_t launch_axpy(int n, const double *a, double t, const double *b, double *out,
                        cudaStream_t st);
cudaError_t launch_lbfgs_direction(int n, int hist, int newest, int cap, double gamma, bool use_pair,
                                   int hist_acc, int newest_acc,
                                   Workspace &ws, cudaStream_t st);
// Push of the pair (Wt - W, gft - gf) into `slot` with its Gram entries against
// the nprev slots before it; with dir, also the coefficients of the direction
// for the gradient gft (taken with the pair if it passes the curvature test:
// hist_acc pairs; else the hist pairs before it and gamma).  launch_lbfgs_pdir
// then forms p from the last coefficients and the gradient ws.gf.
cudaError_t launch_lbfgs_push(int n, int slot, int cap, int nprev, bool dir, int hist, int hist_acc, double gamma,
                              Workspace &ws, cudaStream_t st);
cudaError_t launch_lbfgs_pdir(int n, Workspace &ws, cudaStream_t st);
// Records the pending profiling start event (if any) on st: called by the
// scoring launchers right before the scoring kernel.
inline cudaError_t record_scoring_start(Workspace &ws, cudaStream_t st) {
    cudaEvent_t e = ws.prof_e0;
    if (!e) return cudaSuccess;
    ws.prof_e0 = nullptr;
    return ws.capturing ? cudaEventRecordWithFlags(e, st, cudaEventRecordExternal) : cudaEventRecord(e, st);
}
// graph support: the eval_begin kernel (to find its node), its launch written
// into an instantiated graph's node, and the tensor-core per-axis table
// brought up to date for a grid outside any capture
const void *eval_begin_kernel_fn();
cudaError_t set_eval_begin_node(cudaGraphExec_t exec, cudaGraphNode_t node, int n, const double *W0, double t,
                                const double *pdir, double *Wt, unsigned long long *mom, Workspace &ws,
                                bool form_p, const double *w0, unsigned full_max);
// the direction's coefficients only (p is then formed by the next trial's eval_begin)
cudaError_t launch_lbfgs_coefficients(int n, int hist, int newest, int cap, double gamma, bool use_pair,
                                      int hist_acc, int newest_acc, Workspace &ws, cudaStream_t st);
cudaError_t launch_tc_axis(const GridDev &g, Workspace &ws, cudaStream_t st);
// the incremental pass's re-decision of the pixels within the drift of their recorded gap
cudaError_t launch_tc_band(const GridDev &g, int n, Workspace &ws, cudaStream_t st);
// incremental pass, before scoring: the recorded moments copied in (re-decision)
// or the margin histogram cleared (recording); after rescoring: the record's
// moments, weights and w_ref kept (recording)
cudaError_t launch_inc_prepare(int n, unsigned long long *mom, Workspace &ws, cudaStream_t st);
cudaError_t launch_inc_commit(int n, const unsigned long long *mom, const double *w, Workspace &ws,
                              cudaStream_t st);

}  // namespace apd
