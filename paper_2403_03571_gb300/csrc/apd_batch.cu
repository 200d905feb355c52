// Batched weight solves: many independent APD problems (instances) of one
// dimension, each with its own grid and seed count, solved together.
//
// One iteration evaluates the dual of every unconverged instance and advances
// its solver by one step, with six launches whatever the instance count:
//   schedule  (1 CTA)        list the active instances, prefix-sum their tiles
//   prep      (CTA/instance) seed records at the trial weights, Morton sort
//   assign    (persistent)   one CTA per SM slot pulls (instance, tile) items
//                            from a shared queue, heaviest instances first, and
//                            scores each tile with the FP32 tile routine of the
//                            one-instance path (Algorithm 1 fused with moments)
//   rescore   (CTAs/instance) FP64 near-tie rescoring
//   dual      (CTA/instance) eqs. (2.7)-(2.8) from the integer moments
//   lbfgs     (CTA/instance) one transition of the L-BFGS / strong-Wolfe state
//                            machine of Algorithm 2, writing the next trial point
// The iteration is captured once in a CUDA graph and replayed until no
// instance is active.  The tile shape of the persistent kernel is picked per
// batch by timing every compiled variant on the batch itself (autotune).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "apd_common.cuh"
#include "apd_cost.cuh"
#include "apd_fp32_tile.cuh"

namespace apd {
namespace {

constexpr int kBHist = 16;          // L-BFGS slots per instance (history <= kBHist - 1)
constexpr int kBSortMax = 4096;     // padded seed counts Morton-sorted in shared memory
constexpr int kPrepThreads = 512;
constexpr int kSolveThreads = 256;
constexpr int kRescoreBlocksPerSM = 4;  // CTAs per SM of the persistent rescoring launch
constexpr int kBMaxCount = 50000;   // instances per batch (scheduler table in shared memory)

// solver phases
// PH_INIT_PRED / PH_INIT_ZERO: the two first evaluations of a warm-started
// solve (at the predicted weights, then at zero; the larger g~ is the start).
enum : int {
    PH_INIT = 0, PH_BRACKET = 1, PH_ZOOM = 2, PH_ACCEPT_EVAL = 3, PH_DONE = 4, PH_EVAL_ONLY = 5,
    PH_INIT_PRED = 6, PH_INIT_ZERO = 7
};
__host__ __device__ constexpr bool in_line_search(int ph) {
    return ph == PH_BRACKET || ph == PH_ZOOM || ph == PH_ACCEPT_EVAL;
}

struct BInst {             // per instance, fixed during a call
    GridDev g;
    int n, n_pad, n_chunks;
    int sorted;            // seeds Morton-ordered for the scan
    long long seed_off;    // first row in the concatenated x / A / w / v
    long long rec_off;     // first padded record
    long long flag_off;    // first slot of the instance's rescoring queue (capacity J)
    int tiles_x, tiles_y, tiles_z, ntiles;
    float R_tile;
    int pad0;
    double measure;        // |Omega|
};

struct BSolve {            // per instance state of Algorithm 2
    int phase, active, status, evals, iters, hist, newest, fails, ls_i, zoom_it;
    double f0, dphi0, t, t_prev, phi_prev, dphi_prev;
    double lo, plo, dlo, hi, phi_hi, dhi;
    double best_t, best_phi, cur_t, gamma;
    double best_err, best_g, last_err, last_g, min_v;
    double f_pred;         // f = -g~ at the predicted weights (warm start)
    long long rescored;
    int used_pred;         // the solve started from the predicted weights
    int pad;
};

struct BSched {
    unsigned next_item;    // queue cursor of the persistent kernel
    unsigned total_items;  // tiles of the active instances
    int n_active;          // active instances this iteration
    int next_active;       // instances still active after this iteration's step
    unsigned rescore_next; // queue cursor of the rescoring kernel
    unsigned pad;
};

struct BParams {
    double eps;
    int max_evals;
    int history;
    int check_volumes;
    int pad;
};

struct BArgs {             // everything the per-iteration kernels touch
    int count, dim;
    int prune;             // FP32 scoring skips seed groups by their bounds
    int pad;
    long long total_n;
    const BInst *inst;
    BSolve *sol;
    DevScalars *scs;
    BSched *sched;
    const BParams *prm;
    const int *order;      // instances by decreasing work
    int *act_list;         // active instances in `order` order
    unsigned *act_start;   // [count + 1] tile prefix over act_list
    const double *x, *A, *v;
    double *W, *Wt, *p, *gf, *gft, *Wbest, *Wout;
    double *S, *Y;         // [kBHist][total_n]
    double *rho;           // [count][kBHist]
    SeedRec *recs, *recs_tmp;
    SeedRec32 *recs32, *recs32s;  // natural order, scan order
    GroupBound *groups;           // [total_rec / 32] bounds of the scan-order groups
    uint32_t *scodes;
    int32_t *perm;
    unsigned long long *mom;  // [total_n][K]
    uint32_t *flags;
    int32_t *flag_gi;            // FP32 best seed of each queued pixel
};

__device__ __forceinline__ int map_bits_dev(int bits) {
    if (bits & ST_NOT_SPD) return APD_ERR_NOT_SPD;
    if (bits & (ST_NONFINITE | ST_BAD_VOLUME)) return APD_ERR_ARG;
    if (bits & ST_TIMEOUT) return APD_ERR_TIMEOUT;
    if (bits & ST_BAD_LABEL) return APD_ERR_CUDA;
    return APD_OK;
}

// ---------------------------------------------------------------------------
// set-up and scheduling
// ---------------------------------------------------------------------------
__global__ void batch_init_kernel(const __grid_constant__ BArgs a, const double *__restrict__ w0, int eval_only,
                                  int judge) {
    const int b = blockIdx.x;
    const BInst &I = a.inst[b];
    for (int i = threadIdx.x; i < I.n; i += blockDim.x) {
        a.Wt[I.seed_off + i] = w0[I.seed_off + i];
        a.Wout[I.seed_off + i] = w0[I.seed_off + i];
        a.Wbest[I.seed_off + i] = w0[I.seed_off + i];
    }
    if (threadIdx.x == 0) {
        BSolve s;
        memset(&s, 0, sizeof s);
        s.phase = eval_only ? PH_EVAL_ONLY : (judge ? PH_INIT_PRED : PH_INIT);
        s.active = 1;
        s.newest = kBHist - 1;
        s.gamma = 1.0;
        s.best_err = __longlong_as_double(0x7ff0000000000000ll);
        s.last_err = s.best_err;
        s.cur_t = -1.0;
        a.sol[b] = s;
        a.scs[b].status = 0;
    }
}

// Active instances (in decreasing-work order) and the prefix sum of their tiles.
__global__ void __launch_bounds__(1024) batch_schedule_kernel(const __grid_constant__ BArgs a) {
    extern __shared__ unsigned sh_tiles[];  // [count]
    for (int k = threadIdx.x; k < a.count; k += blockDim.x) {
        const int b = a.order[k];
        sh_tiles[k] = a.sol[b].active ? (unsigned)a.inst[b].ntiles : 0u;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned acc = 0;
        int m = 0;
        for (int k = 0; k < a.count; ++k) {
            if (sh_tiles[k] == 0u) continue;
            a.act_list[m] = a.order[k];
            a.act_start[m] = acc;
            acc += sh_tiles[k];
            ++m;
        }
        a.act_start[m] = acc;
        a.sched->next_item = 0u;
        a.sched->total_items = acc;
        a.sched->n_active = m;
        a.sched->next_active = 0;
        a.sched->rescore_next = 0u;
    }
}

// Seed records of an active instance at its trial weights Wt (natural order for
// the rescoring, Morton scan order for the scoring), the statistics of the
// rounding bound, and zeroed moments and queue.
template <int D>
__global__ void __launch_bounds__(kPrepThreads) batch_prep_kernel(const __grid_constant__ BArgs a) {
    constexpr int K = moment_width(D);
    extern __shared__ unsigned long long keys[];  // [next pow2 of n_pad] when sorted
    __shared__ double shw[kPrepThreads / 32], shf[kPrepThreads / 32], shl[kPrepThreads / 32];
    const int b = blockIdx.x;
    if (!a.sol[b].active) return;
    const BInst &I = a.inst[b];
    const int n = I.n, n_pad = I.n_pad;
    DevScalars *sc = a.scs + b;
    unsigned long long *mom = a.mom + I.seed_off * K;
    for (int e = threadIdx.x; e < n * K; e += blockDim.x) mom[e] = 0ull;
    const double *x = a.x + I.seed_off * D;
    const double *A = a.A + I.seed_off * D * D;
    const double *w = a.Wt + I.seed_off;
    double wmax = -DBL_MAX, fmx = 0.0, lmn = DBL_MAX;
    for (int i = threadIdx.x; i < n_pad; i += blockDim.x) {
        SeedRec r;
        SeedRec32 r32;
        double wk, fr, lm;
        int bd;
        build_seed<D>(i, n, x, A, w, r, r32, wk, fr, lm, bd);
        if (bd) atomicOr(&sc->status, bd);  // error path only
        if (i < n) {
            wmax = fmax(wmax, wk);
            fmx = fmax(fmx, fr);
            lmn = fmin(lmn, lm);
        }
        a.recs32[I.rec_off + i] = r32;
        if (I.sorted) {
            a.recs_tmp[I.rec_off + i] = r;
            keys[i] = ((unsigned long long)seed_code<D>(I.g, r, i < n) << 32) | (unsigned)i;
        } else {
            a.recs[I.rec_off + i] = r;
            a.recs32s[I.rec_off + i] = r32;
        }
    }
    wmax = warp_max(wmax);
    fmx = warp_max(fmx);
    lmn = warp_min(lmn);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        shw[wid] = wmax;
        shf[wid] = fmx;
        shl[wid] = lmn;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
            shw[0] = fmax(shw[0], shw[k]);
            shf[0] = fmax(shf[0], shf[k]);
            shl[0] = fmin(shl[0], shl[k]);
        }
        sc->flag_count = 0u;
        sc->wref_key = dkey(shw[0]);
        sc->lam_abs_bits = (unsigned long long)__double_as_longlong(shf[0]);
        sc->lam_min_bits = (unsigned long long)__double_as_longlong(shl[0]);
    }
    if (I.sorted) {
        int m = 1;
        while (m < n_pad) m <<= 1;
        for (int i = n_pad + threadIdx.x; i < m; i += blockDim.x) keys[i] = ~0ull - (unsigned long long)i;
        __syncthreads();
        block_bitonic_sort(keys, m);
        for (int i = threadIdx.x; i < n_pad; i += blockDim.x) {
            const unsigned long long k = keys[i];
            const int src = (int)(k & 0xffffffffu);
            a.scodes[I.rec_off + i] = (uint32_t)(k >> 32);
            a.perm[I.rec_off + i] = src;
            a.recs[I.rec_off + i] = a.recs_tmp[I.rec_off + src];
            a.recs32s[I.rec_off + i] = a.recs32[I.rec_off + src];
        }
    }
    // bounds of the scan-order groups of 32 seeds (one warp per group)
    __syncthreads();
    const int ngroups = (n + 31) / 32;
    for (int grp = threadIdx.x >> 5; grp < ngroups; grp += blockDim.x >> 5)
        group_bound_warp<D>(a.recs + I.rec_off, n, grp, a.groups + I.rec_off / 32, shw[0]);
}

// ---------------------------------------------------------------------------
// persistent scoring over the tiles of all active instances
// ---------------------------------------------------------------------------
template <int D, int TX, int P, int TY, int TZ, int MINB>
__global__ void __launch_bounds__(TX *TY *TZ, MINB) batch_assign_kernel(const __grid_constant__ BArgs a) {
    constexpr int K = moment_width(D);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    fp32::SharedLayout<D> &sm = *reinterpret_cast<fp32::SharedLayout<D> *>(smem_raw);
    __shared__ fp32::TileSrc cur;
    __shared__ int txyz[3];
    __shared__ unsigned item_sh;
    fp32::init_shared<D>(sm);
    uint32_t uses[4] = {0u, 0u, 0u, 0u};
    const unsigned total = a.sched->total_items;
    const int n_act = a.sched->n_active;
    for (;;) {
        if (threadIdx.x == 0) item_sh = atomicAdd(&a.sched->next_item, 1u);
        __syncthreads();
        const unsigned item = item_sh;
        if (item >= total) break;
        if (threadIdx.x == 0) {
            int lo = 0, hi = n_act - 1;  // last k with act_start[k] <= item
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (a.act_start[mid] <= item) lo = mid;
                else hi = mid - 1;
            }
            const int b = a.act_list[lo];
            const BInst &I = a.inst[b];
            const unsigned local = item - a.act_start[lo];
            txyz[0] = (int)(local % (unsigned)I.tiles_x);
            const unsigned rest = local / (unsigned)I.tiles_x;
            txyz[1] = (int)(rest % (unsigned)I.tiles_y);
            txyz[2] = (int)(rest / (unsigned)I.tiles_y);
            cur.g = I.g;
            cur.n = I.n;
            cur.n_chunks = I.n_chunks;
            cur.R_tile = I.R_tile;
            cur.recs = a.recs + I.rec_off;
            cur.scodes = I.sorted ? a.scodes + I.rec_off : nullptr;
            cur.perm = I.sorted ? a.perm + I.rec_off : nullptr;
            cur.gmom = a.mom + I.seed_off * K;
            cur.flags = a.flags + I.flag_off;
            cur.flag_gi = a.flag_gi + I.flag_off;
            cur.labels = nullptr;
            cur.sc = a.scs + b;
            cur.groups = a.prune ? a.groups + I.rec_off / 32 : nullptr;
            cur.pairs_scored = nullptr;
            cur.wait_limit = kDefaultWaitPolls;
        }
        __syncthreads();
        if (!fp32::score_tile<D, TX, P, TY, TZ>(sm, cur, txyz[0], txyz[1], txyz[2], uses)) break;
    }
}

// Near-tie rescoring of the queued pixels of all active instances: every warp
// pulls pixels (4 at a time) from one queue over the concatenated per-instance
// queues, so an instance with many queued pixels is spread over the whole GPU.
template <int D>
__global__ void __launch_bounds__(256) batch_rescore_kernel(const __grid_constant__ BArgs a) {
    constexpr int K = moment_width(D);
    extern __shared__ unsigned pre[];  // [n_active + 1] prefix of the queue lengths
    const int n_act = a.sched->n_active;
    for (int k = threadIdx.x; k < n_act; k += blockDim.x) pre[k + 1] = a.scs[a.act_list[k]].flag_count;
    __syncthreads();
    if (threadIdx.x == 0) {
        pre[0] = 0u;
        for (int k = 1; k <= n_act; ++k) pre[k] += pre[k - 1];
    }
    __syncthreads();
    const unsigned total = pre[n_act];
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned it0 = 0;
        if (lane == 0) it0 = atomicAdd(&a.sched->rescore_next, 4u);
        it0 = __shfl_sync(0xffffffffu, it0, 0);
        if (it0 >= total) break;
        const unsigned it1 = min(it0 + 4u, total);
        for (unsigned it = it0; it < it1; ++it) {
            int lo = 0, hi = n_act - 1;  // last k with pre[k] <= it
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (pre[mid] <= it) lo = mid;
                else hi = mid - 1;
            }
            const int b = a.act_list[lo];
            const BInst &I = a.inst[b];
            const unsigned local = it - pre[lo];
            DevScalars *sc = a.scs + b;
            const double wref = dkey_inv(sc->wref_key);
            const float wrh = (float)wref;
            const float wrl = (float)(wref - (double)wrh);
            const RescorePrune pr{a.groups + I.rec_off / 32, a.recs32s + I.rec_off,
                                  I.sorted ? a.perm + I.rec_off : nullptr, (I.n + 31) / 32};
            rescore_pixel<D>(I.g, I.n, a.x + I.seed_off * D, a.A + I.seed_off * D * D, a.Wt + I.seed_off,
                             a.recs32 + I.rec_off, a.flags[I.flag_off + local], a.flag_gi[I.flag_off + local], wrh,
                             wrl, pr, sc, a.mom + I.seed_off * K, nullptr);
        }
    }
}

// eqs. (2.7)-(2.8) per instance; writes grad f = -(v - m|P|) into gft and the
// scalars (g~, max relative error, <grad f, p>, sum v, min v) into the
// instance's DevScalars.  Fixed reduction tree: deterministic.
template <int D>
__global__ void __launch_bounds__(kSolveThreads) batch_dual_kernel(const __grid_constant__ BArgs a) {
    constexpr int K = moment_width(D);
    __shared__ double sh[33];
    const int b = blockIdx.x;
    const BSolve &s = a.sol[b];
    if (!s.active || s.phase == PH_EVAL_ONLY) return;
    const bool with_p = in_line_search(s.phase);
    const BInst &I = a.inst[b];
    const long long off = I.seed_off;
    double gsum = 0.0, emax = 0.0, gp = 0.0, sv = 0.0, vmin = DBL_MAX;
    for (int i = threadIdx.x; i < I.n; i += blockDim.x) {
        const double vi = a.v[off + i], wi = a.Wt[off + i];
        if (!(vi > 0.0) || !isfinite(vi)) atomicOr(&a.scs[b].status, ST_BAD_VOLUME);
        double gr, Q;
        dual_terms<D>(I.g, a.mom + (off + i) * K, vi, a.x + (off + i) * D, a.A + (off + i) * D * D, gr, Q);
        gsum += gr * wi + I.g.cell * Q;
        emax = fmax(emax, __ddiv_rn(fabs(gr), vi));
        a.gft[off + i] = -gr;
        if (with_p) gp += -gr * a.p[off + i];
        sv += vi;
        vmin = fmin(vmin, vi);
    }
    const double G = block_sum(gsum, sh);
    const double GP = block_sum(gp, sh);
    const double SV = block_sum(sv, sh);
    __shared__ double shm[kSolveThreads / 32], shn[kSolveThreads / 32];
    const double em = warp_max(emax), vm = warp_min(vmin);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        shm[wid] = em;
        shn[wid] = vm;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double mx = 0.0, mn = DBL_MAX;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            mx = fmax(mx, shm[k]);
            mn = fmin(mn, shn[k]);
        }
        DevScalars *sc = a.scs + b;
        sc->g = G;
        sc->max_rel_err = mx;
        sc->dot_gp = GP;
        sc->sum_v = SV;
        sc->min_v = mn;
    }
}

// ---------------------------------------------------------------------------
// Algorithm 2 on the device: one transition per evaluation
// ---------------------------------------------------------------------------
// Every thread of the CTA runs the same scalar logic on its own copy of the
// state (all inputs are identical, so the copies agree); vector work is split
// by index (thread t owns i = t, t + blockDim, ...), so only the reductions
// synchronise.  The transitions reproduce the host solver of the one-instance
// path: strong-Wolfe line search (c1 = 1e-4, c2 = 0.9, expansion x4, cubic
// zoom with safeguards) on f = -g~, two-loop recursion, curvature-pair skip,
// best-iterate fallback, stop at the first evaluation with max rel err < eps.
struct SolveCtx {
    const BArgs &a;
    const BInst &I;
    BSolve &s;
    double *sh;
    int b, n, history;
    long long off;
    double *W, *Wt, *p, *gf, *gft, *Wbest, *Wout, *rho;

    __device__ void copy(double *dst, const double *src) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
    }
    __device__ void set_trial(double t) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) Wt[i] = W[i] + t * p[i];
        s.cur_t = t;
        s.active = 1;
    }
    __device__ void finish(int status, const double *src) {
        copy(Wout, src);
        s.status = status;
        s.phase = PH_DONE;
        s.active = 0;
    }
    // p = -H gf (two-loop recursion, H0 = gamma I); returns <gf, p>
    __device__ double direction() {
        double al[kBHist];
        for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = gf[i];
        for (int k = 0; k < s.hist; ++k) {
            const int idx = (s.newest - k + kBHist) % kBHist;
            const double *sk = a.S + (size_t)idx * a.total_n + off;
            const double *yk = a.Y + (size_t)idx * a.total_n + off;
            double d = 0.0;
            for (int i = threadIdx.x; i < n; i += blockDim.x) d += sk[i] * p[i];
            al[idx] = rho[idx] * block_sum(d, sh);
            for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] -= al[idx] * yk[i];
        }
        for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] *= s.gamma;
        for (int k = s.hist - 1; k >= 0; --k) {
            const int idx = (s.newest - k + kBHist) % kBHist;
            const double *sk = a.S + (size_t)idx * a.total_n + off;
            const double *yk = a.Y + (size_t)idx * a.total_n + off;
            double d = 0.0;
            for (int i = threadIdx.x; i < n; i += blockDim.x) d += yk[i] * p[i];
            const double bta = rho[idx] * block_sum(d, sh);
            for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] += sk[i] * (al[idx] - bta);
        }
        double d = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            p[i] = -p[i];
            d += gf[i] * p[i];
        }
        return block_sum(d, sh);
    }
    // store s = Wt - W, y = gft - gf in the next slot; returns whether it was kept
    __device__ void push_pair() {
        const int slot = (s.newest + 1) % kBHist;
        double *sk = a.S + (size_t)slot * a.total_n + off;
        double *yk = a.Y + (size_t)slot * a.total_n + off;
        double sy = 0.0, yy = 0.0, ss = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const double si = Wt[i] - W[i];
            const double yi = gft[i] - gf[i];
            sk[i] = si;
            yk[i] = yi;
            sy += si * yi;
            yy += yi * yi;
            ss += si * si;
        }
        sy = block_sum(sy, sh);
        yy = block_sum(yy, sh);
        ss = block_sum(ss, sh);
        if (threadIdx.x == 0) rho[slot] = sy != 0.0 ? 1.0 / sy : 0.0;
        __syncthreads();
        if (sy > 1e-12 * sqrt(ss * yy) && yy > 0.0) {
            s.newest = slot;
            s.hist = min(s.hist + 1, history);
            s.gamma = sy / yy;
        }
    }
};

enum : int { NX_NONE = 0, NX_NEWDIR, NX_ACCEPT, NX_LSEND, NX_FAIL, NX_ZOOM, NX_GIVEUP };

__global__ void __launch_bounds__(kSolveThreads) batch_lbfgs_kernel(const __grid_constant__ BArgs a) {
    __shared__ double sh[33];
    const int b = blockIdx.x;
    BSolve s = a.sol[b];
    if (!s.active) return;
    const BInst &I = a.inst[b];
    const BParams prm = *a.prm;
    DevScalars *sc = a.scs + b;
    const long long off = I.seed_off;
    SolveCtx c{a,          I,           s,           sh,          b,          I.n,  prm.history,
               off,        a.W + off,   a.Wt + off,  a.p + off,   a.gf + off, a.gft + off,
               a.Wbest + off, a.Wout + off, a.rho + (size_t)b * kBHist};
    const double c1 = 1e-4, c2 = 0.9;
    const int dim = I.g.dim;

    const int bits = sc->status;
    const double gval = sc->g, err = sc->max_rel_err;
    const double phi = -gval, dphi = sc->dot_gp;
    s.rescored += sc->flag_count;
    __syncthreads();
    int next = NX_NONE;
    double phi_acc = 0.0;
    if (s.phase == PH_EVAL_ONLY) {
        s.active = 0;
        s.phase = PH_DONE;
        s.status = map_bits_dev(bits);
        s.evals += 1;
    } else if (bits) {
        s.evals += 1;
        c.finish(map_bits_dev(bits), c.Wbest);
        if (threadIdx.x == 0) sc->status = 0;
    } else {
        s.evals += 1;
        s.last_g = gval;
        s.last_err = err;
        const bool first = s.phase == PH_INIT || s.phase == PH_INIT_PRED;
        if (first) s.min_v = sc->min_v;
        const bool bad_volumes = first && prm.check_volumes &&
                                 (!(sc->min_v > 0.0) || fabs(sc->sum_v - I.measure) > 1e-9 * I.measure);
        if (err < s.best_err) {
            s.best_err = err;
            s.best_g = gval;
            c.copy(c.Wbest, c.Wt);
        }
        if (bad_volumes) {
            c.finish(APD_ERR_ARG, c.Wt);
        } else if (err < prm.eps) {
            if (in_line_search(s.phase)) s.iters += 1;
            if (s.phase == PH_INIT_PRED) s.used_pred = 1;
            const bool infeasible = I.g.cell > prm.eps * s.min_v / (double)(1 << dim);
            c.finish(infeasible ? APD_WARN_TOL_INFEASIBLE : APD_OK, c.Wt);
        } else if (s.phase == PH_INIT) {
            s.f0 = phi;
            c.copy(c.W, c.Wt);
            c.copy(c.gf, c.gft);
            next = NX_NEWDIR;
        } else if (s.phase == PH_INIT_PRED) {
            // keep the predicted start in W / gf, evaluate zero next
            s.f_pred = phi;
            c.copy(c.W, c.Wt);
            c.copy(c.gf, c.gft);
            for (int i = threadIdx.x; i < c.n; i += blockDim.x) c.Wt[i] = 0.0;
            s.cur_t = -1.0;
            s.phase = PH_INIT_ZERO;
            s.active = 1;
        } else if (s.phase == PH_INIT_ZERO) {
            if (phi <= s.f_pred) {  // g~(0) >= g~(W_pred): the plain start
                c.copy(c.W, c.Wt);
                c.copy(c.gf, c.gft);
                s.f0 = phi;
                s.used_pred = 0;
            } else {
                s.f0 = s.f_pred;
                s.used_pred = 1;
            }
            next = NX_NEWDIR;
        } else if (s.phase == PH_BRACKET) {
            const double t = s.t;
            if (phi > s.f0 + c1 * t * s.dphi0 || (s.ls_i > 0 && phi >= s.phi_prev)) {
                s.lo = s.t_prev, s.plo = s.phi_prev, s.dlo = s.dphi_prev;
                s.hi = t, s.phi_hi = phi, s.dhi = dphi;
                s.zoom_it = 0;
                next = NX_ZOOM;
            } else {
                if (phi < s.best_phi) {
                    s.best_phi = phi;
                    s.best_t = t;
                }
                if (fabs(dphi) <= -c2 * s.dphi0) {
                    phi_acc = phi;
                    next = NX_ACCEPT;
                } else if (dphi >= 0.0) {
                    s.lo = t, s.plo = phi, s.dlo = dphi;
                    s.hi = s.t_prev, s.phi_hi = s.phi_prev, s.dhi = s.dphi_prev;
                    s.zoom_it = 0;
                    next = NX_ZOOM;
                } else {
                    s.t_prev = t;
                    s.phi_prev = phi;
                    s.dphi_prev = dphi;
                    s.t = fmin(4.0 * t, 1e12);
                    s.ls_i += 1;
                    if (s.ls_i >= 30) next = NX_LSEND;
                    else if (s.evals >= prm.max_evals) next = NX_GIVEUP;
                    else c.set_trial(s.t);
                }
            }
        } else if (s.phase == PH_ZOOM) {
            const double tt = s.cur_t;
            bool accepted = false;
            if (phi > s.f0 + c1 * tt * s.dphi0 || phi >= s.plo) {
                s.hi = tt, s.phi_hi = phi, s.dhi = dphi;
            } else {
                if (phi < s.best_phi) {
                    s.best_phi = phi;
                    s.best_t = tt;
                }
                if (fabs(dphi) <= -c2 * s.dphi0) {
                    phi_acc = phi;
                    next = NX_ACCEPT;
                    accepted = true;
                } else {
                    if (dphi * (s.hi - s.lo) >= 0.0) {
                        s.hi = s.lo, s.phi_hi = s.plo, s.dhi = s.dlo;
                    }
                    s.lo = tt, s.plo = phi, s.dlo = dphi;
                }
            }
            if (!accepted) {
                s.zoom_it += 1;
                if (fabs(s.hi - s.lo) <= 1e-14 * fmax(1.0, fabs(s.lo)) || s.zoom_it >= 20) next = NX_LSEND;
                else next = NX_ZOOM;
            }
        } else if (s.phase == PH_ACCEPT_EVAL) {
            phi_acc = phi;
            next = NX_ACCEPT;
        }
    }
    // chained transitions until the next trial point is set or the solve ends
    for (int guard = 0; guard < 16 && next != NX_NONE; ++guard) {
        const int cur = next;
        next = NX_NONE;
        if (cur == NX_ZOOM) {
            if (s.evals >= prm.max_evals) {
                next = NX_GIVEUP;
                continue;
            }
            const double lo = s.lo, hi = s.hi, plo = s.plo, phi_hi = s.phi_hi, dlo = s.dlo, dhi = s.dhi;
            const double lft = fmin(lo, hi), rgt = fmax(lo, hi), wdt = rgt - lft;
            double tt;
            const double d1 = dlo + dhi - 3.0 * (plo - phi_hi) / (lo - hi);
            const double disc = d1 * d1 - dlo * dhi;
            if (disc >= 0.0 && isfinite(disc)) {
                const double d2 = copysign(sqrt(disc), hi - lo);
                const double den = dhi - dlo + 2.0 * d2;
                tt = den != 0.0 ? hi - (hi - lo) * (dhi + d2 - d1) / den : 0.5 * (lft + rgt);
            } else {
                tt = 0.5 * (lft + rgt);
            }
            if (!isfinite(tt) || tt < lft + 0.1 * wdt || tt > rgt - 0.1 * wdt) tt = 0.5 * (lft + rgt);
            s.phase = PH_ZOOM;
            c.set_trial(tt);
        } else if (cur == NX_LSEND) {
            if (s.best_t > 0.0) {
                if (s.cur_t != s.best_t) {
                    s.phase = PH_ACCEPT_EVAL;
                    c.set_trial(s.best_t);
                } else {
                    phi_acc = s.best_phi;
                    next = NX_ACCEPT;
                }
            } else {
                next = NX_FAIL;
            }
        } else if (cur == NX_ACCEPT) {
            s.fails = 0;
            s.iters += 1;
            c.push_pair();
            c.copy(c.W, c.Wt);
            c.copy(c.gf, c.gft);
            s.f0 = phi_acc;
            next = NX_NEWDIR;
        } else if (cur == NX_FAIL) {
            if (s.hist == 0 || ++s.fails > 3) {
                next = NX_GIVEUP;
            } else {
                s.hist = 0;
                s.gamma = 1.0;
                next = NX_NEWDIR;
            }
        } else if (cur == NX_NEWDIR) {
            if (s.evals >= prm.max_evals) {
                next = NX_GIVEUP;
                continue;
            }
            const double gp0 = c.direction();
            if (!(gp0 < 0.0)) {
                if (s.hist == 0) {
                    next = NX_GIVEUP;
                } else {
                    s.hist = 0;
                    s.gamma = 1.0;
                    next = NX_NEWDIR;
                }
                continue;
            }
            double t0 = 1.0;
            if (s.hist == 0) {
                // first step: t0 ~ 1 / H_ii with H_ii ~ D V^(1 - 2/D), V = |Omega| / n
                const double V = I.measure / (double)I.n;
                t0 = 0.5 * pow(V, 2.0 / dim - 1.0) / dim;
            }
            s.phase = PH_BRACKET;
            s.ls_i = 0;
            s.t = t0;
            s.t_prev = 0.0;
            s.phi_prev = s.f0;
            s.dphi_prev = gp0;
            s.dphi0 = gp0;
            s.best_t = 0.0;
            s.best_phi = s.f0;
            c.set_trial(t0);
        } else if (cur == NX_GIVEUP) {
            c.finish(APD_NOT_CONVERGED, c.Wbest);
        }
    }
    if (next != NX_NONE) c.finish(APD_NOT_CONVERGED, c.Wbest);  // guard exhausted (not expected)
    __syncthreads();
    if (threadIdx.x == 0) {
        a.sol[b] = s;
        if (s.active) atomicAdd(&a.sched->next_active, 1);
    }
}

// ---------------------------------------------------------------------------
// tile variants of the persistent kernel
// ---------------------------------------------------------------------------
struct Variant {
    int TX, P, TY, TZ, threads;  // tile (TX P) x TY x TZ
    const void *fn;
    cudaError_t (*launch)(const BArgs &, int grid, size_t smem, cudaStream_t);
};

template <int D, int TX, int P, int TY, int TZ, int MINB>
cudaError_t launch_variant(const BArgs &a, int grid, size_t smem, cudaStream_t st) {
    batch_assign_kernel<D, TX, P, TY, TZ, MINB><<<grid, TX * TY * TZ, smem, st>>>(a);
    return cudaGetLastError();
}

template <int D, int TX, int P, int TY, int TZ, int MINB>
Variant make_variant() {
    return Variant{TX, P, TY, TZ, TX * TY * TZ, (const void *)batch_assign_kernel<D, TX, P, TY, TZ, MINB>,
                   &launch_variant<D, TX, P, TY, TZ, MINB>};
}

// Candidate tiles: compact squares and near-squares (short distances from the
// tile centre keep the rounding bound small and the per-group skips frequent)
// in CTAs of 256 and 128 threads.
const std::vector<Variant> &variants(int dim) {
    static const std::vector<Variant> v2 = {
        make_variant<2, 4, 16, 64, 1, 2>(),  make_variant<2, 2, 16, 128, 1, 2>(), make_variant<2, 8, 16, 32, 1, 2>(),
        make_variant<2, 4, 16, 32, 1, 4>(),  make_variant<2, 2, 16, 64, 1, 4>(),  make_variant<2, 1, 16, 256, 1, 2>()};
    static const std::vector<Variant> v3 = {make_variant<3, 1, 16, 16, 16, 2>(), make_variant<3, 1, 16, 8, 16, 4>(),
                                            make_variant<3, 2, 8, 8, 16, 2>()};
    return dim == 3 ? v3 : v2;
}

}  // namespace
}  // namespace apd

using namespace apd;

struct apd_batch {
    int dim = 0, count = 0, device = 0;
    long long total_n = 0, total_rec = 0, total_j = 0;
    std::vector<GridDev> grids;
    std::vector<apd_grid> src_grids;   // as passed to apd_batch_create
    apd_batch *coarse = nullptr;       // coarse-grid batch of the coarse-to-fine solve
    int coarse_factor = 0;
    std::vector<int> n;
    std::vector<long long> seed_off, rec_off, flag_off;
    std::vector<double> measure;
    std::vector<int> order;
    int variant = -1;                  // chosen tile variant (-1: autotune pending)
    std::vector<double> variant_ms;    // autotune timings
    int grid_blocks = 0, rescore_blocks = 0;
    size_t smem_assign = 0, smem_prep = 0, smem_sched = 0;
    BArgs args{};
    BInst *d_inst = nullptr;
    BSolve *h_sol = nullptr;           // pinned
    BSched *h_sched = nullptr;         // pinned
    BParams *h_prm = nullptr;          // pinned
    double *d_w0 = nullptr;
    void *blocks[32] = {};
    int nblocks = 0;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_variant = -1;
    long long launches = 0;
};

namespace {

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? APD_OK : APD_ERR_CUDA; }

#define BTRY(expr)                     \
    do {                               \
        int _rc = (expr);              \
        if (_rc != APD_OK) return _rc; \
    } while (0)

std::vector<BInst> instance_table(const apd_batch &bt, int vi) {
    const Variant &V = variants(bt.dim)[vi];
    std::vector<BInst> t(bt.count);
    for (int b = 0; b < bt.count; ++b) {
        BInst &I = t[b];
        std::memset(&I, 0, sizeof I);
        I.g = bt.grids[b];
        I.n = bt.n[b];
        I.n_chunks = (I.n + kChunk - 1) / kChunk;
        I.n_pad = I.n_chunks * kChunk;
        I.sorted = I.n_pad <= kBSortMax ? 1 : 0;
        I.seed_off = bt.seed_off[b];
        I.rec_off = bt.rec_off[b];
        I.flag_off = bt.flag_off[b];
        I.tiles_x = (I.g.res[0] + V.TX * V.P - 1) / (V.TX * V.P);
        I.tiles_y = (I.g.res[1] + V.TY - 1) / V.TY;
        I.tiles_z = bt.dim == 3 ? (I.g.res[2] + V.TZ - 1) / V.TZ : 1;
        I.ntiles = I.tiles_x * I.tiles_y * I.tiles_z;
        const double hx = 0.5 * V.TX * V.P * I.g.h[0], hy = 0.5 * V.TY * I.g.h[1];
        const double hz = bt.dim == 3 ? 0.5 * V.TZ * I.g.h[2] : 0.0;
        I.R_tile = (float)(std::sqrt(hx * hx + hy * hy + hz * hz) * (1.0 + 1e-6));
        I.measure = bt.measure[b];
    }
    return t;
}

int use_variant(apd_batch &bt, int vi, cudaStream_t st) {
    const Variant &V = variants(bt.dim)[vi];
    const std::vector<BInst> t = instance_table(bt, vi);
    BTRY(cuda_rc(cudaMemcpyAsync(bt.d_inst, t.data(), t.size() * sizeof(BInst), cudaMemcpyHostToDevice, st)));
    BTRY(cuda_rc(cudaStreamSynchronize(st)));
    const size_t smem = bt.dim == 3 ? sizeof(fp32::SharedLayout<3>) : sizeof(fp32::SharedLayout<2>);
    BTRY(cuda_rc(cudaFuncSetAttribute(V.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)));
    int per_sm = 0, sms = 0;
    BTRY(cuda_rc(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, V.fn, V.threads, smem)));
    BTRY(cuda_rc(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, bt.device)));
    bt.grid_blocks = std::max(1, per_sm) * sms;
    bt.smem_assign = smem;
    return APD_OK;
}

// The per-iteration launches (also the body of the captured graph).
int enqueue_iteration(apd_batch &bt, int vi, bool solve_steps, cudaStream_t st) {
    const Variant &V = variants(bt.dim)[vi];
    const BArgs &a = bt.args;
    batch_schedule_kernel<<<1, 1024, bt.smem_sched, st>>>(a);
    if (bt.dim == 3) batch_prep_kernel<3><<<bt.count, kPrepThreads, bt.smem_prep, st>>>(a);
    else batch_prep_kernel<2><<<bt.count, kPrepThreads, bt.smem_prep, st>>>(a);
    BTRY(cuda_rc(cudaGetLastError()));
    BTRY(cuda_rc(V.launch(a, bt.grid_blocks, bt.smem_assign, st)));
    if (bt.dim == 3) batch_rescore_kernel<3><<<bt.rescore_blocks, 256, bt.smem_sched + 4, st>>>(a);
    else batch_rescore_kernel<2><<<bt.rescore_blocks, 256, bt.smem_sched + 4, st>>>(a);
    bt.launches += 4;
    if (solve_steps) {
        if (bt.dim == 3) batch_dual_kernel<3><<<bt.count, kSolveThreads, 0, st>>>(a);
        else batch_dual_kernel<2><<<bt.count, kSolveThreads, 0, st>>>(a);
        batch_lbfgs_kernel<<<bt.count, kSolveThreads, 0, st>>>(a);
        bt.launches += 2;
    }
    return cuda_rc(cudaGetLastError());
}

int load_inputs(apd_batch &bt, const double *x, const double *A, const double *w, const double *v,
                cudaStream_t st) {
    const size_t N = (size_t)bt.total_n, D = (size_t)bt.dim;
    BTRY(cuda_rc(cudaMemcpyAsync((void *)bt.args.x, x, N * D * sizeof(double), cudaMemcpyDeviceToDevice, st)));
    BTRY(cuda_rc(cudaMemcpyAsync((void *)bt.args.A, A, N * D * D * sizeof(double), cudaMemcpyDeviceToDevice, st)));
    BTRY(cuda_rc(cudaMemcpyAsync(bt.d_w0, w, N * sizeof(double), cudaMemcpyDeviceToDevice, st)));
    if (v) BTRY(cuda_rc(cudaMemcpyAsync((void *)bt.args.v, v, N * sizeof(double), cudaMemcpyDeviceToDevice, st)));
    return APD_OK;
}

int init_solves(apd_batch &bt, bool eval_only, cudaStream_t st, bool judge = false) {
    batch_init_kernel<<<bt.count, 256, 0, st>>>(bt.args, bt.d_w0, eval_only ? 1 : 0, judge ? 1 : 0);
    bt.launches += 1;
    return cuda_rc(cudaGetLastError());
}

// Times every tile variant on the loaded inputs (one scoring pass each after a
// warm-up) and keeps the fastest.
int autotune(apd_batch &bt, cudaStream_t st) {
    const auto &vs = variants(bt.dim);
    bt.variant_ms.assign(vs.size(), 0.0);
    cudaEvent_t e0, e1;
    BTRY(cuda_rc(cudaEventCreate(&e0)));
    BTRY(cuda_rc(cudaEventCreate(&e1)));
    int best = 0;
    for (int vi = 0; vi < (int)vs.size(); ++vi) {
        BTRY(use_variant(bt, vi, st));
        float best_ms = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            BTRY(init_solves(bt, true, st));
            batch_schedule_kernel<<<1, 1024, bt.smem_sched, st>>>(bt.args);
            if (bt.dim == 3) batch_prep_kernel<3><<<bt.count, kPrepThreads, bt.smem_prep, st>>>(bt.args);
            else batch_prep_kernel<2><<<bt.count, kPrepThreads, bt.smem_prep, st>>>(bt.args);
            BTRY(cuda_rc(cudaEventRecord(e0, st)));
            BTRY(cuda_rc(vs[vi].launch(bt.args, bt.grid_blocks, bt.smem_assign, st)));
            BTRY(cuda_rc(cudaEventRecord(e1, st)));
            BTRY(cuda_rc(cudaEventSynchronize(e1)));
            float ms = 0.f;
            BTRY(cuda_rc(cudaEventElapsedTime(&ms, e0, e1)));
            bt.launches += 4;
            if (rep > 0) best_ms = std::min(best_ms, ms);
        }
        bt.variant_ms[vi] = best_ms;
        if (best_ms < bt.variant_ms[best]) best = vi;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    bt.variant = best;
    return use_variant(bt, best, st);
}

int capture_graph(apd_batch &bt) {
    if (bt.exec && bt.graph_variant == bt.variant) return APD_OK;
    if (bt.exec) cudaGraphExecDestroy(bt.exec);
    if (bt.graph) cudaGraphDestroy(bt.graph);
    bt.exec = nullptr;
    bt.graph = nullptr;
    BTRY(cuda_rc(cudaStreamBeginCapture(bt.cap, cudaStreamCaptureModeThreadLocal)));
    const long long before = bt.launches;
    const int rc = enqueue_iteration(bt, bt.variant, true, bt.cap);
    bt.launches = before;
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(bt.cap, &g);
    if (rc != APD_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    BTRY(cuda_rc(e));
    bt.graph = g;
    BTRY(cuda_rc(cudaGraphInstantiate(&bt.exec, bt.graph, 0)));
    bt.graph_variant = bt.variant;
    return APD_OK;
}

int prepare(apd_batch &bt, cudaStream_t st) {
    if (bt.variant < 0) BTRY(autotune(bt, st));
    return APD_OK;
}

}  // namespace

extern "C" {

int apd_batch_create(apd_batch **out, int32_t dim, int32_t count, const apd_grid *grids, const int32_t *n,
                     int32_t tile) {
    if (!out) return APD_ERR_ARG;
    *out = nullptr;
    if ((dim != 2 && dim != 3) || count < 1 || count > kBMaxCount || !grids || !n) return APD_ERR_ARG;
    const int nv = (int)variants(dim).size();
    if (tile < -1 || tile >= nv) return APD_ERR_ARG;
    apd_batch *bt = new (std::nothrow) apd_batch();
    if (!bt) return APD_ERR_CUDA;
    bt->dim = dim;
    bt->count = count;
    cudaGetDevice(&bt->device);
    bt->grids.resize(count);
    bt->src_grids.assign(grids, grids + count);
    bt->n.resize(count);
    bt->seed_off.resize(count);
    bt->rec_off.resize(count);
    bt->flag_off.resize(count);
    bt->measure.resize(count);
    long long so = 0, ro = 0, fo = 0, maxpad = 0;
    for (int b = 0; b < count; ++b) {
        if (grids[b].dim != dim || n[b] < 1 || validate_grid(&grids[b], bt->grids[b]) != APD_OK) {
            delete bt;
            return APD_ERR_ARG;
        }
        bt->n[b] = n[b];
        bt->seed_off[b] = so;
        bt->rec_off[b] = ro;
        bt->flag_off[b] = fo;
        bt->measure[b] = domain_measure(&grids[b]);
        const long long pad = (long long)((n[b] + kChunk - 1) / kChunk) * kChunk;
        maxpad = std::max(maxpad, pad);
        so += n[b];
        ro += pad;
        fo += bt->grids[b].J;
    }
    bt->total_n = so;
    bt->total_rec = ro;
    bt->total_j = fo;
    bt->order.resize(count);
    std::iota(bt->order.begin(), bt->order.end(), 0);
    std::stable_sort(bt->order.begin(), bt->order.end(), [&](int p, int q) {
        return (double)bt->n[p] * (double)bt->grids[p].J > (double)bt->n[q] * (double)bt->grids[q].J;
    });
    int m = 1;  // keys of the largest instance that is sorted in shared memory
    while (m < maxpad && m < kBSortMax) m <<= 1;
    bt->smem_prep = (size_t)m * sizeof(unsigned long long);
    bt->smem_sched = (size_t)count * sizeof(unsigned);

    const size_t N = (size_t)so, D = (size_t)dim, K = (size_t)moment_width(dim);
    bool ok = true;
    auto alloc = [&](void **p, size_t bytes) {
        if (!ok) return;
        if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
            ok = false;
            return;
        }
        bt->blocks[bt->nblocks++] = *p;
    };
    BArgs &a = bt->args;
    a.count = count;
    a.dim = dim;
    a.total_n = so;
    alloc((void **)&bt->d_inst, count * sizeof(BInst));
    a.inst = bt->d_inst;
    alloc((void **)&a.sol, count * sizeof(BSolve));
    alloc((void **)&a.scs, count * sizeof(DevScalars));
    alloc((void **)&a.sched, sizeof(BSched));
    alloc((void **)&a.prm, sizeof(BParams));
    alloc((void **)&a.order, count * sizeof(int));
    alloc((void **)&a.act_list, count * sizeof(int));
    alloc((void **)&a.act_start, (count + 1) * sizeof(unsigned));
    alloc((void **)&a.x, N * D * sizeof(double));
    alloc((void **)&a.A, N * D * D * sizeof(double));
    alloc((void **)&a.v, N * sizeof(double));
    alloc((void **)&bt->d_w0, N * sizeof(double));
    double **vecs[] = {&a.W, &a.Wt, &a.p, &a.gf, &a.gft, &a.Wbest, &a.Wout};
    for (double **pp : vecs) alloc((void **)pp, N * sizeof(double));
    alloc((void **)&a.S, (size_t)kBHist * N * sizeof(double));
    alloc((void **)&a.Y, (size_t)kBHist * N * sizeof(double));
    alloc((void **)&a.rho, (size_t)count * kBHist * sizeof(double));
    alloc((void **)&a.recs, (size_t)ro * sizeof(SeedRec));
    alloc((void **)&a.recs_tmp, (size_t)ro * sizeof(SeedRec));
    alloc((void **)&a.recs32, (size_t)ro * sizeof(SeedRec32));
    alloc((void **)&a.recs32s, (size_t)ro * sizeof(SeedRec32));
    alloc((void **)&a.groups, (size_t)(ro / 32) * sizeof(GroupBound));
    alloc((void **)&a.scodes, (size_t)ro * sizeof(uint32_t));
    alloc((void **)&a.perm, (size_t)ro * sizeof(int32_t));
    alloc((void **)&a.mom, N * K * sizeof(unsigned long long));
    alloc((void **)&a.flags, (size_t)fo * sizeof(uint32_t));
    alloc((void **)&a.flag_gi, (size_t)fo * sizeof(int32_t));
    if (ok && cudaMallocHost((void **)&bt->h_sol, count * sizeof(BSolve)) != cudaSuccess) ok = false;
    if (ok && cudaMallocHost((void **)&bt->h_sched, sizeof(BSched)) != cudaSuccess) ok = false;
    if (ok && cudaMallocHost((void **)&bt->h_prm, sizeof(BParams)) != cudaSuccess) ok = false;
    if (ok && cudaStreamCreateWithFlags(&bt->cap, cudaStreamNonBlocking) != cudaSuccess) ok = false;
    if (ok && cudaMemset(a.scs, 0, count * sizeof(DevScalars)) != cudaSuccess) ok = false;
    if (ok && cudaMemset(a.sol, 0, count * sizeof(BSolve)) != cudaSuccess) ok = false;
    if (ok && cudaMemset(a.recs, 0, (size_t)ro * sizeof(SeedRec)) != cudaSuccess) ok = false;
    if (ok && cudaMemcpy((void *)a.order, bt->order.data(), count * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
        ok = false;
    if (ok && dim == 3 &&
        cudaFuncSetAttribute(batch_prep_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bt->smem_prep) !=
            cudaSuccess)
        ok = false;
    if (ok && dim == 2 &&
        cudaFuncSetAttribute(batch_prep_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bt->smem_prep) !=
            cudaSuccess)
        ok = false;
    if (ok && cudaFuncSetAttribute(batch_schedule_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)bt->smem_sched) != cudaSuccess)
        ok = false;
    if (ok && cudaFuncSetAttribute(dim == 3 ? (const void *)batch_rescore_kernel<3> : (const void *)batch_rescore_kernel<2>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bt->smem_sched + 4) != cudaSuccess)
        ok = false;
    int sms = 0;
    if (ok && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, bt->device) != cudaSuccess) ok = false;
    bt->rescore_blocks = std::max(1, sms) * kRescoreBlocksPerSM;
    if (ok && tile >= 0) {
        bt->variant = tile;
        if (use_variant(*bt, tile, nullptr) != APD_OK) ok = false;
    }
    if (ok && cudaDeviceSynchronize() != cudaSuccess) ok = false;
    if (!ok) {
        apd_batch_destroy(bt);
        return APD_ERR_CUDA;
    }
    *out = bt;
    return APD_OK;
}

void apd_batch_destroy(apd_batch *bt) {
    if (!bt) return;
    apd_batch_destroy(bt->coarse);
    if (bt->exec) cudaGraphExecDestroy(bt->exec);
    if (bt->graph) cudaGraphDestroy(bt->graph);
    if (bt->cap) cudaStreamDestroy(bt->cap);
    for (int k = 0; k < bt->nblocks; ++k) cudaFree(bt->blocks[k]);
    if (bt->h_sol) cudaFreeHost(bt->h_sol);
    if (bt->h_sched) cudaFreeHost(bt->h_sched);
    if (bt->h_prm) cudaFreeHost(bt->h_prm);
    delete bt;
}

int apd_batch_tile_info(apd_batch *bt, int32_t *tile, int32_t *n_variants, double *ms, int32_t *shape) {
    if (!bt) return APD_ERR_ARG;
    const auto &vs = variants(bt->dim);
    if (tile) *tile = bt->variant;
    if (n_variants) *n_variants = (int32_t)vs.size();
    for (int k = 0; k < (int)vs.size(); ++k) {
        if (ms) ms[k] = k < (int)bt->variant_ms.size() ? bt->variant_ms[k] : -1.0;
        if (shape) {
            shape[3 * k] = vs[k].TX * vs[k].P;
            shape[3 * k + 1] = vs[k].TY;
            shape[3 * k + 2] = vs[k].TZ;
        }
    }
    return APD_OK;
}

int64_t apd_batch_kernel_launches(apd_batch *bt) { return bt ? bt->launches : -1; }

int apd_batch_set_pruning(apd_batch *bt, int32_t enable) {
    if (!bt) return APD_ERR_ARG;
    const int want = enable != 0;
    if (bt->args.prune != want) {
        bt->args.prune = want;
        // the captured graph holds the old argument block
        if (bt->exec) cudaGraphExecDestroy(bt->exec);
        if (bt->graph) cudaGraphDestroy(bt->graph);
        bt->exec = nullptr;
        bt->graph = nullptr;
        bt->graph_variant = -1;
    }
    if (bt->coarse) apd_batch_set_pruning(bt->coarse, enable);
    return APD_OK;
}

int apd_batch_cell_moments(apd_batch *bt, const double *x, const double *A, const double *w, int64_t *moments,
                           apd_stream_t stream) {
    if (!bt || !x || !A || !w || !moments) return APD_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    BTRY(load_inputs(*bt, x, A, w, nullptr, st));
    BTRY(prepare(*bt, st));
    BTRY(init_solves(*bt, true, st));
    BTRY(enqueue_iteration(*bt, bt->variant, false, st));
    const size_t K = (size_t)moment_width(bt->dim);
    BTRY(cuda_rc(cudaMemcpyAsync(moments, bt->args.mom, (size_t)bt->total_n * K * sizeof(int64_t),
                                 cudaMemcpyDeviceToDevice, st)));
    std::vector<DevScalars> sc(bt->count);
    BTRY(cuda_rc(cudaMemcpyAsync(sc.data(), bt->args.scs, bt->count * sizeof(DevScalars), cudaMemcpyDeviceToHost, st)));
    BTRY(cuda_rc(cudaStreamSynchronize(st)));
    int bits = 0;
    for (const DevScalars &s : sc) bits |= s.status;
    if (bits) {
        BTRY(cuda_rc(cudaMemset(bt->args.scs, 0, bt->count * sizeof(DevScalars))));
        return map_bits(bits);
    }
    return APD_OK;
}

static int batch_solve(apd_batch *bt, const double *x, const double *A, const double *w0, const double *v,
                       double *w_out, const apd_solve_opts *opts, apd_solve_info *info, int32_t *used,
                       bool judge, apd_stream_t stream) {
    if (!bt || !x || !A || !w0 || !v || !w_out) return APD_ERR_ARG;
    apd_solve_opts o;
    apd_solve_opts_default(&o);
    if (opts) o = *opts;
    if (!(o.eps > 0.0) || o.max_evals < 1 || o.history < 1) return APD_ERR_ARG;
    if (o.precision != APD_FP32) return APD_ERR_UNSUPPORTED;
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t st = (cudaStream_t)stream;
    BTRY(load_inputs(*bt, x, A, w0, v, st));
    bt->h_prm->eps = o.eps;
    bt->h_prm->max_evals = o.max_evals;
    bt->h_prm->history = std::max(1, std::min(o.history, kBHist - 1));
    bt->h_prm->check_volumes = o.check_volumes != 0;
    BTRY(cuda_rc(cudaMemcpyAsync((void *)bt->args.prm, bt->h_prm, sizeof(BParams), cudaMemcpyHostToDevice, st)));
    BTRY(prepare(*bt, st));
    BTRY(capture_graph(*bt));
    BTRY(init_solves(*bt, false, st, judge));
    // Each replay is one evaluation of every active instance; a finished batch
    // replays as six near-empty launches, so the host polls every few replays.
    const int max_iters = o.max_evals + 8;
    int iters = 0;
    for (;;) {
        const int burst = iters < 8 ? 2 : 8;
        for (int r = 0; r < burst; ++r) {
            BTRY(cuda_rc(cudaGraphLaunch(bt->exec, st)));
            bt->launches += 6;
        }
        iters += burst;
        BTRY(cuda_rc(cudaMemcpyAsync(bt->h_sched, bt->args.sched, sizeof(BSched), cudaMemcpyDeviceToHost, st)));
        BTRY(cuda_rc(cudaStreamSynchronize(st)));
        if (bt->h_sched->next_active == 0 || iters >= max_iters) break;
    }
    BTRY(cuda_rc(cudaMemcpyAsync(w_out, bt->args.Wout, (size_t)bt->total_n * sizeof(double),
                                 cudaMemcpyDeviceToDevice, st)));
    BTRY(cuda_rc(cudaMemcpyAsync(bt->h_sol, bt->args.sol, bt->count * sizeof(BSolve), cudaMemcpyDeviceToHost, st)));
    BTRY(cuda_rc(cudaStreamSynchronize(st)));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    int err = APD_OK;
    bool any_nc = false, any_warn = false;
    for (int b = 0; b < bt->count; ++b) {
        const BSolve &s = bt->h_sol[b];
        const int status = s.phase == PH_DONE ? s.status : APD_NOT_CONVERGED;
        if (info) {
            apd_solve_info &inf = info[b];
            std::memset(&inf, 0, sizeof inf);
            inf.status = status;
            inf.iterations = s.iters;
            inf.evaluations = s.evals;
            inf.solves = 1;
            const bool conv = status == APD_OK || status == APD_WARN_TOL_INFEASIBLE;
            inf.max_rel_err = conv ? s.last_err : s.best_err;
            inf.g = conv ? s.last_g : s.best_g;
            inf.rescored_fp64 = s.rescored;
            inf.seconds = secs;
        }
        if (used) used[b] = s.used_pred;
        if (status < 0 && err == APD_OK) err = status;
        any_nc |= status == APD_NOT_CONVERGED;
        any_warn |= status == APD_WARN_TOL_INFEASIBLE;
    }
    if (err != APD_OK) return err;
    return any_nc ? APD_NOT_CONVERGED : (any_warn ? APD_WARN_TOL_INFEASIBLE : APD_OK);
}

int apd_batch_solve_weights(apd_batch *bt, const double *x, const double *A, const double *w0, const double *v,
                            double *w_out, const apd_solve_opts *opts, apd_solve_info *info, apd_stream_t stream) {
    return batch_solve(bt, x, A, w0, v, w_out, opts, info, nullptr, false, stream);
}

int apd_batch_solve_weights_judged(apd_batch *bt, const double *x, const double *A, const double *w_pred,
                                   const double *v, double *w_out, const apd_solve_opts *opts, apd_solve_info *info,
                                   int32_t *used_pred, apd_stream_t stream) {
    return batch_solve(bt, x, A, w_pred, v, w_out, opts, info, used_pred, true, stream);
}

int apd_batch_solve_weights_multires(apd_batch *bt, const double *x, const double *A, const double *w0,
                                     const double *v, double *w_out, const apd_solve_opts *opts,
                                     const apd_multires_opts *mo, int32_t judge, apd_solve_info *info,
                                     int32_t *used_pred, apd_stream_t stream) {
    if (!bt || !x || !A || !w0 || !v || !w_out) return APD_ERR_ARG;
    const auto t0 = std::chrono::steady_clock::now();
    apd_multires_opts m;
    apd_multires_opts_default(&m);
    if (mo) m = *mo;
    if (m.factor < 2 || !(m.coarse_eps > 0.0) || m.coarse_max_evals < 1) return APD_ERR_ARG;
    apd_solve_opts o;
    apd_solve_opts_default(&o);
    if (opts) o = *opts;
    if (!bt->coarse || bt->coarse_factor != m.factor) {
        apd_batch_destroy(bt->coarse);
        bt->coarse = nullptr;
        std::vector<apd_grid> cg = bt->src_grids;
        for (apd_grid &g : cg)
            for (int d = 0; d < g.dim; ++d) g.res[d] = std::max(4, (g.res[d] + m.factor - 1) / m.factor);
        const int rc = apd_batch_create(&bt->coarse, bt->dim, bt->count, cg.data(), bt->n.data(), -1);
        if (rc != APD_OK) return rc;
        apd_batch_set_pruning(bt->coarse, bt->args.prune);
        bt->coarse_factor = m.factor;
    }
    apd_solve_opts oc = o;
    oc.eps = m.coarse_eps;
    oc.max_evals = m.coarse_max_evals;
    std::vector<apd_solve_info> ci(bt->count);
    // the coarse weights land in w_out and are the fine solve's start (inputs are
    // copied into the batch before anything is written, so w0 may alias w_out)
    int rc = batch_solve(bt->coarse, x, A, w0, v, w_out, &oc, ci.data(), used_pred, judge != 0, stream);
    if (rc < 0) return rc;
    rc = batch_solve(bt, x, A, w_out, v, w_out, &o, info, nullptr, false, stream);
    bt->launches += bt->coarse->launches;
    bt->coarse->launches = 0;
    if (info)
        for (int b = 0; b < bt->count; ++b) {
            info[b].coarse_evaluations = ci[b].evaluations;
            info[b].solves += 1;
            info[b].rescored_fp64 += ci[b].rescored_fp64;
            info[b].seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        }
    return rc;
}

}  // extern "C"
