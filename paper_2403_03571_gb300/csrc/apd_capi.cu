// Host side of the C ABI declared in include/apd.h: argument validation,
// workspace management, the stream-ordered evaluation sequence (Algorithm 1 +
// moments + eqs. (2.7)-(2.8)), the L-BFGS weight solve of Algorithm 2 and the
// Lloyd loop of Algorithm 3.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <utility>

#include "apd_internal.cuh"

struct apd_workspace {
    apd::Workspace w;
};

using namespace apd;

namespace apd {

int map_bits(int bits) {
    if (bits & ST_NOT_SPD) return APD_ERR_NOT_SPD;
    if (bits & (ST_NONFINITE | ST_BAD_VOLUME)) return APD_ERR_ARG;
    if (bits & ST_TIMEOUT) return APD_ERR_TIMEOUT;
    if (bits & ST_BAD_LABEL) return APD_ERR_CUDA;
    return APD_OK;
}

int validate_grid(const apd_grid *gr, GridDev &g) {
    if (!gr) return APD_ERR_ARG;
    if (gr->dim != 2 && gr->dim != 3) return APD_ERR_ARG;
    std::memset(&g, 0, sizeof g);
    g.dim = gr->dim;
    long long J = 1;
    double cell = 1.0;
    for (int d = 0; d < 3; ++d) {
        if (d < gr->dim) {
            if (gr->res[d] < 1) return APD_ERR_ARG;
            if (!std::isfinite(gr->lo[d]) || !std::isfinite(gr->hi[d]) || !(gr->hi[d] > gr->lo[d]))
                return APD_ERR_ARG;
            g.res[d] = gr->res[d];
            g.lo[d] = gr->lo[d];
            g.h[d] = (gr->hi[d] - gr->lo[d]) / (double)gr->res[d];
            g.h32[d] = (float)g.h[d];
            J *= gr->res[d];
            cell *= g.h[d];
            if (J >= (1ll << 31)) return APD_ERR_ARG;
        } else {
            g.res[d] = 1;
            g.lo[d] = 0.0;
            g.h[d] = 1.0;
            g.h32[d] = 1.f;
        }
    }
    g.J = J;
    g.cell = cell;
    return APD_OK;
}

void shard_range(int res, int rank, int world, int &k_begin, int &k_count) {
    const long long b = (long long)res * rank / world, e = (long long)res * (rank + 1) / world;
    k_begin = (int)b;
    k_count = (int)(e - b);
}

double domain_measure(const apd_grid *gr) {
    double m = 1.0;
    for (int d = 0; d < gr->dim; ++d) m *= gr->hi[d] - gr->lo[d];
    return m;
}

}  // namespace apd

namespace {

constexpr int kHistCap = 32;

int validate_seeds(const apd_seeds *s) {
    if (!s || s->n < 1 || !s->x || !s->A || !s->w) return APD_ERR_ARG;
    return APD_OK;
}

// The workspace holds n seeds and the pixels of one scoring pass: the whole
// grid, or this rank's slab when the workspace is sharded.
int check_ws(const apd_workspace *ws, const GridDev &g, int n) {
    if (!ws) return APD_ERR_ARG;
    long long pix = g.J;
    if (ws->w.shard_world > 1) {
        int kb = 0, kc = 0;
        shard_range(g.res[g.dim - 1], ws->w.shard_rank, ws->w.shard_world, kb, kc);
        pix = g.J / g.res[g.dim - 1] * (long long)kc;
    }
    if (ws->w.dim != g.dim || n > ws->w.max_n || pix > ws->w.max_j) return APD_ERR_WORKSPACE;
    return APD_OK;
}

int cuda_ok(cudaError_t e) { return e == cudaSuccess ? APD_OK : APD_ERR_CUDA; }

#define APD_TRY(expr)                  \
    do {                               \
        int _rc = (expr);              \
        if (_rc != APD_OK) return _rc; \
    } while (0)

// Algorithm 1 + moments (+ FP64 rescoring of near ties) on `st`.
// A trial point W + t p of the weight solve, written to the evaluated weights.
struct TrialStep {
    const double *W;
    double t;
    const double *p;
};

constexpr size_t kGraphCap = 16;  // evaluation graphs kept per workspace

void destroy_graph(EvalGraph &e) {
    if (e.exec) cudaGraphExecDestroy(e.exec);
    if (e.graph) cudaGraphDestroy(e.graph);
    if (e.e0) cudaEventDestroy(e.e0);
    if (e.e1) cudaEventDestroy(e.e1);
    e = EvalGraph();
}

// Whether a pass scores with the tensor-core kernel: asked for, a grid the
// workspace's tile scratch covers, and seeds conditioned well enough for its
// certificate and candidate bounds (max ||A||_F / min lambda_min <= kTcMaxCond;
// beyond that the FP32 kernel is faster and gives the same labels: measured on
// the runtime tests' 3D alpha laws, the tensor-core form wins at ratios up to
// 7.4 and loses 3.6x at 11.7).  The
// conditioning comes from the seed preparation: read back once per preparation
// (a stream synchronisation); passes that reuse the records reuse the value.
constexpr double kTcMaxCond = 10.0;
bool use_tensor_cores(const GridDev &g, apd_precision prec, Workspace &ws, bool weights_only, cudaStream_t st) {
    if (prec == APD_FP32 || tc_tile_count(g) > ws.tc_tile_cap) return false;
    if (!weights_only) {
        unsigned long long bits[2] = {0ull, 0ull};  // lam_abs_bits, lam_min_bits
        if (cudaMemcpyAsync(&ws.sc_host->lam_abs_bits, &ws.sc->lam_abs_bits, 2 * sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, st) == cudaSuccess &&
            cudaStreamSynchronize(st) == cudaSuccess) {
            bits[0] = ws.sc_host->lam_abs_bits;
            bits[1] = ws.sc_host->lam_min_bits;
        }
        double lam_abs = 0.0, lam_min = 0.0;
        std::memcpy(&lam_abs, &bits[0], sizeof lam_abs);
        std::memcpy(&lam_min, &bits[1], sizeof lam_min);
        ws.tc_cond = lam_min > 0.0 ? lam_abs / lam_min : INFINITY;
    }
    return ws.tc_cond <= kTcMaxCond;
}

// Incremental passes (weight solves, pruned tensor-core scorer, one rank).  A
// pass queued with kIncAuto either re-decides from the solve's record or
// records afresh; the trial-weights kernel chooses on the device (sc->inc_go):
// a re-decision when a record exists and at most kIncFullMax of the pixels can
// need a full one (see tc_band_kernel).  The first pass of a solve records.
constexpr int kIncNone = 0, kIncAuto = 1;
constexpr double kIncFullMax = 0.08;
// Below this many pixels a full pass costs about as much as the three extra
// launches of an incremental one (apd_workspace_set_incremental mode 1).
constexpr long long kIncMinPixels = 1ll << 20;

// The buffers of the incremental passes, allocated on first use (never inside a
// graph capture).
static int inc_alloc(Workspace &ws) {
    if (ws.inc_labels) return APD_OK;
    const size_t K = (size_t)moment_width(ws.dim);
    bool ok = cudaMalloc((void **)&ws.inc_labels, (size_t)ws.max_j * sizeof(int32_t)) == cudaSuccess &&
              cudaMalloc((void **)&ws.inc_gap, (size_t)ws.max_j * sizeof(float)) == cudaSuccess &&
              cudaMalloc((void **)&ws.inc_rec, (size_t)ws.max_j * sizeof(float4)) == cudaSuccess &&
              cudaMalloc((void **)&ws.inc_hist, kIncBins * sizeof(unsigned)) == cudaSuccess &&
              cudaMalloc((void **)&ws.inc_drift, (size_t)ws.max_n * sizeof(float2)) == cudaSuccess &&
              cudaMalloc((void **)&ws.inc_mom0, (size_t)ws.max_n * K * sizeof(unsigned long long)) == cudaSuccess &&
              cudaMalloc((void **)&ws.inc_w0, (size_t)ws.max_n * sizeof(double)) == cudaSuccess &&
              cudaMalloc((void **)&ws.inc_aux, 2 * sizeof(unsigned long long)) == cudaSuccess;
    return ok ? APD_OK : APD_ERR_CUDA;
}

// Queues one pass of scoring + rescoring + moments at weights w.  With
// weights_only the records of the previous pass (same x, A, n) are reused and
// only the weights change; with a step, w (device, n) is first set to
// step->W + step->t step->p.  inc = kIncAuto makes it an incremental pass where
// the form allows (ws.inc_recorded says whether it was queued as one).
int enqueue_assign(const GridDev &g_in, int n, const double *x, const double *A, const double *w,
                   apd_precision prec, Workspace &ws, int32_t *labels, unsigned long long *mom,
                   cudaStream_t st, bool weights_only = false, const TrialStep *step = nullptr,
                   int inc = kIncNone) {
    ws.inc_recorded = false;
    if (prec != APD_FP32 && prec != APD_TC_TF32 && prec != APD_TC_BF16) return APD_ERR_UNSUPPORTED;
    GridDev g = g_in;
    const bool sharded = ws.shard_world > 1 && !g.kz1;
    if (sharded) {
        int kb = 0, kc = 0;
        shard_range(g.res[g.dim - 1], ws.shard_rank, ws.shard_world, kb, kc);
        g.kz0 = kb;
        g.kz1 = kb + kc;
    }
    const bool empty = g.kz1 && g.kz1 <= g.kz0;  // an empty slab: moments stay zero
    const size_t K = (size_t)moment_width(g.dim);
    // an incremental pass needs the pruned tensor-core scorer on one rank (its
    // buffers are allocated by the caller, outside any graph capture)
    const bool inc_form = inc == kIncAuto && !sharded && !empty && ws.prune && ws.inc_labels &&
                          prec != APD_FP32;
    bool tc = false, inc_on = false;
    if (weights_only) {
        tc = !empty && use_tensor_cores(g, prec, ws, true, st);
        inc_on = inc_form && tc;
        // one launch: moments and counters cleared, trial weights into the records
        // the first trial of a new L-BFGS direction forms p too (see Solver::iterate)
        const bool form_p = ws.p_pending && step && step->p == ws.p;
        ws.p_pending = false;
        const unsigned full_max = (unsigned)(kIncFullMax * (double)win_pixels(g));
        APD_TRY(cuda_ok(launch_eval_begin(n, step ? step->W : w, step ? step->t : 0.0, step ? step->p : nullptr,
                                          const_cast<double *>(w), mom, ws, st, form_p,
                                          inc_on ? ws.inc_w0 : nullptr, full_max)));
    } else {
        if (step) APD_TRY(cuda_ok(launch_axpy(n, step->W, step->t, step->p, const_cast<double *>(w), st)));
        APD_TRY(cuda_ok(cudaMemsetAsync(mom, 0, (size_t)n * K * sizeof(unsigned long long), st)));
        APD_TRY(cuda_ok(launch_eval_reset(ws, st, false)));  // also: no record, this pass records
        APD_TRY(cuda_ok(launch_seed_prep(g, n, x, A, w, ws, st)));
        APD_TRY(cuda_ok(launch_group_bounds(n, ws, st)));
        tc = !empty && use_tensor_cores(g, prec, ws, false, st);
        inc_on = inc_form && tc;
    }
    if (inc_on) APD_TRY(cuda_ok(launch_inc_prepare(n, mom, ws, st)));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ws.profiling && ws.capturing) {
        // the graph's own events; the replay reads them after its synchronisation
        e0 = ws.cap_e0;
        e1 = ws.cap_e1;
    } else if (ws.profiling) {
        while (ws.ev.size() < ws.ev_used + 2) {
            cudaEvent_t e;
            APD_TRY(cuda_ok(cudaEventCreate(&e)));
            ws.ev.push_back(e);
        }
        e0 = ws.ev[ws.ev_used];
        e1 = ws.ev[ws.ev_used + 1];
        ws.ev_used += 2;
        ws.prof_pairs += win_pixels(g) * (long long)n;
    }
    // recorded right before the scoring kernel itself (after the tensor-core
    // form's candidate pre-pass), so the events time that kernel alone
    ws.prof_e0 = e0;
    // the tensor-core tiling needs per-tile scratch; grids too thin for the
    // workspace's tile capacity are scored by the FP32 kernel (same labels)
    if (empty) {
    } else if (!tc)
        APD_TRY(cuda_ok(launch_assign_fp32(g, n, ws, labels, mom, st)));
    else {
        // an incremental pass: the pre-pass and the scorer (recording variant, the
        // labels into the record) do nothing when the device chose a re-decision
        if (inc_on) {
            labels = ws.inc_labels;
            ws.rec_gap = ws.inc_gap;
            ws.inc_auto = true;
        }
        const cudaError_t e = launch_assign_tc(g, n, ws, labels, mom, prec == APD_TC_TF32 ? 0 : 1, st);
        ws.rec_gap = nullptr;
        ws.inc_auto = false;
        APD_TRY(cuda_ok(e));
        ws.inc_recorded = inc_on;
    }
    APD_TRY(cuda_ok(record_scoring_start(ws, st)));  // nothing launched (an empty slab)
    if (e1) APD_TRY(cuda_ok(ws.capturing ? cudaEventRecordWithFlags(e1, st, cudaEventRecordExternal)
                                         : cudaEventRecord(e1, st)));
    // the re-decision (nothing when the pass records), the rescoring in the mode
    // the device chose, and a recording's moments, weights and w_ref kept
    if (inc_on) APD_TRY(cuda_ok(launch_tc_band(g, n, ws, st)));
    if (!empty)
        APD_TRY(cuda_ok(launch_rescore_fp64(g, n, x, A, w, ws, labels, mom, st, inc_on ? ws.inc_labels : nullptr,
                                            inc_on ? &ws.sc->inc_go : nullptr)));
    if (inc_on) APD_TRY(cuda_ok(launch_inc_commit(n, mom, w, ws, st)));
    if (sharded) {
        // every rank's slab moments, summed, before anything reads them
        const apd_seeds cur{n, x, A, w};
        if (ws.shard_fn(ws.shard_ctx, reinterpret_cast<int64_t *>(mom), (int64_t)n * moment_width(g.dim), &cur,
                        (apd_stream_t)st) != 0)
            return APD_ERR_CUDA;
    }
    // the tensor-core launcher counts its pre-pass launches itself
    ws.kernel_launches += (weights_only ? 3 : (ws.sorted ? 6 : 4) + (ws.groups ? 1 : 0) + (step ? 1 : 0)) -
                          (empty ? 2 : 0) +  // an empty slab launches neither scoring nor rescoring
                          (inc_on ? 3 : 0);  // the incremental pass's prepare, re-decision and commit
    ws.last_pixels = win_pixels(g);
    ws.last_pairs = win_pixels(g) * (long long)n;
    return APD_OK;
}

int take_status(Workspace &ws, cudaStream_t st) {
    int bits = 0;
    APD_TRY(cuda_ok(cudaStreamSynchronize(st)));
    APD_TRY(cuda_ok(cudaMemcpy(&bits, &ws.sc->status, sizeof(int), cudaMemcpyDeviceToHost)));
    if (bits) APD_TRY(cuda_ok(cudaMemset(&ws.sc->status, 0, sizeof(int))));
    return map_bits(bits);
}

// ----------------------------------------------------------------------------
// Algorithm 2: L-BFGS on f(W) = -g~(W) with a strong-Wolfe line search
// (Nocedal & Wright, Algorithms 3.5/3.6, cubic interpolation), stopping at the
// first evaluation with max_i |v_i - m_i |P|| / v_i < eps.
// ----------------------------------------------------------------------------
struct Solver {
    GridDev g;
    int n;
    const double *x, *A, *v;
    Workspace &ws;
    apd_precision prec;
    cudaStream_t st;
    double eps;
    int max_evals;
    int history;
    bool check_volumes;
    double measure;

    int evals = 0, iters = 0;
    long long rescored = 0;
    double best_err = INFINITY, best_g = 0.0;
    int stall_evals = 0;  // > 0: stop after this many evaluations without a 2 % better error
    int last_gain = 0;    // evaluation count at the last such improvement
    double last_g = 0.0, last_err = INFINITY;
    const double *last_point = nullptr;  // device pointer evaluated last
    bool last_is_best = false;
    bool first = true;
    bool geometry_ready = false;  // records of x, A built (they are fixed for the solve)
    int inc_mode = kIncNone;  // kIncAuto: every pass incremental (see enqueue_assign)
    int64_t inc_redecided = 0;  // passes the device made re-decisions

    Solver(Workspace &w) : ws(w) {}

    // Evaluate at Wp; gf_out receives grad f = -(v - |P| m); pdir (nullable) for <grad f, p>.
    // With a step, Wp (device, n) is first set to step->W + step->t step->p.
    // The launches of one evaluation at weights Wp (a trial step when given),
    // queued on stream s: scoring, rescoring, moments, dual, scalars read back.
    int enqueue_eval(const double *Wp, double *gf_out, const double *pdir, const TrialStep *step,
                     cudaStream_t s) {
        // the records' positions and matrices are built once per solve
        APD_TRY(enqueue_assign(g, n, x, A, Wp, prec, ws, nullptr, ws.moments, s, geometry_ready, step, inc_mode));
        APD_TRY(cuda_ok(launch_dual(g, n, x, A, Wp, v, pdir, ws.moments, ws, nullptr, ws.grad, gf_out,
                                    nullptr, s)));
        ws.kernel_launches += 1;
        return cuda_ok(cudaMemcpyAsync(ws.sc_host, ws.sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, s));
    }

    // A weights-only evaluation replayed from a captured graph (captured on
    // first use of its arguments); eg stays null where the evaluation is not
    // graphed (sharded workspaces, graphs switched off, a refused capture).
    int graph_eval(const double *Wp, double *gf_out, const double *pdir, const TrialStep *step, EvalGraph *&eg) {
        eg = nullptr;
        if (!ws.graphs || !geometry_ready || ws.shard_world > 1) return APD_OK;
        struct Key {
            int dim, res[3], kz0, kz1, n, prec, prune, sorted, profiling, has_step, form_p, inc;
            uint32_t wait_limit, use_tc;
            double lo[3], h[3];
            const void *ptr[9];
        } k;
        std::memset(&k, 0, sizeof k);
        k.dim = g.dim;
        for (int a = 0; a < 3; ++a) {
            k.res[a] = g.res[a];
            k.lo[a] = g.lo[a];
            k.h[a] = g.h[a];
        }
        k.kz0 = g.kz0;
        k.kz1 = g.kz1;
        k.n = n;
        k.prec = (int)prec;
        k.prune = ws.prune ? 1 : 0;
        k.sorted = ws.sorted ? 1 : 0;
        k.profiling = ws.profiling ? 1 : 0;
        k.has_step = step ? 1 : 0;
        const bool form_p = ws.p_pending && step && step->p == ws.p;  // as enqueue_assign decides it
        k.form_p = form_p ? 1 : 0;
        k.inc = inc_mode;
        k.wait_limit = ws.wait_limit;
        // the scorer the captured pass takes (the seeds' conditioning can change it between solves)
        const bool tc = use_tensor_cores(g, prec, ws, true, st);
        k.use_tc = tc ? 1u : 0u;
        const void *ptrs[9] = {x, A, v, Wp, gf_out, pdir, step ? step->W : nullptr, step ? step->p : nullptr,
                               ws.moments};
        std::memcpy(k.ptr, ptrs, sizeof ptrs);
        const unsigned char *kb = reinterpret_cast<const unsigned char *>(&k);
        for (EvalGraph &e : ws.graph_cache)
            if (e.key.size() == sizeof k && std::memcmp(e.key.data(), kb, sizeof k) == 0) {
                if (e.failed) return APD_OK;
                eg = &e;
                break;
            }
        if (!eg) {
            EvalGraph e;
            e.key.assign(kb, kb + sizeof k);
            if (!ws.cap_stream && cudaStreamCreateWithFlags(&ws.cap_stream, cudaStreamNonBlocking) != cudaSuccess)
                return APD_ERR_CUDA;
            if (ws.profiling &&
                (cudaEventCreate(&e.e0) != cudaSuccess || cudaEventCreate(&e.e1) != cudaSuccess))
                return APD_ERR_CUDA;
            const int64_t kl0 = ws.kernel_launches;
            ws.capturing = true;
            ws.cap_e0 = e.e0;
            ws.cap_e1 = e.e1;
            int rc = cuda_ok(cudaStreamBeginCapture(ws.cap_stream, cudaStreamCaptureModeThreadLocal));
            if (rc == APD_OK) {
                rc = enqueue_eval(Wp, gf_out, pdir, step, ws.cap_stream);
                cudaGraph_t gr = nullptr;
                const cudaError_t ce = cudaStreamEndCapture(ws.cap_stream, &gr);
                if (rc == APD_OK && ce == cudaSuccess && gr &&
                    cudaGraphInstantiate(&e.exec, gr, 0ull) == cudaSuccess) {
                    e.graph = gr;
                } else {
                    if (gr) cudaGraphDestroy(gr);
                    e.failed = true;
                }
            } else {
                e.failed = true;
            }
            ws.capturing = false;
            cudaGetLastError();  // a refused capture leaves no error behind
            e.launches = ws.kernel_launches - kl0;
            ws.kernel_launches = kl0;
            e.pixels = ws.last_pixels;
            e.pairs = ws.last_pairs;
            e.recorded = ws.inc_recorded;
            if (rc != APD_OK && rc != APD_ERR_CUDA) return rc;  // an argument error, as without a graph
            if (!e.failed && step) {
                size_t nn = 0;
                cudaGraphGetNodes(e.graph, nullptr, &nn);
                std::vector<cudaGraphNode_t> nodes(nn);
                if (nn) cudaGraphGetNodes(e.graph, nodes.data(), &nn);
                for (cudaGraphNode_t nd : nodes) {
                    cudaGraphNodeType ty;
                    cudaKernelNodeParams kp{};
                    if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel &&
                        cudaGraphKernelNodeGetParams(nd, &kp) == cudaSuccess && kp.func == eval_begin_kernel_fn())
                        e.begin = nd;
                }
                if (!e.begin) e.failed = true;
            }
            if (ws.graph_cache.size() >= kGraphCap) {  // the least recently used one goes
                size_t old = 0;
                for (size_t i = 1; i < ws.graph_cache.size(); ++i)
                    if (ws.graph_cache[i].used < ws.graph_cache[old].used) old = i;
                destroy_graph(ws.graph_cache[old]);
                ws.graph_cache.erase(ws.graph_cache.begin() + (long)old);
            }
            ws.graph_cache.push_back(e);
            if (ws.graph_cache.back().failed) return APD_OK;
            eg = &ws.graph_cache.back();
        }
        eg->used = ++ws.graph_clock;
        if (tc) APD_TRY(cuda_ok(launch_tc_axis(g, ws, st)));
        ws.p_pending = false;
        if (step)
            APD_TRY(cuda_ok(set_eval_begin_node(eg->exec, eg->begin, n, step->W, step->t, step->p,
                                                const_cast<double *>(Wp), ws.moments, ws, form_p,
                                                eg->recorded ? ws.inc_w0 : nullptr,
                                                (unsigned)(kIncFullMax * (double)win_pixels(g)))));
        APD_TRY(cuda_ok(cudaGraphLaunch(eg->exec, st)));
        ws.kernel_launches += eg->launches;
        ws.last_pixels = eg->pixels;
        ws.last_pairs = eg->pairs;
        ws.inc_recorded = eg->recorded;
        return APD_OK;
    }

    int eval(const double *Wp, double *gf_out, const double *pdir, double &f, double &dphi,
             double &err, const TrialStep *step = nullptr) {
        inc_mode = kIncNone;
        if (ws.incremental && ws.prune && ws.shard_world <= 1 && prec != APD_FP32 &&
            (ws.incremental > 1 || win_pixels(g) >= kIncMinPixels)) {
            APD_TRY(inc_alloc(ws));  // never inside a graph capture
            inc_mode = kIncAuto;
        }
        EvalGraph *eg = nullptr;
        APD_TRY(graph_eval(Wp, gf_out, pdir, step, eg));
        if (!eg) APD_TRY(enqueue_eval(Wp, gf_out, pdir, step, st));
        geometry_ready = true;
        APD_TRY(cuda_ok(cudaStreamSynchronize(st)));
        // a re-decision ran no scoring kernel: its (empty) launch is not timed
        const bool redecided = ws.inc_recorded && ws.sc_host->inc_go;
        if (redecided) {
            ++inc_redecided;
            if (!eg && ws.profiling && ws.ev_used >= 2) {
                ws.ev_used -= 2;
                ws.prof_pairs -= ws.last_pairs;
            }
        }
        if (eg && eg->e0 && ws.profiling && !redecided) {
            float ms = 0.f;
            APD_TRY(cuda_ok(cudaEventElapsedTime(&ms, eg->e0, eg->e1)));
            ws.prof_ms_graph += ms;
            ws.prof_n_graph += 1;
            ws.prof_pairs += eg->pairs;
        }
        ++evals;
        const DevScalars &h = *ws.sc_host;
        rescored += h.flag_count;
        if (h.status) {
            const int rc = map_bits(h.status);
            cudaMemset(&ws.sc->status, 0, sizeof(int));
            return rc;
        }
        if (first) {
            first = false;
            if (check_volumes) {
                if (!(h.min_v > 0.0) || std::fabs(h.sum_v - measure) > 1e-9 * measure) return APD_ERR_ARG;
            }
        }
        f = -h.g;
        dphi = h.dot_gp;
        err = h.max_rel_err;
        last_g = h.g;
        last_err = err;
        last_point = Wp;
        last_is_best = false;
        if (err < 0.98 * best_err) last_gain = evals;
        if (err < best_err) {
            best_err = err;
            best_g = h.g;
            APD_TRY(cuda_ok(cudaMemcpyAsync(ws.Wbest, Wp, (size_t)n * sizeof(double),
                                            cudaMemcpyDeviceToDevice, st)));
            last_is_best = true;
        }
        return APD_OK;
    }

    enum LsResult { LS_ACCEPT, LS_CONVERGED, LS_FAIL, LS_BUDGET, LS_NOT_DESCENT };

    // phi(t) = f(W + t p); on LS_ACCEPT ws.Wt / ws.gft hold the accepted point.
    // The direction kernel's <grad f, p> (phi'(0)) arrives with the first
    // evaluation's scalars, so the direction needs no read of its own; a
    // direction that is not a descent direction ends the search (LS_NOT_DESCENT)
    // unless that first point has already converged.
    int line_search(double f0, double t_init, LsResult &res, double &f_acc) {
        const double c1 = 1e-4, c2 = 0.9;
        double dphi0 = 0.0;
        double t_prev = 0.0, phi_prev = f0, dphi_prev = 0.0;
        double t = t_init;
        double best_t = 0.0, best_phi = f0;
        double cur_t = -1.0;  // t at which Wt/gft were last evaluated
        auto evaluate = [&](double tt, double &phi, double &dphi, double &err) -> int {
            const TrialStep step{ws.W, tt, ws.p};  // Wt = W + tt p, formed by the evaluation's first kernel
            APD_TRY(eval(ws.Wt, ws.gft, ws.p, phi, dphi, err, &step));
            cur_t = tt;
            return APD_OK;
        };
        auto accept = [&](double tt, double phi) -> int {
            if (cur_t != tt) {
                double p2, d2, e2;
                APD_TRY(evaluate(tt, p2, d2, e2));
                if (e2 < eps) {
                    res = LS_CONVERGED;
                    return APD_OK;
                }
                phi = p2;
            }
            res = LS_ACCEPT;
            f_acc = phi;
            return APD_OK;
        };
        auto zoom = [&](double lo, double plo, double dlo, double hi, double phi_hi,
                        double dhi) -> int {
            for (int it = 0; it < 20; ++it) {
                if (evals >= max_evals) {
                    res = LS_BUDGET;
                    return APD_OK;
                }
                const double a = std::min(lo, hi), b = std::max(lo, hi), w = b - a;
                double tt;
                const double d1 = dlo + dhi - 3.0 * (plo - phi_hi) / (lo - hi);
                const double disc = d1 * d1 - dlo * dhi;
                if (disc >= 0.0 && std::isfinite(disc)) {
                    const double d2 = std::copysign(std::sqrt(disc), hi - lo);
                    const double den = dhi - dlo + 2.0 * d2;
                    tt = den != 0.0 ? hi - (hi - lo) * (dhi + d2 - d1) / den : 0.5 * (a + b);
                } else {
                    tt = 0.5 * (a + b);
                }
                if (!std::isfinite(tt) || tt < a + 0.1 * w || tt > b - 0.1 * w) tt = 0.5 * (a + b);
                double phi, dphi, err;
                APD_TRY(evaluate(tt, phi, dphi, err));
                if (err < eps) {
                    res = LS_CONVERGED;
                    return APD_OK;
                }
                if (phi > f0 + c1 * tt * dphi0 || phi >= plo) {
                    hi = tt;
                    phi_hi = phi;
                    dhi = dphi;
                } else {
                    if (phi < best_phi) {
                        best_phi = phi;
                        best_t = tt;
                    }
                    if (std::fabs(dphi) <= -c2 * dphi0) return accept(tt, phi);
                    if (dphi * (hi - lo) >= 0.0) {
                        hi = lo;
                        phi_hi = plo;
                        dhi = dlo;
                    }
                    lo = tt;
                    plo = phi;
                    dlo = dphi;
                }
                if (std::fabs(hi - lo) <= 1e-14 * std::max(1.0, std::fabs(lo))) break;
            }
            if (best_t > 0.0) return accept(best_t, best_phi);
            res = LS_FAIL;
            return APD_OK;
        };
        for (int i = 0; i < 30; ++i) {
            if (evals >= max_evals) {
                res = LS_BUDGET;
                return APD_OK;
            }
            double phi, dphi, err;
            APD_TRY(evaluate(t, phi, dphi, err));
            if (err < eps) {
                res = LS_CONVERGED;
                return APD_OK;
            }
            if (i == 0) {
                dphi0 = ws.sc_host->gp0;
                dphi_prev = dphi0;
                if (!(dphi0 < 0.0)) {
                    res = LS_NOT_DESCENT;
                    return APD_OK;
                }
            }
            if (phi > f0 + c1 * t * dphi0 || (i > 0 && phi >= phi_prev))
                return zoom(t_prev, phi_prev, dphi_prev, t, phi, dphi);
            if (phi < best_phi) {
                best_phi = phi;
                best_t = t;
            }
            if (std::fabs(dphi) <= -c2 * dphi0) return accept(t, phi);
            if (dphi >= 0.0) return zoom(t, phi, dphi, t_prev, phi_prev, dphi_prev);
            t_prev = t;
            phi_prev = phi;
            dphi_prev = dphi;
            t = std::min(4.0 * t, 1e12);
        }
        if (best_t > 0.0) return accept(best_t, best_phi);
        res = LS_FAIL;
        return APD_OK;
    }

    // Runs the solve from W0 (device, n); returns status.  On exit ws.Wbest
    // (or the converged point, copied to out) holds the weights.
    int run(const double *W0, double *out, bool &converged) {
        converged = false;
        ws.p_pending = false;
        APD_TRY(cuda_ok(cudaMemcpyAsync(ws.W, W0, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, st)));
        double f0, d0, err0;
        APD_TRY(eval(ws.W, ws.gf, nullptr, f0, d0, err0));
        if (err0 < eps) {
            converged = true;
            return cuda_ok(cudaMemcpyAsync(out, ws.W, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        }
        return iterate(f0, out, converged);
    }

    // Start from the better of W_pred and W = 0 by g~ (ties: zero); both are
    // evaluated, so the gradient at the chosen start is already known.
    int run_judged(const double *Wpred, double *out, bool &converged, int &used) {
        converged = false;
        ws.p_pending = false;
        used = 1;
        APD_TRY(cuda_ok(cudaMemcpyAsync(ws.W, Wpred, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, st)));
        double fp, dp, ep;
        APD_TRY(eval(ws.W, ws.gf, nullptr, fp, dp, ep));
        if (ep < eps) {
            converged = true;
            return cuda_ok(cudaMemcpyAsync(out, ws.W, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        }
        APD_TRY(cuda_ok(cudaMemsetAsync(ws.Wt, 0, (size_t)n * sizeof(double), st)));
        double fz, dz, ez;
        APD_TRY(eval(ws.Wt, ws.gft, nullptr, fz, dz, ez));
        if (ez < eps) {
            converged = true;
            used = 0;
            return cuda_ok(cudaMemcpyAsync(out, ws.Wt, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        }
        if (fz <= fp) {
            std::swap(ws.W, ws.Wt);
            std::swap(ws.gf, ws.gft);
            used = 0;
            return iterate(fz, out, converged);
        }
        return iterate(fp, out, converged);
    }

    // L-BFGS iterations from the evaluated point ws.W (gradient ws.gf, f0 = f(ws.W)).
    // The direction, the trial point and its evaluation are queued back to back
    // and read once; a pair pushed after an accepted step is taken or dropped by
    // the device (its curvature test) and the host learns which at that read.
    int iterate(double f0, double *out, bool &converged) {
        int hist = 0, newest = kHistCap - 1;
        double gamma = 1.0;
        if (ws.carry_on && ws.carry.valid) {  // continue the history of the previous solve
            hist = std::min(ws.carry.hist, history);
            newest = ws.carry.newest;
            gamma = ws.carry.gamma;
        }
        auto keep = [&]() {
            if (!ws.carry_on) return;
            ws.carry.hist = hist;
            ws.carry.newest = newest;
            ws.carry.gamma = gamma;
            ws.carry.valid = true;
        };
        int fails = 0;
        bool pending = false;  // a pushed pair whose test result is not read yet
        int p_slot = 0;
        bool dir_ready = false;  // the last push also formed this direction's coefficients
        while (evals < max_evals && !(stall_evals > 0 && evals - last_gain >= stall_evals)) {
            const int hist_acc = std::min(hist + 1, history);
            // the coefficients of p come from the last push or from the dots kernel;
            // the first trial's eval_begin forms p from them (and <grad f, p>)
            if (!dir_ready) {
                APD_TRY(cuda_ok(launch_lbfgs_coefficients(n, hist, newest, kHistCap, gamma, pending, hist_acc,
                                                          p_slot, ws, st)));
                ws.kernel_launches += 1;
            }
            ws.p_pending = true;
            dir_ready = false;
            double t0 = 1.0;
            if (!pending && hist == 0) {
                // first step (or after a reset): p = -grad f; take t0 ~ 1 / H_ii with the
                // cell-volume sensitivity H_ii ~ D V^(1 - 2/D) of a cell of volume V = |Omega| / n
                const double V = measure / (double)n;
                t0 = 0.5 * std::pow(V, 2.0 / g.dim - 1.0) / g.dim;
            }
            LsResult res;
            double f_acc = f0;
            const int evals_before = evals;
            APD_TRY(line_search(f0, t0, res, f_acc));
            if (pending && evals > evals_before) {
                if (ws.sc_host->pair_ok) {
                    newest = p_slot;
                    hist = hist_acc;
                    gamma = ws.sc_host->sy / ws.sc_host->yy;
                }
                pending = false;
            }
            if (res == LS_NOT_DESCENT) {
                if (hist == 0) break;
                hist = 0;
                gamma = 1.0;
                continue;
            }
            if (res == LS_CONVERGED) {
                converged = true;
                ++iters;
                keep();
                return cuda_ok(cudaMemcpyAsync(out, ws.Wt, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, st));
            }
            if (res == LS_BUDGET) break;
            if (res == LS_FAIL) {
                if (hist == 0 || ++fails > 3) break;
                hist = 0;
                gamma = 1.0;
                continue;
            }
            fails = 0;
            ++iters;
            const int slot = (newest + 1) % kHistCap;
            // Gram entries with the pairs kept beside it if it is accepted, and the
            // next direction's coefficients for either outcome of its curvature test
            const int next_acc = std::min(hist + 1, history);
            APD_TRY(cuda_ok(launch_lbfgs_push(n, slot, kHistCap, next_acc - 1, true, hist, next_acc, gamma, ws, st)));
            ws.kernel_launches += 1;
            dir_ready = true;
            pending = true;
            p_slot = slot;
            std::swap(ws.W, ws.Wt);
            std::swap(ws.gf, ws.gft);
            f0 = f_acc;
        }
        keep();
        return cuda_ok(cudaMemcpyAsync(out, ws.Wbest, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
};

int solve_impl(const GridDev &g, const apd_grid *grid, int n, const double *x, const double *A,
               const double *w0, const double *v, double *w_out, const apd_solve_opts &o,
               apd_solve_info &info, Workspace &ws, cudaStream_t st, bool need_moments_at_out,
               bool judged = false, int *used = nullptr) {
    Solver s(ws);
    s.g = g;
    s.n = n;
    s.x = x;
    s.A = A;
    s.v = v;
    s.prec = o.precision;
    s.st = st;
    s.eps = o.eps;
    s.max_evals = o.max_evals;
    s.history = std::max(1, std::min(o.history, kHistCap - 1));  // the slot written next is never in use
    s.check_volumes = o.check_volumes != 0;
    s.measure = domain_measure(grid);
    s.stall_evals = ws.solve_stall;
    bool conv = false;
    int used_pred = 0;
    int rc = judged ? s.run_judged(w0, w_out, conv, used_pred) : s.run(w0, w_out, conv);
    if (used) *used = used_pred;
    info.evaluations += s.evals;
    info.iterations += s.iters;
    info.rescored_fp64 += s.rescored;
    info.solves += 1;
    if (rc != APD_OK) return rc;
    if (conv) {
        info.max_rel_err = s.last_err;
        info.g = s.last_g;
    } else {
        info.max_rel_err = s.best_err;
        info.g = s.best_g;
        if (need_moments_at_out) {
            // re-evaluate so that the workspace moments belong to the returned weights
            double f, d, e;
            APD_TRY(s.eval(w_out, ws.gf, nullptr, f, d, e));
        }
    }
    if (!conv) return APD_NOT_CONVERGED;
    const double vmin = ws.sc_host->min_v;
    if (g.cell > o.eps * vmin / std::pow(2.0, g.dim)) return APD_WARN_TOL_INFEASIBLE;
    return APD_OK;
}

}  // namespace

extern "C" {

int32_t apd_version(void) { return 100; }

const char *apd_status_string(int status) {
    switch (status) {
        case APD_OK: return "ok";
        case APD_NOT_CONVERGED: return "not converged: evaluation cap reached";
        case APD_WARN_TOL_INFEASIBLE: return "converged, but the grid is coarser than eq. (2.10) asks";
        case APD_ERR_ARG: return "invalid argument";
        case APD_ERR_NOT_SPD: return "an anisotropy matrix is not symmetric positive definite";
        case APD_ERR_CUDA: return "CUDA error";
        case APD_ERR_WORKSPACE: return "workspace too small or of another dimension";
        case APD_ERR_TIMEOUT: return "a bounded device wait timed out";
        case APD_ERR_UNSUPPORTED: return "unsupported precision or option";
        default: return "unknown status";
    }
}

void apd_solve_opts_default(apd_solve_opts *o) {
    if (!o) return;
    o->eps = 0.01;
    o->max_evals = 1000;
    o->history = 10;
    o->precision = APD_FP32;
    o->check_volumes = 1;
}

int apd_workspace_create(apd_workspace **out, int32_t dim, int32_t max_n, int64_t max_j) {
    if (!out) return APD_ERR_ARG;
    *out = nullptr;
    if ((dim != 2 && dim != 3) || max_n < 1 || max_j < 1 || max_j >= (1ll << 31)) return APD_ERR_ARG;
    apd_workspace *ws = new (std::nothrow) apd_workspace();
    if (!ws) return APD_ERR_CUDA;
    Workspace &w = ws->w;
    w.dim = dim;
    w.max_n = max_n;
    w.max_j = max_j;
    cudaGetDevice(&w.device);
    if (cudaDeviceGetAttribute(&w.sms, cudaDevAttrMultiProcessorCount, w.device) != cudaSuccess || w.sms < 1)
        w.sms = 152;
    w.n_pad_max = ((max_n + kChunk - 1) / kChunk) * kChunk;
    w.hist_cap = kHistCap;
    const size_t K = (size_t)moment_width(dim);
    const size_t nb = std::max<size_t>((size_t)((max_n + 255) / 256), 64);  // dual partials (launch_dual)
    bool ok = true;
    auto alloc = [&](void **p, size_t bytes) {
        if (ok && cudaMalloc(p, bytes) != cudaSuccess) ok = false;
    };
    alloc((void **)&w.recs, (size_t)w.n_pad_max * sizeof(SeedRec));
    alloc((void **)&w.recs32, (size_t)w.n_pad_max * sizeof(SeedRec32));
    if (w.n_pad_max <= kSortMax) {
        alloc((void **)&w.recs_tmp, (size_t)w.n_pad_max * sizeof(SeedRec));
        alloc((void **)&w.codes, (size_t)w.n_pad_max * sizeof(uint32_t));
        alloc((void **)&w.scodes, (size_t)w.n_pad_max * sizeof(uint32_t));
        alloc((void **)&w.perm, (size_t)w.n_pad_max * sizeof(int32_t));
        alloc((void **)&w.recs32s, (size_t)w.n_pad_max * sizeof(SeedRec32));
    }
    alloc((void **)&w.moments, (size_t)max_n * K * sizeof(unsigned long long));
    alloc((void **)&w.flags, (size_t)max_j * sizeof(uint32_t));
    alloc((void **)&w.flag_gi, (size_t)max_j * sizeof(int32_t));
    alloc((void **)&w.pairs_scored, sizeof(unsigned long long));
    alloc((void **)&w.groups, (size_t)(w.n_pad_max / 32) * sizeof(GroupBound));
    alloc((void **)&w.sc, sizeof(DevScalars));
    // tensor-core tiles hold 512 pixels; 2x slack covers ragged grids (thinner grids
    // are scored by the FP32 kernel)
    w.tc_tile_cap = max_j / 256 + 1024;
    alloc((void **)&w.tc_centre, (size_t)w.tc_tile_cap * 6 * sizeof(float));
    alloc((void **)&w.tc_start, (size_t)w.tc_tile_cap * sizeof(int));
    alloc((void **)&w.tc_meta, (size_t)w.tc_tile_cap * sizeof(int4));
    alloc((void **)&w.tc_texcl, (size_t)w.tc_tile_cap * sizeof(float));
    alloc((void **)&w.tc_list, (size_t)w.tc_tile_cap * tc_list_cap() * sizeof(int));
    alloc((void **)&w.tc_bops, (size_t)w.tc_tile_cap * tc_bops_bytes_per_tile());
    alloc((void **)&w.tc_axis, (size_t)3 * w.tc_tile_cap * sizeof(float4));
    // super-tiles: at most one per tile
    w.part_rows = (int)nb;
    alloc((void **)&w.part, nb * kPartStride * sizeof(double));
    alloc((void **)&w.grad, (size_t)max_n * sizeof(double));
    alloc((void **)&w.W, (size_t)max_n * sizeof(double));
    alloc((void **)&w.Wt, (size_t)max_n * sizeof(double));
    alloc((void **)&w.p, (size_t)max_n * sizeof(double));
    alloc((void **)&w.gf, (size_t)max_n * sizeof(double));
    alloc((void **)&w.gft, (size_t)max_n * sizeof(double));
    alloc((void **)&w.Wbest, (size_t)max_n * sizeof(double));
    alloc((void **)&w.S, (size_t)kHistCap * max_n * sizeof(double));
    alloc((void **)&w.Y, (size_t)kHistCap * max_n * sizeof(double));
    alloc((void **)&w.gram, 2 * kHistCap * kHistCap * sizeof(double));
    w.lb_rows = w.sms;
    alloc((void **)&w.lb_part, (size_t)w.lb_rows * kLbfgsDots * sizeof(double));
    alloc((void **)&w.lb_coef, sizeof(LbfgsCoef));
    alloc((void **)&w.rho, kHistCap * sizeof(double));
    alloc((void **)&w.X, (size_t)max_n * dim * sizeof(double));
    alloc((void **)&w.vbuf, (size_t)max_n * sizeof(double));
    alloc((void **)&w.wfeat, (size_t)max_n * kWarmFeatMax * sizeof(float));
    alloc((void **)&w.wpred, (size_t)max_n * sizeof(double));
    if (ok && cudaMallocHost((void **)&w.sc_host, sizeof(DevScalars)) != cudaSuccess) ok = false;
    if (ok && cudaMemset(w.sc, 0, sizeof(DevScalars)) != cudaSuccess) ok = false;
    if (ok && cudaMemset(w.pairs_scored, 0, sizeof(unsigned long long)) != cudaSuccess) ok = false;
    if (ok && cudaMemset(w.recs, 0, (size_t)w.n_pad_max * sizeof(SeedRec)) != cudaSuccess) ok = false;
    if (ok && cudaDeviceSynchronize() != cudaSuccess) ok = false;
    if (!ok) {
        apd_workspace_destroy(ws);
        return APD_ERR_CUDA;
    }
    *out = ws;
    return APD_OK;
}

void apd_workspace_destroy(apd_workspace *ws) {
    if (!ws) return;
    Workspace &w = ws->w;
    for (cudaEvent_t e : w.ev) cudaEventDestroy(e);
    for (EvalGraph &e : w.graph_cache) destroy_graph(e);
    if (w.cap_stream) cudaStreamDestroy(w.cap_stream);
    void *ptrs[] = {w.recs, w.recs32, w.recs_tmp, w.codes, w.scodes, w.perm, w.recs32s, w.tc_centre, w.tc_start, w.tc_meta, w.tc_texcl, w.tc_list, w.tc_bops, w.tc_axis, w.moments, w.flags, w.flag_gi, w.pairs_scored, w.groups, w.sc, w.part, w.grad, w.W, w.Wt, w.p, w.gf, w.gft,
                    w.Wbest, w.S, w.Y, w.gram, w.lb_part, w.lb_coef, w.rho, w.X, w.vbuf, w.wfeat, w.wpred,
                    w.S2, w.Y2, w.gram2, w.rho2, w.inc_labels, w.inc_gap, w.inc_rec, w.inc_hist, w.inc_drift, w.inc_mom0, w.inc_w0, w.inc_aux};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (w.sc_host) cudaFreeHost(w.sc_host);
    delete ws;
}

int apd_profile_read_scored(apd_workspace *ws, int64_t *pairs_scored) {
    if (!ws || !pairs_scored) return APD_ERR_ARG;
    unsigned long long v = 0;
    APD_TRY(cuda_ok(cudaMemcpy(&v, ws->w.pairs_scored, sizeof v, cudaMemcpyDeviceToHost)));
    APD_TRY(cuda_ok(cudaMemset(ws->w.pairs_scored, 0, sizeof v)));
    *pairs_scored = (int64_t)v;
    return APD_OK;
}

int apd_workspace_set_pruning(apd_workspace *ws, int32_t enable) {
    if (!ws) return APD_ERR_ARG;
    ws->w.prune = enable != 0;
    return APD_OK;
}

int apd_profile_enable(apd_workspace *ws, int32_t enable) {
    if (!ws) return APD_ERR_ARG;
    ws->w.profiling = enable != 0;
    return APD_OK;
}

int apd_profile_read(apd_workspace *ws, double *assign_ms, int64_t *launches, int64_t *pairs,
                     int64_t *kernel_launches) {
    if (!ws || !assign_ms || !launches || !pairs || !kernel_launches) return APD_ERR_ARG;
    Workspace &w = ws->w;
    double total = 0.0;
    for (size_t k = 0; k + 1 < w.ev_used; k += 2) {
        APD_TRY(cuda_ok(cudaEventSynchronize(w.ev[k + 1])));
        float ms = 0.f;
        APD_TRY(cuda_ok(cudaEventElapsedTime(&ms, w.ev[k], w.ev[k + 1])));
        total += ms;
    }
    *assign_ms = total + w.prof_ms_graph;
    *launches = (int64_t)(w.ev_used / 2) + w.prof_n_graph;
    w.prof_ms_graph = 0.0;
    w.prof_n_graph = 0;
    *pairs = w.prof_pairs;
    *kernel_launches = w.kernel_launches;
    w.ev_used = 0;
    w.prof_pairs = 0;
    w.kernel_launches = 0;
    return APD_OK;
}

int apd_workspace_status(apd_workspace *ws, apd_stream_t stream) {
    if (!ws) return APD_ERR_ARG;
    return take_status(ws->w, (cudaStream_t)stream);
}

int apd_last_stats(apd_workspace *ws, apd_eval_stats *out, apd_stream_t stream) {
    if (!ws || !out) return APD_ERR_ARG;
    unsigned int fc = 0;
    APD_TRY(cuda_ok(cudaStreamSynchronize((cudaStream_t)stream)));
    APD_TRY(cuda_ok(cudaMemcpy(&fc, &ws->w.sc->flag_count, sizeof fc, cudaMemcpyDeviceToHost)));
    out->pixels = ws->w.last_pixels;
    out->pairs = ws->w.last_pairs;
    out->rescored_fp64 = fc;
    return APD_OK;
}

int apd_assign(const apd_grid *grid, const apd_seeds *seeds, apd_precision precision, int32_t *labels,
               double *tie_gap, apd_workspace *ws, apd_stream_t stream) {
    GridDev g;
    APD_TRY(validate_grid(grid, g));
    APD_TRY(validate_seeds(seeds));
    if (!labels) return APD_ERR_ARG;
    APD_TRY(check_ws(ws, g, seeds->n));
    cudaStream_t st = (cudaStream_t)stream;
    APD_TRY(enqueue_assign(g, seeds->n, seeds->x, seeds->A, seeds->w, precision, ws->w, labels, ws->w.moments, st));
    if (tie_gap) {
        APD_TRY(cuda_ok(launch_tie_gap(g, seeds->n, seeds->x, seeds->A, seeds->w, ws->w, tie_gap, st)));
        ws->w.kernel_launches += 1;
    }
    return APD_OK;
}

int apd_lbfgs_check(int32_t n, int32_t hist, const double *S, const double *Y, const double *g, int32_t fused,
                    double *p, double *gp) {
    if (n < 1 || hist < 1 || hist > kHistCap - 1 || !S || !Y || !g || !p || !gp || (fused != 0 && fused != 1))
        return APD_ERR_ARG;
    Workspace w;
    bool ok = true;
    std::vector<void *> bufs;
    auto alloc = [&](void **q, size_t bytes) {
        if (ok && cudaMalloc(q, bytes) != cudaSuccess) ok = false;
        if (ok) bufs.push_back(*q);
    };
    const size_t nb = (size_t)n * sizeof(double);
    alloc((void **)&w.W, nb);
    alloc((void **)&w.Wt, nb);
    alloc((void **)&w.gf, nb);
    alloc((void **)&w.gft, nb);
    alloc((void **)&w.p, nb);
    alloc((void **)&w.S, kHistCap * nb);
    alloc((void **)&w.Y, kHistCap * nb);
    alloc((void **)&w.rho, kHistCap * sizeof(double));
    alloc((void **)&w.gram, 2 * kHistCap * kHistCap * sizeof(double));
    cudaGetDevice(&w.device);
    if (cudaDeviceGetAttribute(&w.sms, cudaDevAttrMultiProcessorCount, w.device) != cudaSuccess || w.sms < 1)
        w.sms = 152;
    w.lb_rows = w.sms;
    alloc((void **)&w.lb_part, (size_t)w.lb_rows * kLbfgsDots * sizeof(double));
    alloc((void **)&w.lb_coef, sizeof(LbfgsCoef));
    alloc((void **)&w.sc, sizeof(DevScalars));
    cudaStream_t st = 0;
    // pair k enters as W = 0, Wt = s_k, gf = 0, gft = y_k in slot k
    if (ok) ok = cudaMemset(w.W, 0, nb) == cudaSuccess && cudaMemset(w.gf, 0, nb) == cudaSuccess &&
                 cudaMemset(w.sc, 0, sizeof(DevScalars)) == cudaSuccess;
    const int plain = fused ? hist - 1 : hist;
    for (int k = 0; ok && k < plain; ++k) {
        ok = cudaMemcpy(w.Wt, S + (size_t)k * n, nb, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(w.gft, Y + (size_t)k * n, nb, cudaMemcpyHostToDevice) == cudaSuccess &&
             launch_lbfgs_push(n, k, kHistCap, k, false, 0, 0, 1.0, w, st) == cudaSuccess;
    }
    if (ok && !fused) {
        // the newest pair is the pending one, taken by the direction kernels if it passed
        ok = cudaMemcpy(w.gf, g, nb, cudaMemcpyHostToDevice) == cudaSuccess &&
             launch_lbfgs_direction(n, hist - 1, hist - 2 < 0 ? kHistCap - 1 : hist - 2, kHistCap, 1.0, true, hist,
                                    hist - 1, w, st) == cudaSuccess;
    } else if (ok) {
        // the newest pair enters as W = 0, Wt = s, gft = g, gf = g - y (formed on the device),
        // pushed with the direction for the gradient g; then gf and gft change places
        ok = cudaMemcpy(w.Wt, S + (size_t)(hist - 1) * n, nb, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(w.gft, g, nb, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(w.p, Y + (size_t)(hist - 1) * n, nb, cudaMemcpyHostToDevice) == cudaSuccess &&
             launch_axpy(n, w.gft, -1.0, w.p, w.gf, st) == cudaSuccess &&
             launch_lbfgs_push(n, hist - 1, kHistCap, hist - 1, true, hist - 1, hist, 1.0, w, st) == cudaSuccess;
        std::swap(w.gf, w.gft);
        if (ok) ok = launch_lbfgs_pdir(n, w, st) == cudaSuccess;
    }
    DevScalars h{};
    if (ok) ok = cudaMemcpy(p, w.p, nb, cudaMemcpyDeviceToHost) == cudaSuccess &&
                 cudaMemcpy(&h, w.sc, sizeof h, cudaMemcpyDeviceToHost) == cudaSuccess;
    for (void *q : bufs) cudaFree(q);
    if (!ok) return APD_ERR_CUDA;
    *gp = h.gp0;
    return APD_OK;
}

int apd_workspace_set_incremental(apd_workspace *ws, int32_t enable) {
    if (!ws) return APD_ERR_ARG;
    if (enable < 0 || enable > 2) return APD_ERR_ARG;
    ws->w.incremental = enable;
    return APD_OK;
}

int apd_workspace_set_graphs(apd_workspace *ws, int32_t enable) {
    if (!ws) return APD_ERR_ARG;
    ws->w.graphs = enable != 0;
    return APD_OK;
}

int apd_workspace_set_wait_limit(apd_workspace *ws, int64_t polls) {
    if (!ws || polls > (int64_t)0xffffffffll) return APD_ERR_ARG;
    ws->w.wait_limit = polls < 0 ? kDefaultWaitPolls : (uint32_t)polls;
    return APD_OK;
}

int apd_cell_moments(const apd_grid *grid, const apd_seeds *seeds, apd_precision precision,
                     int64_t *moments, apd_workspace *ws, apd_stream_t stream) {
    GridDev g;
    APD_TRY(validate_grid(grid, g));
    APD_TRY(validate_seeds(seeds));
    if (!moments) return APD_ERR_ARG;
    APD_TRY(check_ws(ws, g, seeds->n));
    return enqueue_assign(g, seeds->n, seeds->x, seeds->A, seeds->w, precision, ws->w, nullptr,
                          reinterpret_cast<unsigned long long *>(moments), (cudaStream_t)stream);
}

int apd_shard_range(int32_t res, int32_t rank, int32_t world, int32_t *k_begin, int32_t *k_count) {
    if (res < 1 || world < 1 || rank < 0 || rank >= world || !k_begin || !k_count) return APD_ERR_ARG;
    int kb = 0, kc = 0;
    shard_range(res, rank, world, kb, kc);
    *k_begin = kb;
    *k_count = kc;
    return APD_OK;
}

int apd_workspace_set_shard(apd_workspace *ws, int32_t rank, int32_t world, apd_reduce_fn fn, void *ctx) {
    if (!ws || world < 1 || rank < 0 || rank >= world || (world > 1 && !fn)) return APD_ERR_ARG;
    ws->w.shard_rank = world > 1 ? rank : 0;
    ws->w.shard_world = world;
    ws->w.shard_fn = world > 1 ? fn : nullptr;
    ws->w.shard_ctx = world > 1 ? ctx : nullptr;
    return APD_OK;
}

int apd_cell_moments_slab(const apd_grid *grid, int32_t k_begin, int32_t k_count, const apd_seeds *seeds,
                          apd_precision precision, int64_t *moments, apd_workspace *ws, apd_stream_t stream) {
    GridDev g;
    APD_TRY(validate_grid(grid, g));
    APD_TRY(validate_seeds(seeds));
    if (!moments || k_begin < 0 || k_count < 1 || (long long)k_begin + k_count > g.res[g.dim - 1]) return APD_ERR_ARG;
    if (!ws) return APD_ERR_ARG;
    g.kz0 = k_begin;
    g.kz1 = k_begin + k_count;
    if (ws->w.dim != g.dim || seeds->n > ws->w.max_n || win_pixels(g) > ws->w.max_j) return APD_ERR_WORKSPACE;
    return enqueue_assign(g, seeds->n, seeds->x, seeds->A, seeds->w, precision, ws->w, nullptr,
                          reinterpret_cast<unsigned long long *>(moments), (cudaStream_t)stream);
}

int apd_dual_value_grad(const apd_grid *grid, const apd_seeds *seeds, const double *v,
                        apd_precision precision, double *g_out, double *grad, double *max_rel_err,
                        apd_workspace *ws, apd_stream_t stream) {
    GridDev g;
    APD_TRY(validate_grid(grid, g));
    APD_TRY(validate_seeds(seeds));
    if (!v || !g_out || !max_rel_err) return APD_ERR_ARG;
    APD_TRY(check_ws(ws, g, seeds->n));
    cudaStream_t st = (cudaStream_t)stream;
    APD_TRY(enqueue_assign(g, seeds->n, seeds->x, seeds->A, seeds->w, precision, ws->w, nullptr,
                           ws->w.moments, st));
    ws->w.kernel_launches += 1;
    return cuda_ok(launch_dual(g, seeds->n, seeds->x, seeds->A, seeds->w, v, nullptr, ws->w.moments,
                               ws->w, g_out, grad, nullptr, max_rel_err, st));
}

static int points_entry(const apd_points *pts, const apd_seeds *seeds, apd_workspace *ws) {
    if (!pts || (pts->dim != 2 && pts->dim != 3) || pts->count < 1 || !pts->y || !pts->mass) return APD_ERR_ARG;
    APD_TRY(validate_seeds(seeds));
    if (!ws) return APD_ERR_ARG;
    if (ws->w.dim != pts->dim || seeds->n > ws->w.max_n) return APD_ERR_WORKSPACE;
    return APD_OK;
}

int apd_points_moments(const apd_points *pts, const apd_seeds *seeds, double *moments, int32_t *labels,
                       apd_workspace *ws, apd_stream_t stream) {
    APD_TRY(points_entry(pts, seeds, ws));
    if (!moments) return APD_ERR_ARG;
    ws->w.kernel_launches += 4;
    return cuda_ok(launch_points_assign(pts->dim, pts->count, pts->y, pts->mass, seeds->n, seeds->x, seeds->A,
                                        seeds->w, moments, labels, ws->w, (cudaStream_t)stream));
}

int apd_points_dual_value_grad(const apd_points *pts, const apd_seeds *seeds, const double *v, double *g_out,
                               double *grad, double *max_rel_err, apd_workspace *ws, apd_stream_t stream) {
    APD_TRY(points_entry(pts, seeds, ws));
    if (!v || !g_out || !max_rel_err) return APD_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    // the workspace's moment buffer ([max_n][K] words) holds the FP64 moments
    double *mom = reinterpret_cast<double *>(ws->w.moments);
    APD_TRY(cuda_ok(launch_points_assign(pts->dim, pts->count, pts->y, pts->mass, seeds->n, seeds->x, seeds->A,
                                         seeds->w, mom, nullptr, ws->w, st)));
    ws->w.kernel_launches += 5;
    return cuda_ok(launch_points_dual(pts->dim, seeds->n, seeds->x, seeds->A, seeds->w, v, mom, ws->w, g_out, grad,
                                      max_rel_err, st));
}

static int masked_entry(const apd_grid *coarse, int32_t refine, const apd_seeds *seeds, const int32_t *coarse_labels,
                        GridDev &gc, GridDev &gf, apd_workspace *ws) {
    APD_TRY(validate_grid(coarse, gc));
    APD_TRY(validate_seeds(seeds));
    if (refine < 1 || !coarse_labels) return APD_ERR_ARG;
    apd_grid fine = *coarse;
    for (int d = 0; d < coarse->dim; ++d) {
        const long long fr = (long long)coarse->res[d] * refine;
        if (fr >= (1ll << 31)) return APD_ERR_ARG;
        fine.res[d] = (int32_t)fr;
    }
    APD_TRY(validate_grid(&fine, gf));
    if (ws && ws->w.shard_world > 1) return APD_ERR_UNSUPPORTED;  // the mask needs every coarse label
    return check_ws(ws, gc, seeds->n);
}

// Algorithm 1 on the coarse grid (labels into coarse_labels, its moments into
// the workspace's scratch), then the mask and the fine scoring into `mom`.
static int masked_enqueue(const GridDev &gc, const GridDev &gf, int32_t refine, const apd_seeds *seeds,
                          int32_t *coarse_labels, unsigned long long *mom, int64_t *refined, Workspace &w,
                          cudaStream_t st) {
    APD_TRY(enqueue_assign(gc, seeds->n, seeds->x, seeds->A, seeds->w, APD_FP32, w, coarse_labels, w.moments, st));
    w.kernel_launches += 2;
    return cuda_ok(launch_masked_refine(gc, gf, refine, seeds->n, seeds->x, seeds->A, seeds->w, coarse_labels, mom,
                                        reinterpret_cast<long long *>(refined), w, st));
}

int apd_masked_moments(const apd_grid *coarse, int32_t refine, const apd_seeds *seeds, int64_t *moments,
                       int32_t *coarse_labels, int64_t *refined, apd_workspace *ws, apd_stream_t stream) {
    GridDev gc, gf;
    APD_TRY(masked_entry(coarse, refine, seeds, coarse_labels, gc, gf, ws));
    if (!moments) return APD_ERR_ARG;
    return masked_enqueue(gc, gf, refine, seeds, coarse_labels, reinterpret_cast<unsigned long long *>(moments),
                          refined, ws->w, (cudaStream_t)stream);
}

int apd_masked_dual_value_grad(const apd_grid *coarse, int32_t refine, const apd_seeds *seeds, const double *v,
                               double *g_out, double *grad, double *max_rel_err, int32_t *coarse_labels,
                               apd_workspace *ws, apd_stream_t stream) {
    GridDev gc, gf;
    APD_TRY(masked_entry(coarse, refine, seeds, coarse_labels, gc, gf, ws));
    if (!v || !g_out || !max_rel_err) return APD_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    APD_TRY(masked_enqueue(gc, gf, refine, seeds, coarse_labels, ws->w.moments, nullptr, ws->w, st));
    ws->w.kernel_launches += 1;
    return cuda_ok(launch_dual(gf, seeds->n, seeds->x, seeds->A, seeds->w, v, nullptr, ws->w.moments, ws->w, g_out,
                               grad, nullptr, max_rel_err, st));
}

static int solve_entry(const apd_grid *grid, const apd_seeds *seeds, const double *v, double *w_out,
                       const apd_solve_opts *opts, GridDev &g, apd_solve_opts &o, apd_workspace *ws,
                       cudaStream_t st) {
    APD_TRY(validate_grid(grid, g));
    APD_TRY(validate_seeds(seeds));
    if (!v || !w_out) return APD_ERR_ARG;
    APD_TRY(check_ws(ws, g, seeds->n));
    if (opts) o = *opts;
    else apd_solve_opts_default(&o);
    if (!(o.eps > 0.0) || o.max_evals < 1 || o.history < 1) return APD_ERR_ARG;
    if (o.precision != APD_FP32 && o.precision != APD_TC_TF32 && o.precision != APD_TC_BF16)
        return APD_ERR_UNSUPPORTED;
    // a status latched by earlier stream-ordered calls is reported first
    return take_status(ws->w, st);
}

int apd_refine_next_grid(const apd_grid *grid, double v_min, double eps, const apd_refine_opts *ro,
                         int64_t max_pixels, apd_grid *next) {
    GridDev g;
    if (!ro || !next || validate_grid(grid, g) != APD_OK) return APD_ERR_ARG;
    if (!(v_min > 0.0) || !(eps > 0.0) || !std::isfinite(v_min) || !std::isfinite(eps) || !(ro->growth > 1.0) ||
        !std::isfinite(ro->growth))
        return APD_ERR_ARG;
    // eq. (2.10) for the smallest target volume: J >= |Omega| 2^D / (eps v_min)
    const double J = (double)g.J;
    const double J_need = domain_measure(grid) * std::pow(2.0, grid->dim) / (eps * v_min);
    const double f = std::max(ro->growth, std::pow(std::max(J_need / J, 1.0), 1.0 / grid->dim));
    apd_grid nxt = *grid;
    double Jn = 1.0;
    for (int d = 0; d < grid->dim; ++d) {
        const double m = std::ceil(grid->res[d] * f);
        const double cap = ro->max_res[d] > 0 ? (double)ro->max_res[d] : 2147483647.0;
        if (!(m <= cap)) return 1;
        nxt.res[d] = (int32_t)m;
        Jn *= m;
    }
    if (max_pixels > 0 && Jn > (double)max_pixels) return 1;
    *next = nxt;
    return APD_OK;
}

void apd_refine_opts_default(apd_refine_opts *ro) {
    if (!ro) return;
    ro->growth = 1.5;
    ro->max_res[0] = ro->max_res[1] = ro->max_res[2] = 0;
    ro->max_rounds = 4;
}

int apd_solve_weights_refine(const apd_grid *grid, const apd_seeds *seeds, const double *v, double *w_out,
                             const apd_solve_opts *opts, const apd_refine_opts *ro, apd_solve_info *info,
                             apd_grid *grid_out, apd_workspace *ws, apd_stream_t stream) {
    auto t0 = std::chrono::steady_clock::now();
    apd_solve_info inf, last;
    std::memset(&inf, 0, sizeof inf);
    GridDev g;
    apd_solve_opts o;
    apd_refine_opts r;
    apd_refine_opts_default(&r);
    if (ro) r = *ro;
    cudaStream_t st = (cudaStream_t)stream;
    // the options are checked before anything touches the device
    int rc = (!(r.growth > 1.0) || !std::isfinite(r.growth) || r.max_rounds < 0) ? APD_ERR_ARG : APD_OK;
    if (rc == APD_OK) rc = solve_entry(grid, seeds, v, w_out, opts, g, o, ws, st);
    for (int d = 0; rc == APD_OK && d < grid->dim; ++d)
        if (r.max_res[d] < 0 || (r.max_res[d] > 0 && r.max_res[d] < grid->res[d])) rc = APD_ERR_ARG;
    apd_grid cur = rc == APD_OK ? *grid : apd_grid{};
    const double *w0 = rc == APD_OK ? seeds->w : nullptr;
    for (int round = 0; rc == APD_OK || rc == APD_NOT_CONVERGED || rc == APD_WARN_TOL_INFEASIBLE; ++round) {
        std::memset(&last, 0, sizeof last);
        rc = solve_impl(g, &cur, seeds->n, seeds->x, seeds->A, w0, v, w_out, o, last, ws->w, st, false);
        inf.evaluations += last.evaluations;
        inf.iterations += last.iterations;
        inf.rescored_fp64 += last.rescored_fp64;
        inf.solves += 1;
        inf.max_rel_err = last.max_rel_err;
        inf.g = last.g;
        if (rc != APD_NOT_CONVERGED && rc != APD_WARN_TOL_INFEASIBLE) break;
        if (round >= r.max_rounds) break;
        apd_grid nxt;
        if (apd_refine_next_grid(&cur, ws->w.sc_host->min_v, o.eps, &r, ws->w.max_j, &nxt) != APD_OK) break;
        GridDev gn;
        if (validate_grid(&nxt, gn) != APD_OK) break;
        cur = nxt;
        g = gn;
        w0 = w_out;  // the weights found carry over
    }
    if (rc >= 0) cudaStreamSynchronize(st);
    if (grid_out && rc >= 0) *grid_out = cur;
    inf.status = rc;
    inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (info) *info = inf;
    return rc;
}

int apd_solve_weights(const apd_grid *grid, const apd_seeds *seeds, const double *v, double *w_out,
                      const apd_solve_opts *opts, apd_solve_info *info, apd_workspace *ws,
                      apd_stream_t stream) {
    auto t0 = std::chrono::steady_clock::now();
    apd_solve_info inf;
    std::memset(&inf, 0, sizeof inf);
    GridDev g;
    apd_solve_opts o;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = solve_entry(grid, seeds, v, w_out, opts, g, o, ws, st);
    if (rc == APD_OK)
        rc = solve_impl(g, grid, seeds->n, seeds->x, seeds->A, seeds->w, v, w_out, o, inf, ws->w, st, false);
    if (rc >= 0) cudaStreamSynchronize(st);
    inf.status = rc;
    inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (info) *info = inf;
    return rc;
}

// The network's predicted weights for one instance into ws.wpred.
static int predict_start(const apd_grid *grid, const apd_seeds *seeds, const double *v, apd_mlp *net, Workspace &ws,
                         apd_stream_t stream) {
    const int64_t offs[2] = {0, seeds->n};
    double box[6] = {0.0, 0.0, 0.0, 1.0, 1.0, 1.0};
    for (int a = 0; a < grid->dim; ++a) {
        box[a] = grid->lo[a];
        box[3 + a] = grid->hi[a];
    }
    ws.kernel_launches += 2;
    APD_TRY(apd_warmstart_features(net, 1, offs, box, seeds->x, seeds->A, v, ws.wfeat, nullptr, stream));
    return apd_warmstart_predict(net, 1, offs, box, ws.wfeat, ws.wpred, stream);
}

int apd_solve_weights_warm(const apd_grid *grid, const apd_seeds *seeds, const double *v, double *w_out,
                           const apd_solve_opts *opts, apd_solve_info *info, apd_workspace *ws, apd_mlp *net,
                           int32_t *used_pred, apd_stream_t stream) {
    auto t0 = std::chrono::steady_clock::now();
    apd_solve_info inf;
    std::memset(&inf, 0, sizeof inf);
    GridDev g;
    apd_solve_opts o;
    cudaStream_t st = (cudaStream_t)stream;
    int used = 0;
    int rc = net ? solve_entry(grid, seeds, v, w_out, opts, g, o, ws, st) : APD_ERR_ARG;
    if (rc == APD_OK && warmstart_dim(net) != g.dim) rc = APD_ERR_ARG;
    if (rc == APD_OK) {
        rc = predict_start(grid, seeds, v, net, ws->w, stream);
    }
    if (rc == APD_OK)
        rc = solve_impl(g, grid, seeds->n, seeds->x, seeds->A, ws->w.wpred, v, w_out, o, inf, ws->w, st, false,
                        true, &used);
    if (rc >= 0) cudaStreamSynchronize(st);
    if (used_pred) *used_pred = used;
    inf.status = rc;
    inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (info) *info = inf;
    return rc;
}

void apd_multires_opts_default(apd_multires_opts *mo) {
    if (!mo) return;
    mo->factor = 2;
    mo->coarse_eps = 0.05;
    mo->coarse_max_evals = 60;
    mo->carry_history = 0;
    mo->min_cell_span = 8;
    mo->coarse_stall_evals = 0;
}

// Coarse grid of a coarse-to-fine solve (same box, ceil(res / factor) >= 4 per axis).
static int coarse_grid(const apd_grid *grid, const apd_multires_opts &m, apd_grid &cg, GridDev &gc) {
    if (m.factor < 2 || !(m.coarse_eps > 0.0) || m.coarse_max_evals < 1 || m.min_cell_span < 0 ||
        m.coarse_stall_evals < 0)
        return APD_ERR_ARG;
    cg = *grid;
    for (int d = 0; d < grid->dim; ++d) cg.res[d] = std::max(4, (grid->res[d] + m.factor - 1) / m.factor);
    return validate_grid(&cg, gc);
}

// Solve on the coarse grid from w0 (judged against zero if asked), then on the
// fine grid from the coarse weights; w_out receives both in turn.  The coarse
// status (often NOT_CONVERGED at its cap) is not an error.
// The second L-BFGS history of a Lloyd run's coarse solves: allocated on the
// first use (the run asked for it with carry_history), exchanged with the main
// one around each coarse solve.
static bool carry_ready(const Workspace &ws) {
    return ws.S2 && ws.Y2 && ws.gram2 && ws.rho2 && ws.carry_enabled;
}
static void swap_history(Workspace &ws) {
    std::swap(ws.S, ws.S2);
    std::swap(ws.Y, ws.Y2);
    std::swap(ws.gram, ws.gram2);
    std::swap(ws.rho, ws.rho2);
}
static int carry_begin(Workspace &ws) {
    if (!ws.S2) {
        bool ok = cudaMalloc((void **)&ws.S2, (size_t)kHistCap * ws.max_n * sizeof(double)) == cudaSuccess &&
                  cudaMalloc((void **)&ws.Y2, (size_t)kHistCap * ws.max_n * sizeof(double)) == cudaSuccess &&
                  cudaMalloc((void **)&ws.gram2, 2 * kHistCap * kHistCap * sizeof(double)) == cudaSuccess &&
                  cudaMalloc((void **)&ws.rho2, kHistCap * sizeof(double)) == cudaSuccess;
        if (!ok) return APD_ERR_CUDA;
    }
    ws.carry.valid = false;
    ws.carry_enabled = true;
    return APD_OK;
}

static int c2f_solve(const GridDev &g, const apd_grid *grid, const GridDev &gc, const apd_grid *cg, int n,
                     const double *x, const double *A, const double *w0, const double *v, double *w_out,
                     const apd_solve_opts &o, const apd_multires_opts &m, apd_solve_info &inf,
                     apd_solve_info &cinf, Workspace &ws, cudaStream_t st, bool judged, int *used,
                     bool need_moments_at_out) {
    // cells of fewer than min_cell_span^D coarse pixels on average cannot reach the
    // coarse tolerance: the solve then runs on the fine grid alone
    const double span_d = std::pow((double)m.min_cell_span, (double)g.dim);
    if (m.min_cell_span > 0 && (double)gc.J < span_d * (double)n)
        return solve_impl(g, grid, n, x, A, w0, v, w_out, o, inf, ws, st, need_moments_at_out, judged, used);
    apd_solve_opts oc = o;
    oc.eps = m.coarse_eps;
    oc.max_evals = m.coarse_max_evals;
    const bool carry = carry_ready(ws);  // the coarse solve runs on the second history
    if (carry) swap_history(ws);
    ws.carry_on = carry;
    ws.solve_stall = m.coarse_stall_evals;
    const int crc = solve_impl(gc, cg, n, x, A, w0, v, w_out, oc, cinf, ws, st, false, judged, used);
    ws.solve_stall = 0;
    ws.carry_on = false;
    if (carry) swap_history(ws);
    if (crc < 0) return crc;
    return solve_impl(g, grid, n, x, A, w_out, v, w_out, o, inf, ws, st, need_moments_at_out);
}

int apd_solve_weights_multires(const apd_grid *grid, const apd_seeds *seeds, const double *v, double *w_out,
                               const apd_solve_opts *opts, const apd_multires_opts *mo, apd_solve_info *info,
                               apd_workspace *ws, apd_mlp *net, int32_t *used_pred, apd_stream_t stream) {
    auto t0 = std::chrono::steady_clock::now();
    apd_solve_info inf, cinf;
    std::memset(&inf, 0, sizeof inf);
    std::memset(&cinf, 0, sizeof cinf);
    GridDev g, gc;
    apd_grid cg;
    apd_solve_opts o;
    apd_multires_opts m;
    apd_multires_opts_default(&m);
    if (mo) m = *mo;
    cudaStream_t st = (cudaStream_t)stream;
    int used = 0;
    int rc = solve_entry(grid, seeds, v, w_out, opts, g, o, ws, st);
    if (rc == APD_OK && net && warmstart_dim(net) != g.dim) rc = APD_ERR_ARG;
    if (rc == APD_OK) rc = coarse_grid(grid, m, cg, gc);
    const double *w0 = seeds->w;
    if (rc == APD_OK && net) {
        rc = predict_start(grid, seeds, v, net, ws->w, stream);
        w0 = ws->w.wpred;
    }
    if (rc == APD_OK)
        rc = c2f_solve(g, grid, gc, &cg, seeds->n, seeds->x, seeds->A, w0, v, w_out, o, m, inf, cinf, ws->w, st,
                       net != nullptr, &used, false);
    if (rc >= 0) cudaStreamSynchronize(st);
    if (used_pred) *used_pred = used;
    inf.status = rc;
    inf.solves += cinf.solves;
    inf.rescored_fp64 += cinf.rescored_fp64;
    inf.coarse_evaluations = cinf.evaluations;
    inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (info) *info = inf;
    return rc;
}

int apd_lloyd_multires(const apd_grid *grid, const apd_seeds *seeds, const double *v, int32_t rounds,
                       double *x_out, double *w_out, const apd_solve_opts *opts, const apd_multires_opts *mo,
                       apd_solve_info *info, apd_workspace *ws, apd_mlp *net, int32_t *used_pred,
                       apd_stream_t stream) {
    auto t0 = std::chrono::steady_clock::now();
    apd_solve_info inf, cinf;
    std::memset(&inf, 0, sizeof inf);
    std::memset(&cinf, 0, sizeof cinf);
    GridDev g, gc;
    apd_grid cg;
    apd_solve_opts o;
    apd_multires_opts m;
    apd_multires_opts_default(&m);
    if (mo) m = *mo;
    cudaStream_t st = (cudaStream_t)stream;
    int used = 0, worst = APD_OK;
    int rc = solve_entry(grid, seeds, v, w_out, opts, g, o, ws, st);
    if (rc == APD_OK && (!x_out || rounds < 0)) rc = APD_ERR_ARG;
    if (rc == APD_OK && net && warmstart_dim(net) != g.dim) rc = APD_ERR_ARG;
    if (rc == APD_OK) rc = coarse_grid(grid, m, cg, gc);
    const int n = seeds->n;
    const double *w0 = w_out;
    if (rc == APD_OK && net) {
        rc = predict_start(grid, seeds, v, net, ws->w, stream);
        w0 = ws->w.wpred;
    }
    if (rc == APD_OK && x_out != seeds->x)
        rc = cuda_ok(cudaMemcpyAsync(x_out, seeds->x, (size_t)n * g.dim * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (rc == APD_OK && w_out != seeds->w)
        rc = cuda_ok(cudaMemcpyAsync(w_out, seeds->w, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (rc == APD_OK && m.carry_history && rounds > 0) rc = carry_begin(ws->w);
    for (int k = 0; rc == APD_OK && k <= rounds; ++k) {
        const bool last = k == rounds;
        const int r = c2f_solve(g, grid, gc, &cg, n, x_out, seeds->A, k == 0 ? w0 : w_out, v, w_out, o, m, inf, cinf,
                                ws->w, st, k == 0 && net != nullptr, k == 0 ? &used : nullptr, !last);
        if (r < 0) {
            rc = r;
            break;
        }
        if (r > worst) worst = r;
        if (!last) {
            // the workspace moments belong to (x_out, w_out): move seeds to the discrete centroids
            ws->w.kernel_launches += 1;
            rc = cuda_ok(launch_centroids(g, n, x_out, ws->w.moments, x_out, st));
        }
    }
    if (ws) {
        ws->w.carry_enabled = false;
        ws->w.carry.valid = false;
    }
    if (rc == APD_OK) rc = worst;
    if (rc >= 0) cudaStreamSynchronize(st);
    if (used_pred) *used_pred = used;
    inf.status = rc;
    inf.solves += cinf.solves;
    inf.rescored_fp64 += cinf.rescored_fp64;
    inf.coarse_evaluations = cinf.evaluations;
    inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (info) *info = inf;
    return rc;
}

static int lloyd_round(const GridDev &g, const apd_grid *grid, int n, const double *x, const double *A,
                       const double *w0, const double *v, double *x_out, double *w_out,
                       const apd_solve_opts &o, apd_solve_info &inf, Workspace &ws, cudaStream_t st,
                       int &worst) {
    int rc = solve_impl(g, grid, n, x, A, w0, v, w_out, o, inf, ws, st, true);
    if (rc < 0) return rc;
    if (rc > worst) worst = rc;
    // the workspace moments belong to (x, w_out): move seeds to the discrete centroids
    ws.kernel_launches += 1;
    return cuda_ok(launch_centroids(g, n, x, ws.moments, x_out, st));
}

int apd_lloyd_step(const apd_grid *grid, const apd_seeds *seeds, const double *v, double *x_out,
                   double *w_out, const apd_solve_opts *opts, apd_solve_info *info,
                   apd_workspace *ws, apd_stream_t stream) {
    auto t0 = std::chrono::steady_clock::now();
    apd_solve_info inf;
    std::memset(&inf, 0, sizeof inf);
    GridDev g;
    apd_solve_opts o;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = solve_entry(grid, seeds, v, w_out, opts, g, o, ws, st);
    if (rc == APD_OK && !x_out) rc = APD_ERR_ARG;
    int worst = APD_OK;
    if (rc == APD_OK) {
        rc = lloyd_round(g, grid, seeds->n, seeds->x, seeds->A, seeds->w, v, x_out, w_out, o, inf, ws->w,
                         st, worst);
        if (rc == APD_OK) rc = worst;
    }
    if (rc >= 0) cudaStreamSynchronize(st);
    inf.status = rc;
    inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (info) *info = inf;
    return rc;
}

int apd_lloyd(const apd_grid *grid, const apd_seeds *seeds, const double *v, int32_t rounds,
              double *x_out, double *w_out, const apd_solve_opts *opts, apd_solve_info *info,
              apd_workspace *ws, apd_stream_t stream) {
    auto t0 = std::chrono::steady_clock::now();
    apd_solve_info inf;
    std::memset(&inf, 0, sizeof inf);
    GridDev g;
    apd_solve_opts o;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = solve_entry(grid, seeds, v, w_out, opts, g, o, ws, st);
    if (rc == APD_OK && (!x_out || rounds < 0)) rc = APD_ERR_ARG;
    int worst = APD_OK;
    if (rc == APD_OK) {
        const int n = seeds->n;
        if (x_out != seeds->x)
            rc = cuda_ok(cudaMemcpyAsync(x_out, seeds->x, (size_t)n * g.dim * sizeof(double),
                                         cudaMemcpyDeviceToDevice, st));
        if (rc == APD_OK && w_out != seeds->w)
            rc = cuda_ok(cudaMemcpyAsync(w_out, seeds->w, (size_t)n * sizeof(double),
                                         cudaMemcpyDeviceToDevice, st));
        for (int k = 0; rc == APD_OK && k < rounds; ++k)
            rc = lloyd_round(g, grid, n, x_out, seeds->A, w_out, v, x_out, w_out, o, inf, ws->w, st, worst);
        if (rc == APD_OK) {
            rc = solve_impl(g, grid, n, x_out, seeds->A, w_out, v, w_out, o, inf, ws->w, st, false);
            if (rc >= 0 && rc > worst) worst = rc;
            if (rc >= 0) rc = worst;
        }
    }
    if (rc >= 0) cudaStreamSynchronize(st);
    inf.status = rc;
    inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (info) *info = inf;
    return rc;
}

int64_t apd_choose_resolution(int32_t dim, double v_min, double eps, double domain_measure_) {
    if ((dim != 2 && dim != 3) || !(v_min > 0.0) || !(eps > 0.0) || !(domain_measure_ > 0.0) ||
        !std::isfinite(v_min) || !std::isfinite(domain_measure_))
        return -1;
    const double bound = eps * v_min / std::pow(2.0, dim);
    const double t = domain_measure_ / bound;
    int64_t m = (int64_t)std::ceil(std::pow(t, 1.0 / dim) - 1e-9);
    if (m < 1) m = 1;
    auto fits = [&](int64_t mm) { return domain_measure_ / std::pow((double)mm, dim) <= bound * (1.0 + 1e-12); };
    while (!fits(m)) ++m;
    while (m > 1 && fits(m - 1)) --m;
    return m;
}

}  // extern "C"
