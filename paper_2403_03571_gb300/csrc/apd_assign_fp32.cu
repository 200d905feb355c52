// Algorithm 1 (pixel method) on CUDA cores in FP32, fused with the per-cell
// integer moment reduction, plus the FP64 rescoring of near ties.
//
// Scoring.  A CTA owns a tile of P x TY x TZ pixels (P along the first axis).
// Each thread owns one row of P pixels that share (k1, k2).  For seed i and a
// row, write the cost of eq. (2.1) / Algorithm 1 around the row's centre
// point z = (c0, y1, y2) and the offset delta = y0 - c0 of each pixel:
//     C(delta) = a + delta * (b + A00 * delta)
//     a = (z - x_i)^T A_i (z - x_i) - (w_i - w_ref),   b = 2 (A_i (z - x_i))_0,
// so a, b cost a handful of FMAs per (row, seed) and every pixel of the row
// costs two FMAs (issued as one packed f32x2 FMA per pixel pair).  Positions
// are recentred on the CTA in FP64 before rounding to FP32, and w_ref = max w
// makes every cost non-negative, so the rounding error of a computed cost is
// bounded by a small multiple of u * T with
//     T <= Lambda (R + sqrt(C*/lambda))^2 + C*
// (Lambda >= max ||A_i||_F, lambda <= min lambda_min(A_i), R = tile
// half-diagonal, C* ~ the best cost of the pixel).  The seed's index inside a
// group of 32 is packed into the 5 low mantissa bits of the cost, so one
// 3-input min and two 2-input min/max keep the two smallest costs of a pixel
// with the index of the smallest.  A pixel whose best and second-best FP32
// costs are closer than twice the bound is queued and rescored in FP64 with
// the reference arithmetic of the cost matrix; every other label is the exact
// argmin.
//
// Seeds stream through shared memory in chunks of 256 records, fetched with
// 1-D bulk async copies (TMA) into a double buffer; each chunk is transformed
// once per CTA into the row-form coefficients above.
//
// Pruning (optional).  Lower bounds of the exact cost over a warp's pixel box,
// per 32-seed group and per seed (lambda_min times the squared distance plus
// the weight gap w_ref - w), skip the groups and seed pairs that cannot enter
// any pixel's top two; groups are taken nearest-bound first and re-tested as
// the second-best costs fall.  Labels and moments equal the dense sweep's.
//
// Moments.  Each thread run-length encodes its row (neighbouring pixels share a
// label), accumulates count, sum u and sum u u^T (u = 2k + 1) per run; the lanes
// of a warp holding the same label sum their runs with shuffles and one lane
// adds the sums to a per-CTA shared-memory hash table keyed by label; the table
// is flushed to the global int64 moments with one atomic per (cell, word).
#include "apd_fp32_tile.cuh"
#include "apd_cost.cuh"

namespace apd {

namespace {

using namespace fp32;

template <int D>
struct Cfg;
template <>
struct Cfg<3> {  // 16^3 voxels, one 16-voxel row per thread
    static constexpr int TX = 1, P = 16, TY = 16, TZ = 16;
};
template <>
struct Cfg<2> {  // 64 x 64 pixels, four 16-pixel row segments per row
    static constexpr int TX = 4, P = 16, TY = 64, TZ = 1;
};

// The grid's last-axis tiles start at tile index `toff` (the first tile of the
// scoring window).
template <int D>
__global__ void __launch_bounds__(256, 2) assign_fp32_kernel(const __grid_constant__ TileSrc src, const int toff) {
    using C = Cfg<D>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    SharedLayout<D> &sm = *reinterpret_cast<SharedLayout<D> *>(smem_raw);
    init_shared<D>(sm);
    uint32_t uses[4] = {0u, 0u, 0u, 0u};
    const int by = D == 2 ? (int)blockIdx.y + toff : (int)blockIdx.y;
    const int bz = D == 3 ? (int)blockIdx.z + toff : 0;
    score_tile<D, C::TX, C::P, C::TY, C::TZ>(sm, src, blockIdx.x, by, bz, uses);
}

// One warp per queued pixel of one instance.
template <int D>
__global__ void __launch_bounds__(256)
    rescore_kernel(const GridDev g, const int n, const double *__restrict__ x,
                   const double *__restrict__ A, const double *__restrict__ w,
                   const SeedRec32 *__restrict__ r32, const uint32_t *__restrict__ flags,
                   const int32_t *__restrict__ flag_gi, const RescorePrune pr,
                   DevScalars *__restrict__ sc, unsigned long long *__restrict__ gmom,
                   int32_t *__restrict__ labels, const int32_t *__restrict__ old_labels,
                   const int *__restrict__ go) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const unsigned count = sc->flag_count;
    if (warp == 0 && (threadIdx.x & 31) == 0 && count)
        atomicAdd((unsigned long long *)&sc->rescored_total, (unsigned long long)count);
    // warps without a queued pixel leave before any FP64 instruction (they issue slowly)
    if ((unsigned)warp >= count) return;
    const double wref = dkey_inv(sc->wref_key);
    const float wrh = (float)wref;
    const float wrl = (float)(wref - (double)wrh);
    // an incremental pass: a re-decision moves words from the recorded labels'
    // cells and keeps the record; a recording writes the labels
    const bool delta = go ? *go != 0 : old_labels != nullptr;
    int32_t *lab = delta && go ? nullptr : labels;
    const int32_t *old = delta ? old_labels : nullptr;
    for (unsigned it = warp; it < count; it += nwarps)
        rescore_pixel<D>(g, n, x, A, w, r32, flags[it], flag_gi ? flag_gi[it] : -1, wrh, wrl, pr, sc, gmom, lab,
                         old);
}

// One warp per pixel: the relative gap of its two smallest FP64 costs.
template <int D>
__global__ void __launch_bounds__(256)
    tie_gap_kernel(const GridDev g, const int n, const double *__restrict__ x, const double *__restrict__ A,
                   const double *__restrict__ w, const RescorePrune pr, const DevScalars *__restrict__ sc,
                   double *__restrict__ gap) {
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const double wref = dkey_inv(sc->wref_key);
    const float wrh = (float)wref;
    const float wrl = (float)(wref - (double)wrh);
    const long long j0 = win_first(g), count = win_pixels(g);
    for (long long t = warp; t < count; t += nwarps) {
        const double v = gap_pixel<D>(g, n, x, A, w, j0 + t, wrh, wrl, pr);
        if ((threadIdx.x & 31) == 0) gap[j0 + t] = v;
    }
}

template <int D>
cudaError_t launch_assign_fp32_t(const GridDev &g, int n, Workspace &ws, int32_t *labels,
                                 unsigned long long *gmom, cudaStream_t st) {
    using C = Cfg<D>;
    const size_t smem = sizeof(SharedLayout<D>);
    constexpr unsigned bit = D == 3 ? kAttrFp32Score3 : kAttrFp32Score2;
    if (!(ws.attr_done & bit)) {
        cudaError_t e = cudaFuncSetAttribute(assign_fp32_kernel<D>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        ws.attr_done |= bit;
    }
    // tiles along the last axis that meet the window [win_lo, win_hi)
    constexpr int TL = D == 3 ? C::TZ : C::TY;
    const int toff = win_lo(g) / TL;
    const int tcount = (win_hi(g) - 1) / TL - toff + 1;
    dim3 grid((g.res[0] + C::TX * C::P - 1) / (C::TX * C::P), D == 2 ? tcount : (g.res[1] + C::TY - 1) / C::TY,
              D == 3 ? tcount : 1);
    const int n_chunks = (n + kChunk - 1) / kChunk;
    double hx = 0.5 * C::TX * C::P * g.h[0], hy = 0.5 * C::TY * g.h[1], hz = D == 3 ? 0.5 * C::TZ * g.h[2] : 0.0;
    const float R = (float)(sqrt(hx * hx + hy * hy + hz * hz) * (1.0 + 1e-6));
    const TileSrc src{g,        n,     n_chunks,   R,      ws.recs, ws.sorted ? ws.scodes : nullptr,
                      ws.sorted ? ws.perm : nullptr, gmom, ws.flags, ws.flag_gi, labels, ws.sc,
                      ws.prune ? ws.groups : nullptr, ws.pairs_scored, ws.wait_limit};
    const cudaError_t ep = record_scoring_start(ws, st);
    if (ep != cudaSuccess) return ep;
    assign_fp32_kernel<D><<<grid, C::TX * C::TY * C::TZ, smem, st>>>(src, toff);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_assign_fp32(const GridDev &g, int n, Workspace &ws, int32_t *labels,
                               unsigned long long *moments, cudaStream_t st) {
    return g.dim == 3 ? launch_assign_fp32_t<3>(g, n, ws, labels, moments, st)
                      : launch_assign_fp32_t<2>(g, n, ws, labels, moments, st);
}

cudaError_t launch_tie_gap(const GridDev &g, int n, const double *x, const double *A, const double *w,
                           Workspace &ws, double *gap, cudaStream_t st) {
    RescorePrune pr{ws.groups, ws.sorted ? ws.recs32s : ws.recs32, ws.sorted ? ws.perm : nullptr, (n + 31) / 32};
    const int blocks = ws.sms * 8;
    if (g.dim == 3)
        tie_gap_kernel<3><<<blocks, 256, 0, st>>>(g, n, x, A, w, pr, ws.sc, gap);
    else
        tie_gap_kernel<2><<<blocks, 256, 0, st>>>(g, n, x, A, w, pr, ws.sc, gap);
    return cudaGetLastError();
}

cudaError_t launch_rescore_fp64(const GridDev &g, int n, const double *x, const double *A,
                                const double *w, Workspace &ws, int32_t *labels,
                                unsigned long long *moments, cudaStream_t st, const int32_t *old_labels,
                                const int *go) {
    // one warp per queued pixel, latency-bound (dependent record loads): as many
    // resident warps as the registers allow
    int &bps = ws.rescore_bps[g.dim == 3 ? 1 : 0];
    if (!bps) {
        const cudaError_t e = g.dim == 3
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, rescore_kernel<3>, 256, 0)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, rescore_kernel<2>, 256, 0);
        if (e != cudaSuccess || bps < 1) bps = 2;
    }
    const int blocks = ws.sms * bps;
    RescorePrune pr{nullptr, nullptr, nullptr, 0};
    if (ws.groups && (!ws.sorted || ws.recs32s)) {
        pr.groups = ws.groups;
        pr.r32s = ws.sorted ? ws.recs32s : ws.recs32;
        pr.perm = ws.sorted ? ws.perm : nullptr;
        pr.n_groups = (n + 31) / 32;
    }
    if (g.dim == 3)
        rescore_kernel<3><<<blocks, 256, 0, st>>>(g, n, x, A, w, ws.recs32, ws.flags, ws.flag_gi, pr, ws.sc, moments,
                                                  labels, old_labels, go);
    else
        rescore_kernel<2><<<blocks, 256, 0, st>>>(g, n, x, A, w, ws.recs32, ws.flags, ws.flag_gi, pr, ws.sc, moments,
                                                  labels, old_labels, go);
    return cudaGetLastError();
}

}  // namespace apd
