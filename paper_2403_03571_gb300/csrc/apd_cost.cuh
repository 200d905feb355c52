// Exact-arithmetic helpers shared by the scoring kernels: the FP64 cost with
// the reference operation order, and the FP32 direct-form cost with a
// rigorous per-seed rounding bound.
#pragma once

#include "apd_internal.cuh"

namespace apd {

// |y - x|^2_A - w in FP64 with the reference operation order of the cost
// matrix: d = y - x; q = sum_a sum_b (d_a * A_ab) * d_b (a outer, b inner,
// from 0, each operation rounded separately, no FMA); C = q - w.
// The quadratic part q = |y - x|^2_A alone, with the operation order of cost64.
template <int D>
__device__ __forceinline__ double quad64(const double *y, const double *__restrict__ xi, const double *__restrict__ Ai) {
    double d[D];
#pragma unroll
    for (int a = 0; a < D; ++a) d[a] = __dsub_rn(y[a], xi[a]);
    double q = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) q = __dadd_rn(q, __dmul_rn(__dmul_rn(d[a], Ai[a * D + b]), d[b]));
    return q;
}

template <int D>
__device__ __forceinline__ double cost64(const double *y, const double *__restrict__ xi,
                                         const double *__restrict__ Ai, double wi) {
    double d[D];
#pragma unroll
    for (int a = 0; a < D; ++a) d[a] = __dsub_rn(y[a], xi[a]);
    double q = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) q = __dadd_rn(q, __dmul_rn(__dmul_rn(d[a], Ai[a * D + b]), d[b]));
    return __dsub_rn(q, wi);
}

// Grid indices k of pixel j, its FP64 centre y = lo + (k + 1/2) h (the
// reference arithmetic) and the FP32 high/low split of y; lane a computes axis
// a, every lane of the warp receives all of them.
template <int D>
__device__ __forceinline__ void pixel_centre_warp(const GridDev &g, const long long j, int (&k)[3], double (&y)[D],
                                                  float (&yh)[3], float (&yl)[3]) {
    const int lane = threadIdx.x & 31;
    long long rr = j;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        k[a] = (int)(rr % g.res[a]);
        rr /= g.res[a];
    }
    double ya = 0.0;
    float yha = 0.f, yla = 0.f;
    if (lane < D) {
        const int ka = lane == 0 ? k[0] : (lane == 1 ? k[1] : k[2]);
        const double loa = lane == 0 ? g.lo[0] : (lane == 1 ? g.lo[1] : g.lo[D - 1]);
        const double ha = lane == 0 ? g.h[0] : (lane == 1 ? g.h[1] : g.h[D - 1]);
        ya = __dadd_rn(loa, __dmul_rn((double)ka + 0.5, ha));
        yha = (float)ya;
        yla = (float)(ya - (double)yha);
    }
#pragma unroll
    for (int a = 0; a < D; ++a) {
        y[a] = __shfl_sync(0xffffffffu, ya, a);
        yh[a] = __shfl_sync(0xffffffffu, yha, a);
        yl[a] = __shfl_sync(0xffffffffu, yla, a);
    }
}

template <int D>
__device__ __forceinline__ void cost32_bound(const SeedRec32 &r, const float (&yh)[3], const float (&yl)[3],
                                             float wrh, float wrl, float &c, float &E) {
    float d[D];
#pragma unroll
    for (int a = 0; a < D; ++a) d[a] = (yh[a] - r.xh[a]) + (yl[a] - r.xl[a]);
    float q, qa;
    if (D == 3) {
        const float A00 = r.a[0], A01 = r.a[1], A02 = r.a[2], A11 = r.a[3], A12 = r.a[4], A22 = r.a[5];
        const float t0 = fmaf(A02, d[2], fmaf(A01, d[1], A00 * d[0]));
        const float t1 = fmaf(A12, d[2], fmaf(A11, d[1], A01 * d[0]));
        const float t2 = fmaf(A22, d[2], fmaf(A12, d[1], A02 * d[0]));
        q = fmaf(d[2], t2, fmaf(d[1], t1, d[0] * t0));
        const float e0 = fabsf(d[0]), e1 = fabsf(d[1]), e2 = fabsf(d[2]);
        const float s0 = fmaf(fabsf(A02), e2, fmaf(fabsf(A01), e1, fabsf(A00) * e0));
        const float s1 = fmaf(fabsf(A12), e2, fmaf(fabsf(A11), e1, fabsf(A01) * e0));
        const float s2 = fmaf(fabsf(A22), e2, fmaf(fabsf(A12), e1, fabsf(A02) * e0));
        qa = fmaf(e2, s2, fmaf(e1, s1, e0 * s0));
    } else {
        const float A00 = r.a[0], A01 = r.a[1], A11 = r.a[2];
        const float t0 = fmaf(A01, d[1], A00 * d[0]);
        const float t1 = fmaf(A11, d[1], A01 * d[0]);
        q = fmaf(d[1], t1, d[0] * t0);
        const float e0 = fabsf(d[0]), e1 = fabsf(d[1]);
        const float s0 = fmaf(fabsf(A01), e1, fabsf(A00) * e0);
        const float s1 = fmaf(fabsf(A11), e1, fabsf(A01) * e0);
        qa = fmaf(e1, s1, e0 * s0);
    }
    const float wp = (r.wh - wrh) + (r.wl - wrl);
    c = q - wp;
    E = 16.f * 5.9604644775390625e-8f * (qa + fabsf(wp) + fabsf(c)) + 1e-37f;
}

// FP32 direct-form cost and bound for a pixel given relative to a centre c:
// y = c + yp with c = ch + cl (FP32 high/low split of an FP64 point) and yp an
// FP32 offset with |yp - (y - c)| <= 2u |yp|.  d = ((ch - xh) + (cl - xl)) + yp
// then errs by at most u (5 |yp| + 3 |d|) per axis, which adds
// 12 u sum_ab |A_ab| |yp_a| |d_b| to the bound of cost32_bound.
template <int D>
__device__ __forceinline__ void cost32_bound_rel(const SeedRec32 &r, const float (&ch)[3], const float (&cl)[3],
                                                 const float (&yp)[3], float wrh, float wrl, float &c,
                                                 float &E) {
    float d[D];
#pragma unroll
    for (int a = 0; a < D; ++a) d[a] = ((ch[a] - r.xh[a]) + (cl[a] - r.xl[a])) + yp[a];
    float q, qa, ya;
    if (D == 3) {
        const float A00 = r.a[0], A01 = r.a[1], A02 = r.a[2], A11 = r.a[3], A12 = r.a[4], A22 = r.a[5];
        const float t0 = fmaf(A02, d[2], fmaf(A01, d[1], A00 * d[0]));
        const float t1 = fmaf(A12, d[2], fmaf(A11, d[1], A01 * d[0]));
        const float t2 = fmaf(A22, d[2], fmaf(A12, d[1], A02 * d[0]));
        q = fmaf(d[2], t2, fmaf(d[1], t1, d[0] * t0));
        const float e0 = fabsf(d[0]), e1 = fabsf(d[1]), e2 = fabsf(d[2]);
        const float s0 = fmaf(fabsf(A02), e2, fmaf(fabsf(A01), e1, fabsf(A00) * e0));
        const float s1 = fmaf(fabsf(A12), e2, fmaf(fabsf(A11), e1, fabsf(A01) * e0));
        const float s2 = fmaf(fabsf(A22), e2, fmaf(fabsf(A12), e1, fabsf(A02) * e0));
        qa = fmaf(e2, s2, fmaf(e1, s1, e0 * s0));
        ya = fmaf(fabsf(yp[2]), s2, fmaf(fabsf(yp[1]), s1, fabsf(yp[0]) * s0));
    } else {
        const float A00 = r.a[0], A01 = r.a[1], A11 = r.a[2];
        const float t0 = fmaf(A01, d[1], A00 * d[0]);
        const float t1 = fmaf(A11, d[1], A01 * d[0]);
        q = fmaf(d[1], t1, d[0] * t0);
        const float e0 = fabsf(d[0]), e1 = fabsf(d[1]);
        const float s0 = fmaf(fabsf(A01), e1, fabsf(A00) * e0);
        const float s1 = fmaf(fabsf(A11), e1, fabsf(A01) * e0);
        qa = fmaf(e1, s1, e0 * s0);
        ya = fmaf(fabsf(yp[1]), s1, fabsf(yp[0]) * s0);
    }
    const float wp = (r.wh - wrh) + (r.wl - wrl);
    c = q - wp;
    E = 5.9604644775390625e-8f * (16.f * (qa + fabsf(wp) + fabsf(c)) + 12.f * ya) + 1e-37f;
}

// Rescoring of a queued pixel, one warp per pixel, lanes over seeds.
// Pass 1: FP32 direct-form cost of every seed with y - x formed from FP32
// high/low splits (error <= 2u |y - x|), and a per-seed rounding bound
//     E_k = 16 u (sum_ab |A_ab| |d_a| |d_b| + |w'_k| + |C_k|),
// covering the roundings of d, A, the two 3-term dot products, w' and the final
// subtraction (about 11 u of them) and the FP64 reference's own error.  The
// threshold is min_k (C_k + E_k).  Pass 2: every seed with C_k - E_k <= threshold
// is recomputed in FP64 with the reference arithmetic; the smallest FP64 cost
// wins, ties to the lowest index.  Any seed left out has an exact cost above the
// exact minimum by more than the FP64 rounding, so the result equals the FP64
// argmin over all seeds.
//
// Pruned form (group bounds available and the scoring pass's best seed `gi`
// known): the threshold is C_gi + E_gi (>= the full threshold, so the
// candidate set only grows), and a group of 32 scan-order seeds is skipped
// when a lower bound of the exact cost of all its seeds at y,
//     lam_g dist(y, box_g)^2 + (w_ref - wmax_g),
// evaluated with outward rounding, exceeds the threshold by a margin of
// 1e-6 (|thr| + |bound| + |w_ref - wmax_g|) (far above the FP64 rounding of any
// seed whose exact cost is near the bound): none of its seeds can be a
// candidate, nor the FP64 argmin.
template <int D>
__device__ __forceinline__ void rescore_finish(const GridDev &g, const int n, const long long j, const int (&k)[3],
                                               double best, int bi, DevScalars *__restrict__ sc,
                                               unsigned long long *__restrict__ gmom, int32_t *__restrict__ labels,
                                               const int32_t *__restrict__ old_labels = nullptr) {
    constexpr int K = moment_width(D);
    const int lane = threadIdx.x & 31;
    // smallest (cost, index) over the few lanes holding a candidate (FP64 compares
    // are slow on this part: visit those lanes only, every lane computing the same)
    unsigned cm = __ballot_sync(0xffffffffu, bi != 0x7fffffff);
    double b = __longlong_as_double(0x7ff0000000000000ll);
    int ib = 0x7fffffff;
    while (cm) {
        const int l = __ffs(cm) - 1;
        cm &= cm - 1u;
        const double ob = __shfl_sync(0xffffffffu, best, l);
        const int oi = __shfl_sync(0xffffffffu, bi, l);
        if (ob < b || (ob == b && oi < ib)) {
            b = ob;
            ib = oi;
        }
    }
    best = b;
    bi = ib;
    if (lane == 0) {
        if (bi < 0 || bi >= n) {
            atomicOr(&sc->status, ST_BAD_LABEL);
        } else {
            if (labels) labels[j] = bi;
            // with old_labels the moments hold another labelling's sums: move the
            // pixel's words from its old cell to its new one (two's-complement
            // subtraction; nothing when the label is unchanged)
            int old = old_labels ? old_labels[j] : -1;
            if (old >= n) old = -1;
            if (old != bi) {
                unsigned long long u[3];
#pragma unroll
                for (int a = 0; a < D; ++a) u[a] = 2ull * (unsigned long long)k[a] + 1ull;
                unsigned long long words[K];
                words[0] = 1ull;
#pragma unroll
                for (int a = 0; a < D; ++a) words[1 + a] = u[a];
                int e = 1 + D;
#pragma unroll
                for (int a = 0; a < D; ++a)
#pragma unroll
                    for (int b = a; b < D; ++b) words[e++] = u[a] * u[b];
                unsigned long long *o = gmom + (size_t)bi * K;
#pragma unroll
                for (int v = 0; v < K; ++v) atomicAdd(&o[v], words[v]);
                if (old >= 0) {
                    unsigned long long *q = gmom + (size_t)old * K;
#pragma unroll
                    for (int v = 0; v < K; ++v) atomicAdd(&q[v], 0ull - words[v]);
                }
            }
        }
    }
}

// Optional pruning inputs of rescore_pixel (all null / 0 disables pruning).
struct RescorePrune {
    const GroupBound *groups;   // [n_groups] bounds of the scan-order groups
    const SeedRec32 *r32s;      // [n_groups * 32] records in scan order
    const int32_t *perm;        // scan position -> seed index (null: identity)
    int n_groups;
};

template <int D>
__device__ __forceinline__ void rescore_pixel(const GridDev &g, const int n, const double *__restrict__ x,
                                              const double *__restrict__ A, const double *__restrict__ w,
                                              const SeedRec32 *__restrict__ r32, const uint32_t fj, const int gi,
                                              const float wrh, const float wrl, const RescorePrune &pr,
                                              DevScalars *__restrict__ sc, unsigned long long *__restrict__ gmom,
                                              int32_t *__restrict__ labels,
                                              const int32_t *__restrict__ old_labels = nullptr) {
    const int lane = threadIdx.x & 31;
    const long long j = (long long)fj;
    int k[3] = {0, 0, 0};
    double y[D];
    float yh[3] = {0.f, 0.f, 0.f}, yl[3] = {0.f, 0.f, 0.f};
    pixel_centre_warp<D>(g, j, k, y, yh, yl);
    double best = __longlong_as_double(0x7ff0000000000000ll);
    int bi = 0x7fffffff;
    float thr = __int_as_float(0x7f800000);
    if (pr.groups && gi >= 0 && gi < n) {
        float c, E;
        cost32_bound<D>(r32[gi], yh, yl, wrh, wrl, c, E);
        thr = c + E;
    }
    if (thr < __int_as_float(0x7f800000)) {
        for (int base = 0; base < pr.n_groups; base += 32) {
            const int grp = base + lane;
            bool keep = false;
            if (grp < pr.n_groups) {
                const GroupBound gb = pr.groups[grp];
                float d2 = 0.f;
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    const float slack = 1e-6f * (fabsf(yh[a]) + fabsf(gb.lo[a]) + fabsf(gb.hi[a]));
                    const float t = fmaxf(fmaxf(gb.lo[a] - yh[a], yh[a] - gb.hi[a]) - slack, 0.f);
                    d2 = fmaf(t, t, d2);
                }
                const float wpart = gb.wgap;
                const float lb = __fmul_rd(__fmul_rd(gb.lam, d2), 1.f - 1e-5f) + wpart;
                keep = !(lb > thr + 1e-6f * (fabsf(thr) + fabsf(lb) + fabsf(wpart)) + 1e-30f);
            }
            unsigned mask = __ballot_sync(0xffffffffu, keep);
            while (mask) {
                const int kk = __ffs(mask) - 1;
                mask &= mask - 1;
                const int pos = (base + kk) * 32 + lane;
                if (pos < n) {
                    const int s = pr.perm ? pr.perm[pos] : pos;
                    float c, E;
                    cost32_bound<D>(pr.r32s[pos], yh, yl, wrh, wrl, c, E);
                    if (c - E <= thr) {
                        const double c64 = cost64<D>(y, x + (size_t)s * D, A + (size_t)s * D * D, w[s]);
                        if (c64 < best || (c64 == best && s < bi)) {
                            best = c64;
                            bi = s;
                        }
                    }
                }
            }
        }
        rescore_finish<D>(g, n, j, k, best, bi, sc, gmom, labels, old_labels);
        return;
    }
    // full scan: pass 1, threshold = min over seeds of (C + E)
    for (int s = lane; s < n; s += 32) {
        float c, E;
        cost32_bound<D>(r32[s], yh, yl, wrh, wrl, c, E);
        thr = fminf(thr, c + E);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) thr = fminf(thr, __shfl_xor_sync(0xffffffffu, thr, off));
    // pass 2: FP64 reference cost of the candidates
    for (int s = lane; s < n; s += 32) {
        float c, E;
        cost32_bound<D>(r32[s], yh, yl, wrh, wrl, c, E);
        if (!(c - E <= thr)) continue;
        const double c64 = cost64<D>(y, x + (size_t)s * D, A + (size_t)s * D * D, w[s]);
        if (c64 < best) {
            best = c64;
            bi = s;
        }
    }
    rescore_finish<D>(g, n, j, k, best, bi, sc, gmom, labels, old_labels);
}

// Relative gap of the two smallest costs at pixel j (one warp), the quantity
// the near-tie tolerance of the labels is stated in:
//     gap_j = (c_(2) - c_(1)) / (|q_(1)| + |q_(2)| + |w_(1)| + |w_(2)|),
// c_(1) <= c_(2) the two smallest costs of Algorithm 1's cost matrix at y_j
// (ordered by cost, then seed index, so an exact tie gives 0), q the quadratic
// part of each, +inf for a single seed.  Both costs come from the FP64
// reference arithmetic (cost64), so the value is that of a full FP64 scan.
// Search: the 32-seed groups are visited in increasing order of their cost
// lower bound (lanes over groups, in blocks of 32 groups); in a visited group
// every lane takes one seed's FP32 direct-form cost c with its bound E, the
// two smallest upper bounds c + E seen so far give t2 >= the exact second
// smallest cost, seeds with c - E <= t2 are recomputed in FP64, and the
// remaining groups of a block are skipped once the smallest bound among them
// exceeds t2 (the margins are those of rescore_pixel).
__device__ __forceinline__ unsigned f_key(float v) {
    const unsigned u = __float_as_uint(v);
    return u ^ ((u >> 31) ? 0xffffffffu : 0x80000000u);
}
__device__ __forceinline__ float f_unkey(unsigned k) {
    return __uint_as_float(k ^ ((k >> 31) ? 0x80000000u : 0xffffffffu));
}

template <int D>
__device__ __forceinline__ double gap_pixel(const GridDev &g, const int n, const double *__restrict__ x,
                                            const double *__restrict__ A, const double *__restrict__ w,
                                            const long long j, const float wrh, const float wrl,
                                            const RescorePrune &pr) {
    const int lane = threadIdx.x & 31;
    int k[3] = {0, 0, 0};
    double y[D];
    float yh[3] = {0.f, 0.f, 0.f}, yl[3] = {0.f, 0.f, 0.f};
    pixel_centre_warp<D>(g, j, k, y, yh, yl);
    const double inf = __longlong_as_double(0x7ff0000000000000ll);
    if (n < 2) return inf;
    const float finf = __int_as_float(0x7f800000);
    float t1 = finf, t2 = finf;                          // warp-uniform
    double c1 = inf, c2 = inf;                           // this lane's two smallest (cost, index)
    int i1 = 0x7fffffff, i2 = 0x7fffffff;
    for (int base = 0; base < pr.n_groups; base += 32) {
        const int grp = base + lane;
        float lb = finf, wpart = 0.f;
        if (grp < pr.n_groups) {
            const GroupBound gb = pr.groups[grp];
            float d2 = 0.f;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const float slack = 1e-6f * (fabsf(yh[a]) + fabsf(gb.lo[a]) + fabsf(gb.hi[a]));
                const float t = fmaxf(fmaxf(gb.lo[a] - yh[a], yh[a] - gb.hi[a]) - slack, 0.f);
                d2 = fmaf(t, t, d2);
            }
            wpart = gb.wgap;
            lb = __fmul_rd(__fmul_rd(gb.lam, d2), 1.f - 1e-5f) + wpart;
        }
        unsigned live = __ballot_sync(0xffffffffu, grp < pr.n_groups);
        while (live) {
            const unsigned key = ((live >> lane) & 1u) ? f_key(lb) : 0xffffffffu;
            const unsigned kmin = __reduce_min_sync(0xffffffffu, key);
            const int kg = __ffs(__ballot_sync(0xffffffffu, ((live >> lane) & 1u) && key == kmin)) - 1;
            const float lbk = __shfl_sync(0xffffffffu, lb, kg);
            const float wpk = __shfl_sync(0xffffffffu, wpart, kg);
            if (t2 < finf && lbk > t2 + 1e-6f * (fabsf(t2) + fabsf(lbk) + fabsf(wpk)) + 1e-30f) break;
            live &= ~(1u << kg);
            const int pos = (base + kg) * 32 + lane;
            float c = finf, E = 0.f;
            int s = -1;
            if (pos < n) {
                s = pr.perm ? pr.perm[pos] : pos;
                cost32_bound<D>(pr.r32s[pos], yh, yl, wrh, wrl, c, E);
            }
            // the two smallest upper bounds of this group, merged into (t1, t2)
            const unsigned ku = pos < n ? f_key(c + E) : 0xffffffffu;
            const unsigned k1 = __reduce_min_sync(0xffffffffu, ku);
            const unsigned k2 = __popc(__ballot_sync(0xffffffffu, ku == k1)) >= 2
                                    ? k1
                                    : __reduce_min_sync(0xffffffffu, ku == k1 ? 0xffffffffu : ku);
            const float m1 = k1 == 0xffffffffu ? finf : f_unkey(k1);
            const float m2 = k2 == 0xffffffffu ? finf : f_unkey(k2);
            const float nt1 = fminf(t1, m1);
            t2 = fminf(fmaxf(t1, m1), fminf(t2, m2));
            t1 = nt1;
            if (pos < n && c - E <= t2) {
                const double c64 = cost64<D>(y, x + (size_t)s * D, A + (size_t)s * D * D, w[s]);
                if (c64 < c1 || (c64 == c1 && s < i1)) {
                    c2 = c1;
                    i2 = i1;
                    c1 = c64;
                    i1 = s;
                } else if (c64 < c2 || (c64 == c2 && s < i2)) {
                    c2 = c64;
                    i2 = s;
                }
            }
        }
    }
    // merge the lanes' pairs: the two smallest (cost, index) of the warp
    double b1 = c1, b2 = c2;
    int j1 = i1, j2 = i2;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double o1 = __shfl_xor_sync(0xffffffffu, b1, off), o2 = __shfl_xor_sync(0xffffffffu, b2, off);
        const int p1 = __shfl_xor_sync(0xffffffffu, j1, off), p2 = __shfl_xor_sync(0xffffffffu, j2, off);
        // two smallest of the sorted pairs (b1, b2) and (o1, o2)
        const bool mine_first = b1 < o1 || (b1 == o1 && j1 < p1);
        const double f1 = mine_first ? b1 : o1;
        const int g1 = mine_first ? j1 : p1;
        const double sa = mine_first ? b2 : b1, sb = mine_first ? o1 : o2;  // second candidates
        const int ja = mine_first ? j2 : j1, jb = mine_first ? p1 : p2;
        const bool a_second = sa < sb || (sa == sb && ja < jb);
        b1 = f1;
        j1 = g1;
        b2 = a_second ? sa : sb;
        j2 = a_second ? ja : jb;
    }
    if (j1 >= n || j2 >= n || !(b2 < inf)) return inf;
    const double q1 = quad64<D>(y, x + (size_t)j1 * D, A + (size_t)j1 * D * D);
    const double q2 = quad64<D>(y, x + (size_t)j2 * D, A + (size_t)j2 * D * D);
    const double sc = fabs(q1) + fabs(q2) + fabs(w[j1]) + fabs(w[j2]);
    return sc > 0.0 ? (b2 - b1) / sc : (b2 - b1 > 0.0 ? inf : 0.0);
}

}  // namespace apd
