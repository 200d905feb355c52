// Exact-arithmetic helpers shared by the scoring kernels: the FP64 cost with
// the reference operation order, and the FP32 direct-form cost with a
// rigorous per-seed rounding bound.
#pragma once

#include "apd_internal.cuh"

namespace apd {

// |y - x|^2_A - w in FP64 with the reference operation order of the cost
// matrix: d = y - x; q = sum_a sum_b (d_a * A_ab) * d_b (a outer, b inner,
// from 0, each operation rounded separately, no FMA); C = q - w.
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
                                               unsigned long long *__restrict__ gmom, int32_t *__restrict__ labels) {
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
            unsigned long long u[3];
#pragma unroll
            for (int a = 0; a < D; ++a) u[a] = 2ull * (unsigned long long)k[a] + 1ull;
            unsigned long long *o = gmom + (size_t)bi * K;
            atomicAdd(&o[0], 1ull);
#pragma unroll
            for (int a = 0; a < D; ++a) atomicAdd(&o[1 + a], u[a]);
            int e = 1 + D;
#pragma unroll
            for (int a = 0; a < D; ++a)
#pragma unroll
                for (int b = a; b < D; ++b) atomicAdd(&o[e++], u[a] * u[b]);
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
                                              int32_t *__restrict__ labels) {
    const int lane = threadIdx.x & 31;
    const long long j = (long long)fj;
    int k[3] = {0, 0, 0};
    long long rr = j;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        k[a] = (int)(rr % g.res[a]);
        rr /= g.res[a];
    }
    // the pixel centre (FP64) and its FP32 split: lane a computes axis a
    double y[D];
    float yh[3] = {0.f, 0.f, 0.f}, yl[3] = {0.f, 0.f, 0.f};
    {
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
        rescore_finish<D>(g, n, j, k, best, bi, sc, gmom, labels);
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
    rescore_finish<D>(g, n, j, k, best, bi, sc, gmom, labels);
}

}  // namespace apd
