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

}  // namespace apd
