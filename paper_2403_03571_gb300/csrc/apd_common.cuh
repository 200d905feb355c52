// Device helpers shared by the one-instance and batched kernels: block
// reductions, seed records and their statistics, the Morton sort, and the
// per-cell terms of the dual.
#pragma once

#include <float.h>

#include "apd_internal.cuh"

namespace apd {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
    return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, off));
    return v;
}

// Deterministic block sum (fixed tree), result valid in every thread.
__device__ __forceinline__ double block_sum(double v, double *sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        r = lane < nw ? sh[lane] : 0.0;
        r = warp_sum(r);
        if (lane == 0) sh[32] = r;
    }
    __syncthreads();
    return sh[32];
}

// Smallest eigenvalue of a symmetric positive-definite 2x2 or 3x3 matrix (FP64):
// 2x2 from the characteristic quadratic; 3x3 from the trigonometric solution of
// the characteristic cubic (shifted by the mean eigenvalue, scaled by the root
// mean square deviation).  Returned with a small relative safety margin.
template <int D>
__device__ __forceinline__ double lambda_min_sym(const double (&s)[D][D]) {
    if (D == 2) {
        const double m = 0.5 * (s[0][0] + s[1][1]);
        const double h = 0.5 * (s[0][0] - s[1][1]);
        const double r = sqrt(h * h + s[0][1] * s[0][1]);
        // m - r computed as det / (m + r) to avoid cancellation
        const double det = s[0][0] * s[1][1] - s[0][1] * s[0][1];
        return (det / (m + r)) * (1.0 - 1e-9);
    } else {
        const double p1 = s[0][1] * s[0][1] + s[0][2] * s[0][2] + s[1][2] * s[1][2];
        const double q = (s[0][0] + s[1][1] + s[2][2]) / 3.0;
        const double a0 = s[0][0] - q, a1 = s[1][1] - q, a2 = s[2][2] - q;
        const double p2 = a0 * a0 + a1 * a1 + a2 * a2 + 2.0 * p1;
        if (!(p2 > 1e-30 * q * q)) return q * (1.0 - 1e-9);  // multiple of the identity
        const double p = sqrt(p2 / 6.0);
        const double b00 = a0 / p, b11 = a1 / p, b22 = a2 / p;
        const double b01 = s[0][1] / p, b02 = s[0][2] / p, b12 = s[1][2] / p;
        double r = 0.5 * (b00 * (b11 * b22 - b12 * b12) - b01 * (b01 * b22 - b12 * b02) +
                          b02 * (b01 * b12 - b11 * b02));
        r = fmin(1.0, fmax(-1.0, r));
        const double phi = acos(r) / 3.0;
        const double lmin = q + 2.0 * p * cos(phi + 2.0943951023931957);  // + 2 pi / 3
        // relative and absolute margins cover the rounding of the formula
        return fmax(lmin * (1.0 - 1e-9) - 1e-12 * q, 0.0);
    }
}

// Largest eigenvalue of the same matrices (2x2: m + r; 3x3: the largest root
// of the trigonometric solution), with a small relative margin upwards.
template <int D>
__device__ __forceinline__ double lambda_max_sym(const double (&s)[D][D]) {
    if (D == 2) {
        const double m = 0.5 * (s[0][0] + s[1][1]);
        const double h = 0.5 * (s[0][0] - s[1][1]);
        return (m + sqrt(h * h + s[0][1] * s[0][1])) * (1.0 + 1e-9);
    } else {
        const double p1 = s[0][1] * s[0][1] + s[0][2] * s[0][2] + s[1][2] * s[1][2];
        const double q = (s[0][0] + s[1][1] + s[2][2]) / 3.0;
        const double a0 = s[0][0] - q, a1 = s[1][1] - q, a2 = s[2][2] - q;
        const double p2 = a0 * a0 + a1 * a1 + a2 * a2 + 2.0 * p1;
        if (!(p2 > 1e-30 * q * q)) return q * (1.0 + 1e-9);
        const double p = sqrt(p2 / 6.0);
        const double b00 = a0 / p, b11 = a1 / p, b22 = a2 / p;
        const double b01 = s[0][1] / p, b02 = s[0][2] / p, b12 = s[1][2] / p;
        double r = 0.5 * (b00 * (b11 * b22 - b12 * b12) - b01 * (b01 * b22 - b12 * b02) +
                          b02 * (b01 * b12 - b11 * b02));
        r = fmin(1.0, fmax(-1.0, r));
        return (q + 2.0 * p * cos(acos(r) / 3.0)) * (1.0 + 1e-9) + 1e-12 * fabs(q);
    }
}

__device__ __forceinline__ void split_f32(double v, float &hi, float &lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
}


// Records of seed i (i < n) for the scoring and rescoring kernels, plus the
// statistics the rounding bounds need; padding records (n <= i) get zeros.
// `wkey` = w_i for the max-weight reference (-DBL_MAX if not finite), `frob` =
// ||sym A_i||_F, `lam` = a lower bound of lambda_min(sym A_i); `bad` collects
// ST_NONFINITE / ST_NOT_SPD.
template <int D>
__device__ __forceinline__ void build_seed(const int i, const int n, const double *__restrict__ x,
                                           const double *__restrict__ A, const double *__restrict__ w,
                                           SeedRec &r, SeedRec32 &r32, double &wkey, double &frob,
                                           double &lam, int &bad) {
#pragma unroll
    for (int a = 0; a < 3; ++a) r.x[a] = 0.0;
    r.w = 0.0;
#pragma unroll
    for (int a = 0; a < 6; ++a) r.a[a] = 0.f;
    r.pad[0] = r.pad[1] = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) r32.xh[a] = r32.xl[a] = 0.f;
    r32.wh = r32.wl = 0.f;
#pragma unroll
    for (int a = 0; a < 6; ++a) r32.a[a] = 0.f;
    r32.pad[0] = r32.pad[1] = 0.f;
    wkey = -DBL_MAX;
    frob = 0.0;
    lam = DBL_MAX;
    bad = 0;
    if (i >= n) return;
    double xx[D], M[D][D];
    bool finite = true;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        xx[a] = x[(size_t)i * D + a];
        finite = finite && isfinite(xx[a]);
    }
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) {
            M[a][b] = A[(size_t)i * D * D + a * D + b];
            finite = finite && isfinite(M[a][b]);
        }
    const double wi = w[i];
    finite = finite && isfinite(wi);
    double s[D][D];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) s[a][b] = 0.5 * (M[a][b] + M[b][a]);
    double det, m2 = s[0][0] * s[1][1] - s[0][1] * s[0][1];
    if (D == 2) {
        det = m2;
    } else {
        det = s[0][0] * (s[1][1] * s[2][2] - s[1][2] * s[1][2]) -
              s[0][1] * (s[0][1] * s[2][2] - s[1][2] * s[0][2]) +
              s[0][2] * (s[0][1] * s[1][2] - s[1][1] * s[0][2]);
    }
    const bool spd = (s[0][0] > 0.0) && (m2 > 0.0) && (det > 0.0);
    double f2 = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) f2 += s[a][b] * s[a][b];
    frob = sqrt(f2);
    lam = spd ? lambda_min_sym<D>(s) : 0.0;
    const double lmax = spd ? fmin(lambda_max_sym<D>(s), sqrt(f2) * (1.0 + 1e-12)) : 0.0;
    if (!finite) bad = ST_NONFINITE;
    else if (!spd) bad = ST_NOT_SPD;
    if (!finite) {
        frob = 0.0;
        lam = 0.0;
    }
#pragma unroll
    for (int a = 0; a < D; ++a) r.x[a] = xx[a];
    r.w = wi;
    if (D == 2) {
        r.a[0] = (float)s[0][0];
        r.a[1] = (float)s[0][1];
        r.a[2] = (float)s[1][1];
    } else {
        r.a[0] = (float)s[0][0];
        r.a[1] = (float)s[0][1];
        r.a[2] = (float)s[0][2];
        r.a[3] = (float)s[1][1];
        r.a[4] = (float)s[1][2];
        r.a[5] = (float)s[2][2];
    }
    wkey = finite ? wi : -DBL_MAX;
    r.pad[0] = __double2float_rd(lam);  // lower bound of lambda_min for the group bounds
#pragma unroll
    for (int a = 0; a < D; ++a) split_f32(xx[a], r32.xh[a], r32.xl[a]);
    split_f32(wi, r32.wh, r32.wl);
#pragma unroll
    for (int a = 0; a < 6; ++a) r32.a[a] = r.a[a];
    r32.pad[0] = r.pad[0];
    r32.pad[1] = __double2float_ru(lmax);  // upper bound of lambda_max (candidate lists only)
}

// Bounds of group `grp` (32 consecutive records, positions >= n are padding),
// computed by one warp and written by lane 0.
template <int D>
__device__ __forceinline__ void group_bound_warp(const SeedRec *__restrict__ recs, const int n, const int grp,
                                                 GroupBound *__restrict__ out, const double wref) {
    const int lane = threadIdx.x & 31;
    const int pos = grp * 32 + lane;
    const bool real = pos < n;
    float lo[3], hi[3];
    float lam = real ? recs[pos].pad[0] : FLT_MAX;
    double wm = real ? recs[pos].w : -DBL_MAX;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double xa = (real && a < D) ? recs[pos].x[a] : 0.0;
        lo[a] = real ? __double2float_rd(xa) : FLT_MAX;
        hi[a] = real ? __double2float_ru(xa) : -FLT_MAX;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], off));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], off));
        }
        lam = fminf(lam, __shfl_xor_sync(0xffffffffu, lam, off));
        wm = fmax(wm, __shfl_xor_sync(0xffffffffu, wm, off));
    }
    if (lane == 0) {
        GroupBound gb;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            gb.lo[a] = lo[a];
            gb.hi[a] = hi[a];
        }
        gb.lam = lam;
        gb.wgap = __double2float_rd(wref - wm);
        gb.wmax = wm;
        out[grp] = gb;
    }
}

// Morton code of a seed position on the grid box (padding sorts last).
template <int D>
__device__ __forceinline__ uint32_t seed_code(const GridDev &g, const SeedRec &r, bool real) {
    if (!real) return 0xffffffffu;
    double frac[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int a = 0; a < D; ++a) frac[a] = (r.x[a] - g.lo[a]) / ((double)g.res[a] * g.h[a]);
    return morton_code(D, frac);
}

// In-place ascending bitonic sort of m (a power of two) 64-bit keys in shared
// memory by the whole block; keys are distinct, so the order is deterministic.
__device__ __forceinline__ void block_bitonic_sort(unsigned long long *keys, const int m) {
    for (int k = 2; k <= m; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < m; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) {
                    const unsigned long long a = keys[i], b = keys[l];
                    const bool up = (i & k) == 0;
                    if ((a > b) == up) {
                        keys[i] = b;
                        keys[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// Per-cell terms of eqs. (2.7)-(2.8) from the integer moments of cell i:
//   m = M0, mean odd coordinate mu = S1 / m, centred second moment
//   C = S2 - S1 S1^T / m (in units of (h/2)^2), centroid offset e = lo + (h/2) mu - x_i,
//   Q = sum_ab A_ab ((h_a h_b / 4) C_ab + m e_a e_b) = sum_{H_j=i} |y_j - x_i|^2_{A_i},
//   gr = v_i - m |P| (two roundings, no contraction, as eq. (2.8) is written).
template <int D>
__device__ __forceinline__ void dual_terms(const GridDev &g, const unsigned long long *__restrict__ mo,
                                           const double vi, const double *__restrict__ xi,
                                           const double *__restrict__ Ai, double &gr, double &Q) {
    const double m = (double)mo[0];
    gr = __dsub_rn(vi, __dmul_rn(m, g.cell));
    Q = 0.0;
    if (mo[0] == 0ull) return;
    // one division (the FP64 divide is a long dependent sequence on this part);
    // the products with 1/m differ from the quotients by a few ulp
    const double inv_m = 1.0 / m;
    double S1[D], e[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        S1[a] = (double)mo[1 + a];
        e[a] = (g.lo[a] + 0.5 * g.h[a] * (S1[a] * inv_m)) - xi[a];
    }
    int t = 1 + D;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = a; b < D; ++b) {
            const double Cab = (double)mo[t++] - S1[a] * S1[b] * inv_m;
            const double Mab = 0.25 * g.h[a] * g.h[b] * Cab + m * e[a] * e[b];
            const double Aab = (a == b) ? Ai[a * D + a] : Ai[a * D + b] + Ai[b * D + a];
            Q += Aab * Mab;
        }
}

// Per-cell dual terms from FP64 element-measure moments (non-uniform
// discretisation): m = sum |P_j|, S1 = sum |P_j| y_j, S2 = sum |P_j| y_j y_j^T
// (upper triangle); Q = sum_j |P_j| (y_j - x)^T A (y_j - x) expanded in them.
template <int D>
__device__ __forceinline__ void dual_terms_points(const double *__restrict__ mo, const double vi,
                                                  const double *__restrict__ xi, const double *__restrict__ Ai,
                                                  double &gr, double &Q) {
    const double m = mo[0];
    gr = vi - m;
    Q = 0.0;
    int t = 1 + D;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = a; b < D; ++b) {
            const double Cab = mo[t++] - mo[1 + a] * xi[b] - xi[a] * mo[1 + b] + m * xi[a] * xi[b];
            const double Aab = (a == b) ? Ai[a * D + a] : Ai[a * D + b] + Ai[b * D + a];
            Q += Aab * Cab;
        }
}

}  // namespace apd
