// Seed preparation, the dual value/gradient of eqs. (2.7)-(2.8) from integer
// moments, the discrete centroids of Algorithm 3, and the vector kernels of
// the L-BFGS weight solve (Algorithm 2).
#include <float.h>
#include <string.h>

#include "apd_common.cuh"

namespace apd {

namespace {

constexpr int kRedThreads = 1024;

__global__ void eval_reset_kernel(DevScalars *sc, const int keep_geometry) {
    sc->flag_count = 0u;
    sc->wref_key = 0ull;
    sc->dual_done = 0u;
    sc->inc_go = 0;     // a full pass: it records (incremental solves) ...
    sc->inc_valid = 0;  // ... and no earlier record holds for its records
    if (!keep_geometry) {
        sc->lam_abs_bits = 0ull;
        sc->lam_min_bits = 0x7ff0000000000000ull;
    }
}

// Start of an evaluation whose records' positions and matrices are unchanged
// (same x, A, n as the last seed preparation): zeroed moments and queue count,
// the trial weights (w = W0 + t p into Wt when p is given, else w = W0), their
// copies in the scored records (scan order) and both rescoring record arrays,
// the reference weight wref = max w (per-block maxima reduced by the last block
// to finish), and each 32-seed group's largest weight and gap wref - wmax.  One
// thread per scan position; a warp covers one group.
// With coef (the first trial of a new L-BFGS direction), the direction itself
// is formed first, p = -gamma gf + sum_k (cy_k y_k + cs_k s_k) from the
// coefficients the direction kernels left (written to pdir), with <gf, p>
// reduced by the last block into sc->gp0: one launch instead of two.
__global__ void __launch_bounds__(256)
    eval_begin_kernel(const int n, const int n_pad, const long long n_mom, const double *__restrict__ W0,
                      const double t, double *__restrict__ pdir, double *__restrict__ Wt,
                      const int32_t *__restrict__ perm, SeedRec *__restrict__ recs,
                      SeedRec32 *__restrict__ recs32, SeedRec32 *__restrict__ recs32s,
                      GroupBound *__restrict__ groups, unsigned long long *__restrict__ mom,
                      double *__restrict__ part, DevScalars *__restrict__ sc, const LbfgsCoef *__restrict__ coef,
                      const double *__restrict__ S, const double *__restrict__ Y, const double *__restrict__ gfv,
                      const double *__restrict__ w0, const unsigned long long *__restrict__ wref0,
                      const unsigned *__restrict__ g3_hist, const unsigned full_max,
                      float2 *__restrict__ drift) {
    __shared__ double shw[8], shg[8], shdx[8], shdn[8];
    __shared__ double ccy[32], ccs[32];
    __shared__ int cslot[32];
    __shared__ bool last;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    int hist = 0;
    double gam = 0.0;
    if (coef) {
        hist = min(coef->hist, 31);
        gam = coef->gamma;
        for (int k = threadIdx.x; k < hist; k += blockDim.x) {
            ccy[k] = coef->cy[k];
            ccs[k] = coef->cs[k];
            cslot[k] = coef->slot[k];
        }
        __syncthreads();
    }
    double gp = 0.0;
    double dhi = -DBL_MAX, dlo = DBL_MAX;  // range of w - w0 (with w0)
    for (long long e = i; e < n_mom; e += (long long)gridDim.x * blockDim.x) mom[e] = 0ull;
    if (i == 0) {
        sc->flag_count = 0u;
        sc->band_count = 0u;
    }
    const int src = i < n_pad ? (perm ? perm[i] : i) : n;
    const bool real = src < n;
    double wkey = -DBL_MAX;
    if (real) {
        double wi;
        if (pdir) {
            double pv;
            if (coef) {
                const double g = gfv[src];
                pv = -gam * g;
#pragma unroll 4
                for (int k = 0; k < hist; ++k) {
                    const size_t o = (size_t)cslot[k] * n + src;
                    pv += ccy[k] * Y[o] + ccs[k] * S[o];
                }
                pdir[src] = pv;
                gp = g * pv;
            } else {
                pv = pdir[src];
            }
            wi = fma(t, pv, W0[src]);
            Wt[src] = wi;
        } else {
            wi = W0[src];
        }
        const bool finite = isfinite(wi);
        if (!finite) atomicOr(&sc->status, ST_NONFINITE);
        recs[i].w = wi;
        float wh, wl;
        split_f32(wi, wh, wl);
        recs32[src].wh = wh;
        recs32[src].wl = wl;
        if (recs32s) {
            recs32s[i].wh = wh;
            recs32s[i].wl = wl;
        }
        wkey = finite ? wi : -DBL_MAX;
        if (w0) {  // rounded outwards, so that the range covers the exact drift
            dhi = __dsub_ru(wi, w0[src]);
            dlo = __dsub_rd(wi, w0[src]);
            if (drift) drift[src] = make_float2(__double2float_rd(dlo), __double2float_ru(dhi));
        }
    }
    const double wmax = warp_max(wkey);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (coef) {
        gp = warp_sum(gp);
        if (lane == 0) shg[wid] = gp;
    }
    if (w0) {
        dhi = warp_max(dhi);
        dlo = warp_min(dlo);
        if (lane == 0) {
            shdx[wid] = dhi;
            shdn[wid] = dlo;
        }
    }
    if (lane == 0) {
        shw[wid] = wmax;
        if (groups && i < n_pad && (i & ~31) < n) groups[i >> 5].wmax = wmax;
    }
    __threadfence();  // group writes before the block's arrival count
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = shw[0];
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) b = fmax(b, shw[k]);
        part[(size_t)blockIdx.x * kPartStride] = b;
        if (coef) {
            double s = 0.0;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += shg[k];
            part[(size_t)blockIdx.x * kPartStride + 1] = s;
        }
        if (w0) {
            double x = -DBL_MAX, m = DBL_MAX;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
                x = fmax(x, shdx[k]);
                m = fmin(m, shdn[k]);
            }
            part[(size_t)blockIdx.x * kPartStride + 2] = x;
            part[(size_t)blockIdx.x * kPartStride + 3] = m;
        }
        __threadfence();
        last = atomicAdd(&sc->dual_done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // block maxima loaded in parallel (max is order-independent)
    double wref = -DBL_MAX;
    for (unsigned k = threadIdx.x; k < gridDim.x; k += blockDim.x)
        wref = fmax(wref, *(volatile double *)&part[(size_t)k * kPartStride]);
    wref = warp_max(wref);
    if ((threadIdx.x & 31) == 0) shw[threadIdx.x >> 5] = wref;
    __syncthreads();
    wref = shw[0];
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) wref = fmax(wref, shw[k]);
    if (groups)
        for (int gidx = threadIdx.x; gidx * 32 < n; gidx += blockDim.x) {
            const double wm = *(volatile double *)&groups[gidx].wmax;
            groups[gidx].wgap = __double2float_rd(wref - wm);
        }
    if (w0 && threadIdx.x < 32) {  // the drift range (max and min are order-independent)
        double x = -DBL_MAX, m = DBL_MAX;
        for (unsigned k = threadIdx.x; k < gridDim.x; k += 32) {
            x = fmax(x, *(volatile double *)&part[(size_t)k * kPartStride + 2]);
            m = fmin(m, *(volatile double *)&part[(size_t)k * kPartStride + 3]);
        }
        x = warp_max(x);
        m = warp_min(m);
        // the pixels a re-decision would settle in full have g3 <= D: bound their
        // count by the record's histogram (every bin up to D's); bin 0 (no
        // certified margin: FP64 near ties) costs a recording as much
        const float bD = __double2float_ru(__dsub_ru(x, m));
        const unsigned eD = bD > 0.f ? min(__float_as_uint(bD) >> 21, (unsigned)kIncBins - 1u) : 0u;
        unsigned cnt = 0u;
        if (g3_hist)
            for (unsigned e = threadIdx.x; e < (unsigned)kIncBins; e += 32u)
                cnt += (e > 0u && e <= eD) ? g3_hist[e] : 0u;
        cnt = __reduce_add_sync(0xffffffffu, cnt);
        if (threadIdx.x == 0) {
            sc->drift_max = x;
            sc->drift_min = m;
            sc->drift_hi = __double2float_ru(x);
            sc->inc_go = (sc->inc_valid && g3_hist && cnt <= full_max) ? 1 : 0;
            // the incremental pass's band width and excluded-seed shift, rounded outwards
            sc->band_D = bD;
            // (less 2^-40 (|w_ref| + |w_ref0|): the scorers take w_ref as a float pair)
            const double wr0 = wref0 ? dkey_inv(*wref0) : wref;
            const double slack = ldexp(fabs(wref) + fabs(wr0), -40);
            sc->band_shift = __double2float_rd(__dsub_rd(__dsub_rd(__dsub_rd(wref, wr0), x), slack));
        }
    }
    if (coef && threadIdx.x < 32) {  // <gf, p>: the blocks' sums, lane-strided, then a fixed tree
        double s = 0.0;
        for (unsigned k = threadIdx.x; k < gridDim.x; k += 32) s += *(volatile double *)&part[(size_t)k * kPartStride + 1];
        s = warp_sum(s);
        if (threadIdx.x == 0) sc->gp0 = s;
    }
    if (threadIdx.x == 0) {
        sc->wref_key = dkey(wref);
        sc->dual_done = 0u;
    }
}

template <int D>
__global__ void seed_prep_kernel(const GridDev g, const int n, const int n_pad,
                                 const double *__restrict__ x, const double *__restrict__ A,
                                 const double *__restrict__ w, SeedRec *__restrict__ recs,
                                 SeedRec32 *__restrict__ recs32, uint32_t *__restrict__ codes,
                                 DevScalars *__restrict__ sc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    SeedRec r;
    SeedRec32 r32;
    double wkey, frob, lam;
    int bad;
    build_seed<D>(i, n, x, A, w, r, r32, wkey, frob, lam, bad);
    const bool active = i < n;
    if (bad) atomicOr(&sc->status, bad);
    if (i < n_pad) {
        recs[i] = r;
        recs32[i] = r32;
        if (codes) codes[i] = seed_code<D>(g, r, active);
    }
    // one atomic per warp for each statistic
    const double wmax = warp_max(active ? wkey : -DBL_MAX);
    const double fmx = warp_max(active ? frob : 0.0);
    const double lmn = warp_min(active ? lam : DBL_MAX);
    const bool any = __any_sync(0xffffffffu, active);
    if ((threadIdx.x & 31) == 0 && any) {
        atomicMax(&sc->wref_key, dkey(wmax));
        atomicMax(&sc->lam_abs_bits, (unsigned long long)__double_as_longlong(fmx));
        atomicMin(&sc->lam_min_bits, (unsigned long long)__double_as_longlong(lmn));
    }
}

// Bitonic sort of (Morton code, seed index) pairs in shared memory, one block;
// the pair order is total, so the result is deterministic.  m = power of two.
__global__ void __launch_bounds__(1024)
    morton_sort_kernel(const int n_pad, const int m, const uint32_t *__restrict__ codes,
                       uint32_t *__restrict__ scodes, int32_t *__restrict__ perm) {
    extern __shared__ unsigned long long keys[];  // (code << 32) | index
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const uint32_t c = i < n_pad ? codes[i] : 0xffffffffu;
        keys[i] = ((unsigned long long)c << 32) | (unsigned)i;
    }
    __syncthreads();
    block_bitonic_sort(keys, m);
    for (int i = threadIdx.x; i < n_pad; i += blockDim.x) {
        scodes[i] = (uint32_t)(keys[i] >> 32);
        perm[i] = (int32_t)(keys[i] & 0xffffffffu);
    }
}

template <int D>
__global__ void group_bounds_kernel(const int n, const SeedRec *__restrict__ recs, GroupBound *__restrict__ groups,
                                    const DevScalars *__restrict__ sc) {
    const int grp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (grp * 32 < n) group_bound_warp<D>(recs, n, grp, groups, dkey_inv(sc->wref_key));
}

__global__ void gather_recs_kernel(const int n_pad, const int32_t *__restrict__ perm,
                                   const SeedRec *__restrict__ src, SeedRec *__restrict__ dst,
                                   const SeedRec32 *__restrict__ src32, SeedRec32 *__restrict__ dst32) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_pad) {
        dst[i] = src[perm[i]];
        if (dst32) dst32[i] = src32[perm[i]];
    }
}

// Pair p (of D (D + 1) / 2, a <= b in row order) of the upper triangle.
template <int D>
__device__ __forceinline__ void pair_ab(const int p, int &a, int &b) {
    if (D == 3) {
        a = p < 3 ? 0 : (p < 5 ? 1 : 2);
        b = p < 3 ? p : (p < 5 ? p - 2 : 2);
    } else {
        a = p < 2 ? 0 : 1;
        b = p < 2 ? p : 1;
    }
}
__device__ __forceinline__ double sel3(const double (&v)[3], const int a) {
    return a == 0 ? v[0] : (a == 1 ? v[1] : v[2]);
}

// The pair terms of Q_i = sum_j (y_j - x_i)^T A_i (y_j - x_i) over cell i's
// pixels (|P| Q_i is the integral term of eq. (2.7)) that lane q of the cell's
// four lanes takes: pairs q and q + 4.  Q_ab = A_ab M_ab (A_ab + A_ba off the
// diagonal) with M_ab = sum_j (y - x)_a (y - x)_b written through the integer
// moments m, S1 = sum u, S2 = sum u u^T (u = 2k + 1, y = lo + h u / 2):
// M_ab = h_a h_b / 4 (S2_ab - S1_a S1_b / m) + m e_a e_b, e = centroid - x.
template <int D>
__device__ __forceinline__ double dual_pair_terms(const GridDev &g, const unsigned long long *__restrict__ mo,
                                                  const double *__restrict__ xi, const double *__restrict__ Ai,
                                                  const int q) {
    constexpr int NP = D * (D + 1) / 2;
    // no early exit on an empty cell: every load is issued before the first result
    // is needed (one memory round trip), and an empty cell's terms are dropped at the end
    const unsigned long long m0 = mo[0];
    const double m = (double)m0;
    const double inv_m = 1.0 / m;  // one division; products with it differ from quotients by a few ulp
    double Q = 0.0;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int p = q + 4 * r;
        if (p < NP) {
            int a, b;
            pair_ab<D>(p, a, b);
            const double S1a = (double)mo[1 + a], S1b = (double)mo[1 + b];
            const double ea = (sel3(g.lo, a) + 0.5 * sel3(g.h, a) * (S1a * inv_m)) - xi[a];
            const double eb = (sel3(g.lo, b) + 0.5 * sel3(g.h, b) * (S1b * inv_m)) - xi[b];
            const double Cab = (double)mo[1 + D + p] - S1a * S1b * inv_m;
            const double Mab = 0.25 * sel3(g.h, a) * sel3(g.h, b) * Cab + m * ea * eb;
            const double Aab = a == b ? Ai[a * D + a] : Ai[a * D + b] + Ai[b * D + a];
            Q += Aab * Mab;
        }
    }
    return m0 == 0ull ? 0.0 : Q;
}

// The same from FP64 element-measure moments (non-uniform discretisation):
// m = sum |P_j|, S1 = sum |P_j| y_j, S2 = sum |P_j| y_j y_j^T, and
// Q_ab = A_ab (S2_ab - S1_a x_b - x_a S1_b + m x_a x_b).
template <int D>
__device__ __forceinline__ double points_pair_terms(const double *__restrict__ mo, const double *__restrict__ xi,
                                                    const double *__restrict__ Ai, const int q) {
    constexpr int NP = D * (D + 1) / 2;
    const double m = mo[0];
    double Q = 0.0;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int p = q + 4 * r;
        if (p < NP) {
            int a, b;
            pair_ab<D>(p, a, b);
            const double Cab = mo[1 + D + p] - mo[1 + a] * xi[b] - xi[a] * mo[1 + b] + m * xi[a] * xi[b];
            const double Aab = a == b ? Ai[a * D + a] : Ai[a * D + b] + Ai[b * D + a];
            Q += Aab * Cab;
        }
    }
    return Q;
}

// Per-cell dual terms, four lanes per cell (FP64 issues slowly; the pair terms
// are split over the lanes), then a deterministic reduction: block sums through
// fixed shuffle trees, block partials reduced by the last block to finish.
//   g_i = (v_i - m_i |P|) w_i + |P| Q_i,  grad_i = v_i - m_i |P|  (eqs. (2.7), (2.8))
// kPoints: FP64 element-measure moments of a non-uniform discretisation
// (mom_pts), g_i = (v_i - m_i) w_i + Q_i, grad_i = v_i - m_i.
// The largest relative volume error max_i |grad_i| / v_i is tracked as the
// pair (|grad_k|, v_k) of its cell and divided once at the end.
constexpr int kDualThreads = 256;  // 64 cells per block round
template <int D, bool kPoints = false>
__global__ void __launch_bounds__(kDualThreads)
    dual_kernel(const GridDev g, const int n, const double *__restrict__ x,
                const double *__restrict__ A, const double *__restrict__ w,
                const double *__restrict__ v, const double *__restrict__ p_dir,
                const unsigned long long *__restrict__ mom, double *__restrict__ part,
                DevScalars *__restrict__ sc, double *g_out, double *grad_out, double *gf_out,
                double *err_out, const double *__restrict__ mom_pts = nullptr) {
    constexpr int K = moment_width(D);
    constexpr int NQ = kPartStride;  // g, <grad f, p>, sum v, max error (numerator, denominator), min v
    __shared__ double shq[kDualThreads / 32][NQ];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, q = lane & 3;
    double gsum = 0.0, gp = 0.0, sv = 0.0, en = 0.0, ed = 1.0, vmin = DBL_MAX;
    const int stride = gridDim.x * (kDualThreads / 4);
    const int rounds = (n + stride - 1) / stride;  // the same for every lane (converged shuffles)
    int i = (blockIdx.x * kDualThreads + threadIdx.x) >> 2;
    for (int r = 0; r < rounds; ++r, i += stride) {
        const bool real = i < n;
        double Qp = 0.0, vi = 1.0, wi = 0.0, pd = 0.0;
        if (real) {  // the cell's scalars too, before the pair terms' arithmetic
            vi = v[i];
            wi = w[i];
            if (p_dir) pd = p_dir[i];
        }
        if (real)
            Qp = kPoints ? points_pair_terms<D>(mom_pts + (size_t)i * K, x + (size_t)i * D, A + (size_t)i * D * D, q)
                         : dual_pair_terms<D>(g, mom + (size_t)i * K, x + (size_t)i * D, A + (size_t)i * D * D, q);
        Qp += __shfl_xor_sync(0xffffffffu, Qp, 1);
        Qp += __shfl_xor_sync(0xffffffffu, Qp, 2);
        if (real && q == 0) {
            if (!(vi > 0.0) || !isfinite(vi)) atomicOr(&sc->status, ST_BAD_VOLUME);
            const double gr = kPoints ? vi - mom_pts[(size_t)i * K] : __dsub_rn(vi, __dmul_rn((double)mom[(size_t)i * K], g.cell));
            gsum += kPoints ? gr * wi + Qp : gr * wi + g.cell * Qp;
            const double ag = fabs(gr);
            if (ag * ed > en * vi) {
                en = ag;
                ed = vi;
            }
            if (grad_out) grad_out[i] = gr;
            if (gf_out) gf_out[i] = -gr;
            if (p_dir) gp += -gr * pd;
            sv += vi;
            vmin = fmin(vmin, vi);
        }
    }
    // warp: the cells' lanes q = 0 (lanes 0, 4, ..., 28) by a fixed tree
#pragma unroll
    for (int off = 4; off < 32; off <<= 1) {
        gsum += __shfl_xor_sync(0xffffffffu, gsum, off);
        gp += __shfl_xor_sync(0xffffffffu, gp, off);
        sv += __shfl_xor_sync(0xffffffffu, sv, off);
        const double on = __shfl_xor_sync(0xffffffffu, en, off), od = __shfl_xor_sync(0xffffffffu, ed, off);
        if (on * ed > en * od) {
            en = on;
            ed = od;
        }
        vmin = fmin(vmin, __shfl_xor_sync(0xffffffffu, vmin, off));
    }
    if (lane == 0) {
        shq[wid][0] = gsum;
        shq[wid][1] = gp;
        shq[wid][2] = sv;
        shq[wid][3] = en;
        shq[wid][4] = ed;
        shq[wid][5] = vmin;
    }
    __syncthreads();
    // block: warp 0 over the 8 warps' values by a fixed tree; lane 0 stores the partials
    if (wid == 0) {
        const int k = lane < kDualThreads / 32 ? lane : 0;
        const bool own = lane < kDualThreads / 32;
        double b0 = own ? shq[k][0] : 0.0, b1 = own ? shq[k][1] : 0.0, b2 = own ? shq[k][2] : 0.0;
        double b3 = own ? shq[k][3] : 0.0, b4 = own ? shq[k][4] : 1.0, b5 = own ? shq[k][5] : DBL_MAX;
#pragma unroll
        for (int off = 1; off < kDualThreads / 32; off <<= 1) {
            b0 += __shfl_xor_sync(0xffffffffu, b0, off);
            b1 += __shfl_xor_sync(0xffffffffu, b1, off);
            b2 += __shfl_xor_sync(0xffffffffu, b2, off);
            const double on = __shfl_xor_sync(0xffffffffu, b3, off), od = __shfl_xor_sync(0xffffffffu, b4, off);
            if (on * b4 > b3 * od) {
                b3 = on;
                b4 = od;
            }
            b5 = fmin(b5, __shfl_xor_sync(0xffffffffu, b5, off));
        }
        if (lane == 0) {
            double *pp = part + (size_t)blockIdx.x * NQ;
            pp[0] = b0;
            pp[1] = b1;
            pp[2] = b2;
            pp[3] = b3;
            pp[4] = b4;
            pp[5] = b5;
            __threadfence();
            last = atomicAdd(&sc->dual_done, 1u) == gridDim.x - 1;
        }
    }
    __syncthreads();
    if (!last || wid != 0) return;
    __threadfence();
    // the last block: lanes take the blocks in order (lane, lane + 32, ...), then a fixed tree
    double G = 0.0, GP = 0.0, SV = 0.0, EN = 0.0, ED = 1.0, VM = DBL_MAX;
    for (unsigned b = lane; b < gridDim.x; b += 32) {
        const volatile double *pp = part + (size_t)b * NQ;
        G += pp[0];
        GP += pp[1];
        SV += pp[2];
        const double on = pp[3], od = pp[4];
        if (on * ED > EN * od) {
            EN = on;
            ED = od;
        }
        VM = fmin(VM, pp[5]);
    }
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        G += __shfl_xor_sync(0xffffffffu, G, off);
        GP += __shfl_xor_sync(0xffffffffu, GP, off);
        SV += __shfl_xor_sync(0xffffffffu, SV, off);
        const double on = __shfl_xor_sync(0xffffffffu, EN, off), od = __shfl_xor_sync(0xffffffffu, ED, off);
        if (on * ED > EN * od) {
            EN = on;
            ED = od;
        }
        VM = fmin(VM, __shfl_xor_sync(0xffffffffu, VM, off));
    }
    if (lane == 0) {
        const double E = __ddiv_rn(EN, ED);
        sc->g = G;
        sc->max_rel_err = E;
        sc->dot_gp = GP;
        sc->sum_v = SV;
        sc->min_v = VM;
        sc->dual_done = 0u;
        if (g_out) *g_out = G;
        if (err_out) *err_out = E;
    }
}

template <int D>
__global__ void centroid_kernel(const GridDev g, const int n, const double *__restrict__ x,
                                const unsigned long long *__restrict__ mom, double *x_out) {
    constexpr int K = moment_width(D);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long *mo = mom + (size_t)i * K;
    const double m = (double)mo[0];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const double xa = x[(size_t)i * D + a];
        x_out[(size_t)i * D + a] = mo[0] > 0ull ? g.lo[a] + 0.5 * g.h[a] * ((double)mo[1 + a] / m) : xa;
    }
}

__global__ void axpy_kernel(const int n, const double *a, const double t, const double *b, double *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a[i] + t * b[i];
}

// The L-BFGS pairs (s_k, y_k) live in slots of a ring of `cap`; beside them the
// Gram entries gram[0][i][j] = s_i . y_j and gram[1][i][j] = y_i . y_j (slot
// indices), filled by the push kernel for every pair of slots that can be in
// the history together.  With them the two-loop recursion of the L-BFGS
// direction (Nocedal and Wright, Algorithm 7.4) needs only the 2 hist dot
// products s_k . g, y_k . g over the seeds; its scalar recursion then runs on
// the Gram entries and p is assembled in one pass as
//   p = -gamma g + sum_k gamma alpha_k y_k - sum_k (alpha_k - beta_k) s_k,
// the same vector as the two-loop form in exact arithmetic.
//
// FP64 runs at a few operations per clock per SM and every dependent global
// load costs about a microsecond of latency, so the dot products are spread
// over up to one block per SM (32 seeds per block range, a warp per dot, all
// of a block's loads in flight together) and the last block to finish reduces
// the per-block sums in block order (deterministic) and runs the scalar part
// in one warp, column by column (one shuffle per step).  The push kernel also
// forms the next direction's dot products (for both outcomes of its curvature
// test), so an accepted step costs two launches: push-and-coefficients, then p.
constexpr int kLbfgsMax = 32;    // ring capacity the kernels below support
static_assert(kLbfgsDots >= 5 + 5 * (kLbfgsMax - 1), "partial-sum rows hold the push's products");
constexpr int kLbT = 1024;       // threads per block of the dot-product kernels
constexpr int kLbR = 32;         // seeds per block range
constexpr int kLbP = 64;         // threads per block of the p kernel

// Partial dot products of one block over its ranges of 32 seeds (range r
// starts at (blockIdx.x + r gridDim.x) 32): dot d (of nd) is sum_i f(d, i),
// warp w takes the dots d = w mod 32.  part[blockIdx.x * kLbfgsDots + d]
// receives the block's sums.
template <class F>
__device__ void block_partial_dots(const int nd, const int n, F f, double *part) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int d = wid; d < nd; d += kLbT / 32) {
        double v = 0.0;
        for (int r0 = blockIdx.x * kLbR; r0 < n; r0 += gridDim.x * kLbR)
            if (r0 + lane < n) v += f(d, r0 + lane);
        v = warp_sum(v);
        if (lane == 0) part[(size_t)blockIdx.x * kLbfgsDots + d] = v;
    }
}

// Called by every block after its partial sums are stored: true in the last
// block to arrive (which then sees every block's sums).
__device__ bool lbfgs_last_block(DevScalars *sc) {
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&sc->lbfgs_done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// out[d] = sum over blocks (lane-strided, then the warp tree) of part[.][d], d < nd.
__device__ void reduce_partials(const int nd, const double *part, double *out) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int d = wid; d < nd; d += (int)(blockDim.x >> 5)) {
        double v = 0.0;
        for (unsigned b = lane; b < gridDim.x; b += 32) v += *(const volatile double *)(part + (size_t)b * kLbfgsDots + d);
        v = warp_sum(v);
        if (lane == 0) out[d] = v;
    }
    __syncthreads();
}

// Shared state of the scalar part: the history's Gram entries (padded rows:
// the column-wise steps read one column across the lanes), 1 / s.y, s_k . g,
// y_k . g and the slots, k = 0 the newest pair.
struct LbfgsScalars {
    double sy[kLbfgsMax][kLbfgsMax + 1];  // s_k . y_j
    double yy[kLbfgsMax][kLbfgsMax + 1];  // y_k . y_j
    double rh[kLbfgsMax], sg[kLbfgsMax], yg[kLbfgsMax], al[kLbfgsMax];
    int slot[kLbfgsMax];
};

// The last block's gather of the history's Gram entries and 1 / s.y.
__device__ void load_gram(LbfgsScalars &L, const int hist, const int cap, const double *__restrict__ gram,
                          const double *__restrict__ rho) {
    for (int e = threadIdx.x; e < hist * hist; e += blockDim.x) {
        const int k = e / hist, j = e % hist;
        L.sy[k][j] = gram[(size_t)L.slot[k] * cap + L.slot[j]];
        L.yy[k][j] = gram[(size_t)cap * cap + (size_t)L.slot[k] * cap + L.slot[j]];
    }
    for (int k = threadIdx.x; k < hist; k += blockDim.x) L.rh[k] = rho[L.slot[k]];
    __syncthreads();
}

// The two-loop recursion on the Gram entries, by warp 0, column by column:
// alpha_k = rho_k (s_k . g - sum_{j<k} alpha_j s_k . y_j)          (newest first)
// c_k = alpha_k - rho_k (gamma y_k . q + sum_{j>k} c_j s_j . y_k)   (oldest first)
// with y_k . q = y_k . g - sum_j alpha_j y_k . y_j; then the coefficients of p.
__device__ void lbfgs_coefficients(LbfgsScalars &L, const int hist, const double gamma, LbfgsCoef *coef) {
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    double t = 0.0, al = 0.0;
    for (int k = 0; k < hist; ++k) {
        double a = lane == k ? L.rh[k] * (L.sg[k] - t) : 0.0;
        a = __shfl_sync(0xffffffffu, a, k);
        if (lane == k) al = a;
        if (lane > k && lane < hist) t += a * L.sy[lane][k];
    }
    if (lane < hist) L.al[lane] = al;
    __syncwarp();
    double yq = 0.0;
    if (lane < hist) {
        yq = L.yg[lane];
        for (int j = 0; j < hist; ++j) yq -= L.al[j] * L.yy[lane][j];
    }
    double u = 0.0, c = 0.0;
    for (int k = hist - 1; k >= 0; --k) {
        double ck = lane == k ? al - L.rh[k] * (gamma * yq + u) : 0.0;
        ck = __shfl_sync(0xffffffffu, ck, k);
        if (lane == k) c = ck;
        if (lane < k) u += ck * L.sy[k][lane];
    }
    // p = -gamma g + sum_k gamma alpha_k y_k - sum_k (alpha_k - beta_k) s_k
    if (lane < hist) {
        coef->cs[lane] = -c;
        coef->cy[lane] = gamma * al;
        coef->slot[lane] = L.slot[lane];
    }
    if (lane == 0) {
        coef->hist = hist;
        coef->gamma = gamma;
    }
}

// Coefficients of p = -H gf (H0 = gamma I, the stored pairs newest at slot
// `newest`).  With use_pair, the pair just pushed (slot newest_acc) is used if
// it passed the push kernel's curvature test: then hist_acc pairs and
// gamma = s.y / y.y.
__global__ void __launch_bounds__(kLbT)
    lbfgs_dots_kernel(const int n, int hist, int newest, const int cap, double gamma, const int use_pair,
                      const int hist_acc, const int newest_acc, const double *__restrict__ S,
                      const double *__restrict__ Y, const double *__restrict__ rho,
                      const double *__restrict__ gram, const double *__restrict__ gf, double *part,
                      LbfgsCoef *coef, DevScalars *sc) {
    __shared__ LbfgsScalars L;
    __shared__ double dots[2 * kLbfgsMax];
    if (use_pair && sc->pair_ok) {
        hist = hist_acc;
        newest = newest_acc;
        gamma = sc->sy / sc->yy;
    }
    hist = min(hist, kLbfgsMax - 1);
    for (int k = threadIdx.x; k < hist; k += blockDim.x) L.slot[k] = (newest - k + cap) % cap;
    __syncthreads();
    // dots 2k: s_k . g, 2k + 1: y_k . g
    block_partial_dots(2 * hist, n, [&](int d, int i) {
        return ((d & 1) ? Y : S)[(size_t)L.slot[d >> 1] * n + i] * gf[i];
    }, part);
    if (!lbfgs_last_block(sc)) return;
    reduce_partials(2 * hist, part, dots);
    for (int k = threadIdx.x; k < hist; k += blockDim.x) {
        L.sg[k] = dots[2 * k];
        L.yg[k] = dots[2 * k + 1];
    }
    load_gram(L, hist, cap, gram, rho);
    lbfgs_coefficients(L, hist, gamma, coef);
    if (threadIdx.x == 0) sc->lbfgs_done = 0u;
}

// p = -gamma gf + sum_k (cy_k y_k + cs_k s_k) and <gf, p> into sc->gp0.
__global__ void __launch_bounds__(kLbP)
    lbfgs_pdir_kernel(const int n, const LbfgsCoef *__restrict__ coef, const double *__restrict__ S,
                      const double *__restrict__ Y, const double *__restrict__ gf, double *__restrict__ p,
                      double *part, DevScalars *sc) {
    __shared__ double cy[kLbfgsMax], cs[kLbfgsMax];
    __shared__ int slot[kLbfgsMax];
    __shared__ double red[kLbP / 32];
    const int hist = coef->hist;
    const double gamma = coef->gamma;
    for (int k = threadIdx.x; k < hist; k += blockDim.x) {
        cy[k] = coef->cy[k];
        cs[k] = coef->cs[k];
        slot[k] = coef->slot[k];
    }
    __syncthreads();
    double d = 0.0;
    for (int i = blockIdx.x * kLbP + threadIdx.x; i < n; i += gridDim.x * kLbP) {
        const double g = gf[i];
        double v = -gamma * g;
#pragma unroll 8
        for (int k = 0; k < hist; ++k) {
            const size_t o = (size_t)slot[k] * n + i;
            v += cy[k] * Y[o] + cs[k] * S[o];
        }
        p[i] = v;
        d += g * v;
    }
    d = warp_sum(d);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kLbP / 32; ++w) t += red[w];
        part[(size_t)blockIdx.x * kLbfgsDots] = t;
    }
    if (!lbfgs_last_block(sc)) return;
    if (threadIdx.x < 32) {
        double t = 0.0;
        for (unsigned b = threadIdx.x; b < gridDim.x; b += 32) t += *(const volatile double *)(part + (size_t)b * kLbfgsDots);
        t = warp_sum(t);
        if (threadIdx.x == 0) {
            sc->gp0 = t;
            sc->lbfgs_done = 0u;
        }
    }
}

// Store the pair s = Wt - W, y = gft - gf in slot `slot`; sy, yy, ss, the
// curvature test and 1 / s.y into sc and rho; the Gram entries of the new pair
// with itself and with the nprev pairs in the slots before it (slot - 1, ...,
// slot - nprev, cyclically).  With dir, also the coefficients of the next
// direction for the gradient gft: the pair taken (then min(hist + 1, hist_acc)
// = hist_acc pairs newest first from `slot`, gamma = s.y / y.y) if it passes
// the test, else the hist pairs before it with the given gamma.
__global__ void __launch_bounds__(kLbT)
    lbfgs_push_kernel(const int n, const int slot, const int cap, const int nprev,
                      const double *__restrict__ W, const double *__restrict__ Wt,
                      const double *__restrict__ gf, const double *__restrict__ gft, double *S,
                      double *Y, double *__restrict__ rho, double *__restrict__ gram, double *part,
                      DevScalars *sc, const int dir, const int hist, const int hist_acc, const double gamma,
                      LbfgsCoef *coef) {
    __shared__ LbfgsScalars L;
    __shared__ double dots[kLbfgsDots];
    double *s = S + (size_t)slot * n;
    double *y = Y + (size_t)slot * n;
    for (int i = (blockIdx.x + (int)(threadIdx.x >> 5) * gridDim.x) * kLbR + (threadIdx.x & 31); i < n;
         i += gridDim.x * kLbT) {
        s[i] = Wt[i] - W[i];
        y[i] = gft[i] - gf[i];
    }
    __syncthreads();  // the block's global writes are visible to the block after the barrier
    // dots 0..2: s.y, y.y, s.s; 3 + 3j..: s . y_j, s_j . y, y . y_j (j < np, slot j = slot - 1 - j);
    // with dir, at o = 3 + 3 np: s . g, y . g, then s_j . g, y_j . g (j < nh)
    const int np = min(nprev, kLbfgsMax - 1);
    const int nh = dir ? min(hist, kLbfgsMax - 1) : 0;
    const int o = 3 + 3 * np;
    const int nd = o + (dir ? 2 + 2 * nh : 0);
    block_partial_dots(nd, n, [&](int d, int i) {
        if (d < 3) return d == 0 ? s[i] * y[i] : d == 1 ? y[i] * y[i] : s[i] * s[i];
        if (d < o) {
            const int j = (d - 3) / 3, c = (d - 3) % 3;
            const size_t q = (size_t)((slot - 1 - j + 2 * cap) % cap) * n + i;
            return c == 0 ? s[i] * Y[q] : c == 1 ? S[q] * y[i] : y[i] * Y[q];
        }
        if (d < o + 2) return (d == o ? s[i] : y[i]) * gft[i];
        const int e = d - o - 2;
        const size_t q = (size_t)((slot - 1 - (e >> 1) + 2 * cap) % cap) * n + i;
        return ((e & 1) ? Y[q] : S[q]) * gft[i];
    }, part);
    if (!lbfgs_last_block(sc)) return;
    reduce_partials(nd, part, dots);
    double *gsy = gram, *gyy = gram + (size_t)cap * cap;
    for (int j = threadIdx.x; j < np; j += blockDim.x) {
        const int sj = (slot - 1 - j + 2 * cap) % cap;
        gsy[(size_t)slot * cap + sj] = dots[3 + 3 * j];
        gsy[(size_t)sj * cap + slot] = dots[4 + 3 * j];
        gyy[(size_t)slot * cap + sj] = dots[5 + 3 * j];
        gyy[(size_t)sj * cap + slot] = dots[5 + 3 * j];
    }
    const double vsy = dots[0], vyy = dots[1], vss = dots[2];
    const bool ok = vsy > 1e-12 * sqrt(vss * vyy) && vyy > 0.0;
    if (threadIdx.x == 0) {
        gsy[(size_t)slot * cap + slot] = vsy;
        gyy[(size_t)slot * cap + slot] = vyy;
        sc->sy = vsy;
        sc->yy = vyy;
        sc->ss = vss;
        sc->pair_ok = ok ? 1 : 0;
        rho[slot] = vsy != 0.0 ? 1.0 / vsy : 0.0;
    }
    if (dir) {
        __syncthreads();  // the Gram entries and rho written above, read by load_gram
        const int h = ok ? min(hist_acc, kLbfgsMax - 1) : nh;
        for (int k = threadIdx.x; k < h; k += blockDim.x) {
            const int j = ok ? k - 1 : k;  // index among the previous pairs (-1: the new pair)
            L.slot[k] = (slot - 1 - j + 2 * cap) % cap;
            L.sg[k] = j < 0 ? dots[o] : dots[o + 2 + 2 * j];
            L.yg[k] = j < 0 ? dots[o + 1] : dots[o + 3 + 2 * j];
        }
        __syncthreads();
        load_gram(L, h, cap, gram, rho);
        lbfgs_coefficients(L, h, ok ? vsy / vyy : gamma, coef);
    }
    if (threadIdx.x == 0) sc->lbfgs_done = 0u;
}

}  // namespace

cudaError_t launch_eval_reset(Workspace &ws, cudaStream_t st, bool keep_geometry) {
    eval_reset_kernel<<<1, 1, 0, st>>>(ws.sc, keep_geometry ? 1 : 0);
    return cudaGetLastError();
}

// Threads per block of eval_begin_kernel: 64 (two warps, spreading the FP64
// work of forming p and the trial weights over more SMs) while the blocks fit
// the workspace's partial-sum rows, else 256.
static int eval_begin_threads(int n_pad, const Workspace &ws) { return n_pad / 64 <= ws.part_rows ? 64 : 256; }

cudaError_t launch_eval_begin(int n, const double *W0, double t, const double *pdir, double *Wt,
                              unsigned long long *mom, Workspace &ws, cudaStream_t st, bool form_p,
                              const double *w0, unsigned full_max) {
    const unsigned long long *wref0 = w0 ? ws.inc_aux : nullptr;
    const unsigned *hist = w0 ? ws.inc_hist : nullptr;
    const int n_pad = ((n + kChunk - 1) / kChunk) * kChunk;
    const long long n_mom = (long long)n * moment_width(ws.dim);
    if (n_pad == 0) return cudaSuccess;
    const bool fp = form_p && pdir;
    const int tpb = eval_begin_threads(n_pad, ws);
    eval_begin_kernel<<<n_pad / tpb, tpb, 0, st>>>(n, n_pad, n_mom, W0, t, const_cast<double *>(pdir), Wt,
                                                   ws.sorted ? ws.perm : nullptr, ws.recs, ws.recs32,
                                                   ws.sorted ? ws.recs32s : nullptr, ws.groups, mom, ws.part, ws.sc,
                                                   fp ? ws.lb_coef : nullptr, ws.S, ws.Y, ws.gf, w0, wref0,
                                                   hist, full_max, w0 ? ws.inc_drift : nullptr);
    return cudaGetLastError();
}

const void *eval_begin_kernel_fn() { return reinterpret_cast<const void *>(eval_begin_kernel); }

// The same launch as launch_eval_begin, written into a kernel node of an
// instantiated graph (only the trial step t changes between replays).
cudaError_t set_eval_begin_node(cudaGraphExec_t exec, cudaGraphNode_t node, int n, const double *W0, double t,
                                const double *pdir, double *Wt, unsigned long long *mom, Workspace &ws,
                                bool form_p, const double *w0, unsigned full_max) {
    const unsigned long long *wref0 = w0 ? ws.inc_aux : nullptr;
    const unsigned *hist = w0 ? ws.inc_hist : nullptr;
    float2 *drift = w0 ? ws.inc_drift : nullptr;
    int n_pad = ((n + kChunk - 1) / kChunk) * kChunk;
    long long n_mom = (long long)n * moment_width(ws.dim);
    const int32_t *perm = ws.sorted ? ws.perm : nullptr;
    SeedRec *recs = ws.recs;
    SeedRec32 *recs32 = ws.recs32, *recs32s = ws.sorted ? ws.recs32s : nullptr;
    GroupBound *groups = ws.groups;
    double *part = ws.part;
    DevScalars *sc = ws.sc;
    double *pd = const_cast<double *>(pdir);
    const LbfgsCoef *coef = form_p && pdir ? ws.lb_coef : nullptr;
    const double *S = ws.S, *Y = ws.Y, *gfv = ws.gf;
    void *args[] = {&n,      &n_pad,   &n_mom,  &W0,  &t,    &pd, &Wt,   &perm, &recs, &recs32,
                    &recs32s, &groups, &mom, &part, &sc, &coef, &S, &Y, &gfv, &w0, &wref0, &hist, &full_max,
                    &drift};
    cudaKernelNodeParams p{};
    p.func = reinterpret_cast<void *>(eval_begin_kernel);
    const int tpb = eval_begin_threads(n_pad, ws);
    p.gridDim = dim3(n_pad / tpb);
    p.blockDim = dim3(tpb);
    p.sharedMemBytes = 0;
    p.kernelParams = args;
    p.extra = nullptr;
    return cudaGraphExecKernelNodeSetParams(exec, node, &p);
}

// Incremental pass, before scoring: a re-decision starts from the recorded
// moments; a recording clears the margin histogram its scorer fills.
__global__ void inc_prepare_kernel(const long long n_mom, unsigned long long *__restrict__ mom,
                                   const unsigned long long *__restrict__ mom0, unsigned *__restrict__ hist,
                                   const DevScalars *__restrict__ sc) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    if (sc->inc_go) {
        for (long long e = i; e < n_mom; e += stride) mom[e] = mom0[e];
    } else {
        for (long long e = i; e < kIncBins; e += stride) hist[e] = 0u;
    }
}

// Incremental pass, after rescoring: a recording keeps its moments, weights and
// w_ref for the re-decisions that follow.
__global__ void inc_commit_kernel(const int n, const long long n_mom, const unsigned long long *__restrict__ mom,
                                  const double *__restrict__ w, unsigned long long *__restrict__ mom0,
                                  double *__restrict__ w0, unsigned long long *__restrict__ aux,
                                  DevScalars *__restrict__ sc) {
    if (sc->inc_go) return;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (long long e = i; e < n_mom; e += (long long)gridDim.x * blockDim.x) mom0[e] = mom[e];
    for (long long e = i; e < n; e += (long long)gridDim.x * blockDim.x) w0[e] = w[e];
    if (i == 0) {
        aux[0] = sc->wref_key;
        sc->inc_valid = 1;
    }
}

cudaError_t launch_inc_prepare(int n, unsigned long long *mom, Workspace &ws, cudaStream_t st) {
    const long long n_mom = (long long)n * moment_width(ws.dim);
    const int blocks = (int)std::max<long long>(1, std::min<long long>((n_mom + 255) / 256, 4 * ws.sms));
    inc_prepare_kernel<<<blocks, 256, 0, st>>>(n_mom, mom, ws.inc_mom0, ws.inc_hist, ws.sc);
    return cudaGetLastError();
}

cudaError_t launch_inc_commit(int n, const unsigned long long *mom, const double *w, Workspace &ws,
                              cudaStream_t st) {
    const long long n_mom = (long long)n * moment_width(ws.dim);
    const int blocks = (int)std::max<long long>(1, std::min<long long>((n_mom + 255) / 256, 4 * ws.sms));
    inc_commit_kernel<<<blocks, 256, 0, st>>>(n, n_mom, mom, w, ws.inc_mom0, ws.inc_w0, ws.inc_aux, ws.sc);
    return cudaGetLastError();
}

cudaError_t launch_seed_prep(const GridDev &g, int n, const double *x, const double *A,
                             const double *w, Workspace &ws, cudaStream_t st) {
    const int n_pad = ((n + kChunk - 1) / kChunk) * kChunk;
    const int blocks = (n_pad + 255) / 256;
    int m = 1;
    while (m < n_pad) m <<= 1;
    // Morton order for the scoring scan when the workspace has the buffers
    ws.sorted = ws.recs_tmp && ws.codes && ws.scodes && ws.perm && ws.recs32s && m <= kSortMax;
    SeedRec *dst = ws.sorted ? ws.recs_tmp : ws.recs;
    uint32_t *codes = ws.sorted ? ws.codes : nullptr;
    if (g.dim == 3)
        seed_prep_kernel<3><<<blocks, 256, 0, st>>>(g, n, n_pad, x, A, w, dst, ws.recs32, codes, ws.sc);
    else
        seed_prep_kernel<2><<<blocks, 256, 0, st>>>(g, n, n_pad, x, A, w, dst, ws.recs32, codes, ws.sc);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !ws.sorted) return e;
    const size_t smem = (size_t)m * sizeof(unsigned long long);
    if (!(ws.attr_done & kAttrMortonSort)) {
        e = cudaFuncSetAttribute(morton_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(kSortMax * sizeof(unsigned long long)));
        if (e != cudaSuccess) return e;
        ws.attr_done |= kAttrMortonSort;
    }
    morton_sort_kernel<<<1, 1024, smem, st>>>(n_pad, m, ws.codes, ws.scodes, ws.perm);
    gather_recs_kernel<<<blocks, 256, 0, st>>>(n_pad, ws.perm, ws.recs_tmp, ws.recs, ws.recs32, ws.recs32s);
    return cudaGetLastError();
}

cudaError_t launch_group_bounds(int n, Workspace &ws, cudaStream_t st) {
    if (!ws.groups) return cudaSuccess;
    const int groups = (n + 31) / 32;
    const int blocks = (groups * 32 + 255) / 256;
    if (ws.dim == 3) group_bounds_kernel<3><<<blocks, 256, 0, st>>>(n, ws.recs, ws.groups, ws.sc);
    else group_bounds_kernel<2><<<blocks, 256, 0, st>>>(n, ws.recs, ws.groups, ws.sc);
    return cudaGetLastError();
}

// Blocks of the dual kernel: 64 cells each, at most the workspace's partial rows.
static int dual_blocks(int n, const Workspace &ws) {
    return std::max(1, std::min((n + kDualThreads / 4 - 1) / (kDualThreads / 4), ws.part_rows));
}

cudaError_t launch_dual(const GridDev &g, int n, const double *x, const double *A, const double *w,
                        const double *v, const double *p_dir, const unsigned long long *moments,
                        Workspace &ws, double *g_out, double *grad_out, double *gf_out,
                        double *err_out, cudaStream_t st) {
    const int blocks = dual_blocks(n, ws);
    if (g.dim == 3)
        dual_kernel<3><<<blocks, kDualThreads, 0, st>>>(g, n, x, A, w, v, p_dir, moments, ws.part, ws.sc, g_out,
                                                   grad_out, gf_out, err_out);
    else
        dual_kernel<2><<<blocks, kDualThreads, 0, st>>>(g, n, x, A, w, v, p_dir, moments, ws.part, ws.sc, g_out,
                                                   grad_out, gf_out, err_out);
    return cudaGetLastError();
}

cudaError_t launch_points_dual(int dim, int n, const double *x, const double *A, const double *w, const double *v,
                               const double *mom_pts, Workspace &ws, double *g_out, double *grad_out,
                               double *err_out, cudaStream_t st) {
    const int blocks = dual_blocks(n, ws);
    GridDev g;
    memset(&g, 0, sizeof g);
    g.dim = dim;
    if (dim == 3)
        dual_kernel<3, true><<<blocks, kDualThreads, 0, st>>>(g, n, x, A, w, v, nullptr, nullptr, ws.part, ws.sc, g_out,
                                                         grad_out, nullptr, err_out, mom_pts);
    else
        dual_kernel<2, true><<<blocks, kDualThreads, 0, st>>>(g, n, x, A, w, v, nullptr, nullptr, ws.part, ws.sc, g_out,
                                                         grad_out, nullptr, err_out, mom_pts);
    return cudaGetLastError();
}

cudaError_t launch_centroids(const GridDev &g, int n, const double *x,
                             const unsigned long long *moments, double *x_out, cudaStream_t st) {
    const int blocks = (n + 255) / 256;
    if (g.dim == 3)
        centroid_kernel<3><<<blocks, 256, 0, st>>>(g, n, x, moments, x_out);
    else
        centroid_kernel<2><<<blocks, 256, 0, st>>>(g, n, x, moments, x_out);
    return cudaGetLastError();
}

cudaError_t launch_axpy(int n, const double *a, double t, const double *b, double *out,
                        cudaStream_t st) {
    axpy_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, a, t, b, out);
    return cudaGetLastError();
}

// The dot-product kernels take one block per 32 seeds, the p kernel one per 64,
// each at most one block per SM (the workspace's partial-sum rows).
static int lbfgs_blocks(int n, int per, const Workspace &ws) {
    return std::max(1, std::min((n + per - 1) / per, ws.lb_rows));
}

cudaError_t launch_lbfgs_direction(int n, int hist, int newest, int cap, double gamma, bool use_pair,
                                   int hist_acc, int newest_acc, Workspace &ws, cudaStream_t st) {
    if (cap > kLbfgsMax || hist > cap || hist_acc > cap || !ws.lb_part || !ws.lb_coef || ws.lb_rows < 1)
        return cudaErrorInvalidValue;
    const cudaError_t e = launch_lbfgs_coefficients(n, hist, newest, cap, gamma, use_pair, hist_acc, newest_acc, ws, st);
    return e != cudaSuccess ? e : launch_lbfgs_pdir(n, ws, st);
}

cudaError_t launch_lbfgs_coefficients(int n, int hist, int newest, int cap, double gamma, bool use_pair,
                                      int hist_acc, int newest_acc, Workspace &ws, cudaStream_t st) {
    if (cap > kLbfgsMax || hist > cap || hist_acc > cap || !ws.lb_part || !ws.lb_coef || ws.lb_rows < 1)
        return cudaErrorInvalidValue;
    lbfgs_dots_kernel<<<lbfgs_blocks(n, kLbR, ws), kLbT, 0, st>>>(n, hist, newest, cap, gamma, use_pair ? 1 : 0,
                                                                  hist_acc, newest_acc, ws.S, ws.Y, ws.rho, ws.gram,
                                                                  ws.gf, ws.lb_part, ws.lb_coef, ws.sc);
    return cudaGetLastError();
}

cudaError_t launch_lbfgs_pdir(int n, Workspace &ws, cudaStream_t st) {
    if (!ws.lb_part || !ws.lb_coef || ws.lb_rows < 1) return cudaErrorInvalidValue;
    lbfgs_pdir_kernel<<<lbfgs_blocks(n, kLbP, ws), kLbP, 0, st>>>(n, ws.lb_coef, ws.S, ws.Y, ws.gf, ws.p,
                                                                  ws.lb_part, ws.sc);
    return cudaGetLastError();
}

cudaError_t launch_lbfgs_push(int n, int slot, int cap, int nprev, bool dir, int hist, int hist_acc, double gamma,
                              Workspace &ws, cudaStream_t st) {
    if (cap > kLbfgsMax || nprev >= cap || hist >= cap || hist_acc >= cap || !ws.lb_part || !ws.lb_coef ||
        !ws.gram || ws.lb_rows < 1)
        return cudaErrorInvalidValue;
    lbfgs_push_kernel<<<lbfgs_blocks(n, kLbR, ws), kLbT, 0, st>>>(n, slot, cap, nprev, ws.W, ws.Wt, ws.gf, ws.gft,
                                                                  ws.S, ws.Y, ws.rho, ws.gram, ws.lb_part, ws.sc,
                                                                  dir ? 1 : 0, hist, hist_acc, gamma, ws.lb_coef);
    return cudaGetLastError();
}

}  // namespace apd
