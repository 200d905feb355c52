// Seed preparation, the dual value/gradient of eqs. (2.7)-(2.8) from integer
// moments, the discrete centroids of Algorithm 3, and the vector kernels of
// the L-BFGS weight solve (Algorithm 2).
#include <float.h>

#include "apd_internal.cuh"

namespace apd {

namespace {

constexpr int kRedThreads = 1024;

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
__device__ double block_sum(double v, double *sh) {
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

__global__ void eval_reset_kernel(DevScalars *sc) {
    sc->flag_count = 0u;
    sc->wref_key = 0ull;
    sc->lam_abs_bits = 0ull;
    sc->lam_min_bits = 0x7ff0000000000000ull;
    sc->dual_done = 0u;
}

// Smallest eigenvalue of a symmetric positive-definite 2x2 or 3x3 matrix (FP64):
// 2x2 from the characteristic quadratic; 3x3 from the trigonometric solution of
// the characteristic cubic (shifted by the mean eigenvalue, scaled by the root
// mean square deviation).  Returned with a small relative safety margin.
template <int D>
__device__ double lambda_min_sym(const double (&s)[D][D]) {
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

__device__ __forceinline__ void split_f32(double v, float &hi, float &lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

template <int D>
__global__ void seed_prep_kernel(const GridDev g, const int n, const int n_pad,
                                 const double *__restrict__ x, const double *__restrict__ A,
                                 const double *__restrict__ w, SeedRec *__restrict__ recs,
                                 SeedRec32 *__restrict__ recs32, uint32_t *__restrict__ codes,
                                 DevScalars *__restrict__ sc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    SeedRec r;
#pragma unroll
    for (int a = 0; a < 3; ++a) r.x[a] = 0.0;
    r.w = 0.0;
#pragma unroll
    for (int a = 0; a < 6; ++a) r.a[a] = 0.f;
    r.pad[0] = r.pad[1] = 0.f;
    SeedRec32 r32;
#pragma unroll
    for (int a = 0; a < 3; ++a) r32.xh[a] = r32.xl[a] = 0.f;
    r32.wh = r32.wl = 0.f;
#pragma unroll
    for (int a = 0; a < 6; ++a) r32.a[a] = 0.f;
    r32.pad[0] = r32.pad[1] = 0.f;
    double wkey_w = -DBL_MAX, frob = 0.0, lam = DBL_MAX;
    bool active = false;
    if (i < n) {
        active = true;
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
        if (!finite) atomicOr(&sc->status, ST_NONFINITE);
        else if (!spd) atomicOr(&sc->status, ST_NOT_SPD);
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
        wkey_w = finite ? wi : -DBL_MAX;
#pragma unroll
        for (int a = 0; a < D; ++a) split_f32(xx[a], r32.xh[a], r32.xl[a]);
        split_f32(wi, r32.wh, r32.wl);
#pragma unroll
        for (int a = 0; a < 6; ++a) r32.a[a] = r.a[a];
    }
    if (i < n_pad) {
        recs[i] = r;
        recs32[i] = r32;
        if (codes) {
            uint32_t code = 0xffffffffu;  // padding sorts last
            if (i < n) {
                double frac[3] = {0.0, 0.0, 0.0};
#pragma unroll
                for (int a = 0; a < D; ++a) frac[a] = (r.x[a] - g.lo[a]) / ((double)g.res[a] * g.h[a]);
                code = morton_code(D, frac);
            }
            codes[i] = code;
        }
    }
    // one atomic per warp for each statistic
    const double wmax = warp_max(active ? wkey_w : -DBL_MAX);
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
    for (int i = threadIdx.x; i < n_pad; i += blockDim.x) {
        scodes[i] = (uint32_t)(keys[i] >> 32);
        perm[i] = (int32_t)(keys[i] & 0xffffffffu);
    }
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

// Per-cell dual terms from the integer moments, then a deterministic two-phase
// reduction (block partials summed in block order by the last block).
//   m_i = M0, mean odd coordinate mu = S1 / m, centred second moment
//   C = S2 - S1 S1^T / m (in units of (h/2)^2), centroid offset e = lo + (h/2) mu - x_i,
//   Q_i = sum_ab A_ab ((h_a h_b / 4) C_ab + m e_a e_b) = sum_{H_j=i} |y_j - x_i|^2_{A_i},
//   g_i = (v_i - m_i |P|) w_i + |P| Q_i,   grad_i = v_i - m_i |P|.
template <int D>
__global__ void __launch_bounds__(256)
    dual_kernel(const GridDev g, const int n, const double *__restrict__ x,
                const double *__restrict__ A, const double *__restrict__ w,
                const double *__restrict__ v, const double *__restrict__ p_dir,
                const unsigned long long *__restrict__ mom, double *__restrict__ part,
                DevScalars *__restrict__ sc, double *g_out, double *grad_out, double *gf_out,
                double *err_out) {
    constexpr int K = moment_width(D);
    __shared__ double sh[33];
    __shared__ bool last;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double gsum = 0.0, emax = 0.0, gp = 0.0, sv = 0.0, vmin = DBL_MAX;
    if (i < n) {
        const unsigned long long *mo = mom + (size_t)i * K;
        const double m = (double)mo[0];
        const double vi = v[i], wi = w[i];
        if (!(vi > 0.0) || !isfinite(vi)) atomicOr(&sc->status, ST_BAD_VOLUME);
        // v_i - m_i |P| with two roundings (no contraction), as eq. (2.8) is written
        const double gr = __dsub_rn(vi, __dmul_rn(m, g.cell));
        double Q = 0.0;
        if (mo[0] > 0ull) {
            double S1[D], e[D];
#pragma unroll
            for (int a = 0; a < D; ++a) {
                S1[a] = (double)mo[1 + a];
                e[a] = (g.lo[a] + 0.5 * g.h[a] * (S1[a] / m)) - x[(size_t)i * D + a];
            }
            int t = 1 + D;
#pragma unroll
            for (int a = 0; a < D; ++a)
#pragma unroll
                for (int b = a; b < D; ++b) {
                    const double Cab = (double)mo[t++] - S1[a] * S1[b] / m;
                    const double Mab = 0.25 * g.h[a] * g.h[b] * Cab + m * e[a] * e[b];
                    const double Aab = (a == b) ? A[(size_t)i * D * D + a * D + a]
                                                : A[(size_t)i * D * D + a * D + b] +
                                                      A[(size_t)i * D * D + b * D + a];
                    Q += Aab * Mab;
                }
        }
        gsum = gr * wi + g.cell * Q;
        emax = __ddiv_rn(fabs(gr), vi);
        if (grad_out) grad_out[i] = gr;
        if (gf_out) gf_out[i] = -gr;
        if (p_dir) gp = -gr * p_dir[i];
        sv = vi;
        vmin = vi;
    }
    const double bg = block_sum(gsum, sh);
    const double bp = block_sum(gp, sh);
    const double bs = block_sum(sv, sh);
    // max / min through the same tree
    double em = warp_max(emax), vm = warp_min(vmin);
    __shared__ double shm[32], shn[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        shm[wid] = em;
        shn[wid] = vm;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = DBL_MAX;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            a = fmax(a, shm[k]);
            b = fmin(b, shn[k]);
        }
        double *pp = part + (size_t)blockIdx.x * 5;
        pp[0] = bg;
        pp[1] = a;
        pp[2] = bp;
        pp[3] = bs;
        pp[4] = b;
        __threadfence();
        const unsigned t = atomicAdd(&sc->dual_done, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double G = 0.0, E = 0.0, GP = 0.0, SV = 0.0, VM = DBL_MAX;
        for (unsigned k = 0; k < gridDim.x; ++k) {
            const volatile double *pp = part + (size_t)k * 5;
            G += pp[0];
            E = fmax(E, pp[1]);
            GP += pp[2];
            SV += pp[3];
            VM = fmin(VM, pp[4]);
        }
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

// Two-loop recursion: p = -H gf with H0 = gamma I and the stored pairs
// (s_k, y_k), newest at slot `newest`; also <gf, p> into sc->gp0.
__global__ void __launch_bounds__(kRedThreads)
    lbfgs_direction_kernel(const int n, const int hist, const int newest, const int cap,
                           const double gamma, const double *__restrict__ S,
                           const double *__restrict__ Y, const double *__restrict__ rho,
                           double *__restrict__ alpha, const double *__restrict__ gf,
                           double *__restrict__ p, DevScalars *sc) {
    __shared__ double sh[33];
    for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = gf[i];
    for (int k = 0; k < hist; ++k) {
        const int idx = (newest - k + cap) % cap;
        const double *s = S + (size_t)idx * n;
        const double *y = Y + (size_t)idx * n;
        double d = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) d += s[i] * p[i];
        const double a = rho[idx] * block_sum(d, sh);
        if (threadIdx.x == 0) alpha[idx] = a;
        for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] -= a * y[i];
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] *= gamma;
    for (int k = hist - 1; k >= 0; --k) {
        const int idx = (newest - k + cap) % cap;
        const double *s = S + (size_t)idx * n;
        const double *y = Y + (size_t)idx * n;
        double d = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) d += y[i] * p[i];
        const double bta = rho[idx] * block_sum(d, sh);
        __syncthreads();
        const double a = alpha[idx];
        for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] += s[i] * (a - bta);
    }
    double d = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        p[i] = -p[i];
        d += gf[i] * p[i];
    }
    const double gp = block_sum(d, sh);
    if (threadIdx.x == 0) sc->gp0 = gp;
}

// Store the pair s = Wt - W, y = gft - gf in slot `slot`; sy, yy, ss into sc.
__global__ void __launch_bounds__(kRedThreads)
    lbfgs_push_kernel(const int n, const int slot, const double *__restrict__ W,
                      const double *__restrict__ Wt, const double *__restrict__ gf,
                      const double *__restrict__ gft, double *__restrict__ S,
                      double *__restrict__ Y, double *__restrict__ rho, DevScalars *sc) {
    __shared__ double sh[33];
    double sy = 0.0, yy = 0.0, ss = 0.0;
    double *s = S + (size_t)slot * n;
    double *y = Y + (size_t)slot * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double si = Wt[i] - W[i];
        const double yi = gft[i] - gf[i];
        s[i] = si;
        y[i] = yi;
        sy += si * yi;
        yy += yi * yi;
        ss += si * si;
    }
    sy = block_sum(sy, sh);
    yy = block_sum(yy, sh);
    ss = block_sum(ss, sh);
    if (threadIdx.x == 0) {
        sc->sy = sy;
        sc->yy = yy;
        sc->ss = ss;
        rho[slot] = sy != 0.0 ? 1.0 / sy : 0.0;
    }
}

}  // namespace

cudaError_t launch_eval_reset(Workspace &ws, cudaStream_t st) {
    eval_reset_kernel<<<1, 1, 0, st>>>(ws.sc);
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
    static bool attr = false;
    if (!attr) {
        e = cudaFuncSetAttribute(morton_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(kSortMax * sizeof(unsigned long long)));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    morton_sort_kernel<<<1, 1024, smem, st>>>(n_pad, m, ws.codes, ws.scodes, ws.perm);
    gather_recs_kernel<<<blocks, 256, 0, st>>>(n_pad, ws.perm, ws.recs_tmp, ws.recs, ws.recs32, ws.recs32s);
    return cudaGetLastError();
}

cudaError_t launch_dual(const GridDev &g, int n, const double *x, const double *A, const double *w,
                        const double *v, const double *p_dir, const unsigned long long *moments,
                        Workspace &ws, double *g_out, double *grad_out, double *gf_out,
                        double *err_out, cudaStream_t st) {
    const int blocks = (n + 255) / 256;
    if (g.dim == 3)
        dual_kernel<3><<<blocks, 256, 0, st>>>(g, n, x, A, w, v, p_dir, moments, ws.part, ws.sc, g_out,
                                               grad_out, gf_out, err_out);
    else
        dual_kernel<2><<<blocks, 256, 0, st>>>(g, n, x, A, w, v, p_dir, moments, ws.part, ws.sc, g_out,
                                               grad_out, gf_out, err_out);
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

cudaError_t launch_lbfgs_direction(int n, int hist, int newest, int cap, double gamma, Workspace &ws,
                                   cudaStream_t st) {
    lbfgs_direction_kernel<<<1, kRedThreads, 0, st>>>(n, hist, newest, cap, gamma, ws.S, ws.Y, ws.rho,
                                                      ws.alpha, ws.gf, ws.p, ws.sc);
    return cudaGetLastError();
}

cudaError_t launch_lbfgs_push(int n, int slot, Workspace &ws, cudaStream_t st) {
    lbfgs_push_kernel<<<1, kRedThreads, 0, st>>>(n, slot, ws.W, ws.Wt, ws.gf, ws.gft, ws.S, ws.Y,
                                                 ws.rho, ws.sc);
    return cudaGetLastError();
}

}  // namespace apd
