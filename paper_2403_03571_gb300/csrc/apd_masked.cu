// Masked two-level discretisation (the outlook of Section 4: adaptable pixel
// sizes, with the pixels at the cell boundaries found by masking).  After
// Algorithm 1 on a coarse grid G (the one-instance scoring pass, whose labels
// and seed records this file reuses):
//
// Mask.  One thread per coarse pixel compares its label with the 3^D
// neighbourhood inside the grid.  A boundary pixel is appended to a list (one
// atomic per warp).  An interior pixel adds the integer moments of its r^D
// fine pixels in closed form: with U = 2K + 1 its odd coarse coordinate, the
// fine u = 2k + 1 of the block along one axis are r U - (r - 1) + 2j,
// j = 0..r-1, whose sum is r^2 U and sum of squares r^3 U^2 + (r^3 - r) / 3, so
//     count = r^D,  sum u_a = r^(D+1) U_a,  sum u_a u_b = r^(D+2) U_a U_b (a != b),
//     sum u_a^2 = r^(D+2) U_a^2 + r^D (r^2 - 1) / 3.
//
// Refine.  One thread per fine pixel of a listed coarse pixel (a persistent
// grid over the device-side count): the FP64 pixel centre of the fine grid,
// then the two passes of the non-uniform kernel (FP32 direct-form costs with
// their rounding bounds give a threshold; the seeds under it are recomputed in
// FP64 with the reference operation order; lowest index on ties), so the
// label equals Algorithm 1 on the fine grid.  Moments as integers of the fine
// grid.
//
// Both kernels sum the moments of the lanes holding the same label with
// shuffles before one atomic per (label, word).
#include <algorithm>

#include "apd_common.cuh"
#include "apd_cost.cuh"

namespace apd {

namespace {

constexpr int kMaskThreads = 256;

__device__ __forceinline__ unsigned long long warp_sum_ull(unsigned long long v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Adds val to the moments of cell `label` for the lanes with has set; lanes of
// one label are summed first.  Called by all 32 lanes of the warp.
template <int D>
__device__ __forceinline__ void warp_add_moments(bool has, int label, const unsigned long long (&val)[moment_width(D)],
                                                 unsigned long long *__restrict__ gmom) {
    constexpr int K = moment_width(D);
    const int lane = threadIdx.x & 31;
    unsigned todo = __ballot_sync(0xffffffffu, has);
    while (todo) {
        const int leader = __ffs(todo) - 1;
        const int L0 = __shfl_sync(0xffffffffu, label, leader);
        const bool mine = has && label == L0;
        const unsigned grp = __ballot_sync(0xffffffffu, mine);
#pragma unroll
        for (int v = 0; v < K; ++v) {
            const unsigned long long s = warp_sum_ull(mine ? val[v] : 0ull);
            if (lane == leader && s) atomicAdd(&gmom[(size_t)L0 * K + v], s);
        }
        todo &= ~grp;
    }
}

// Integer moments of one fine pixel (u = 2k + 1), word order of apd_cell_moments.
template <int D>
__device__ __forceinline__ void pixel_moments(const int (&k)[3], unsigned long long (&val)[moment_width(D)]) {
    unsigned long long u[3];
#pragma unroll
    for (int a = 0; a < D; ++a) u[a] = 2ull * (unsigned long long)k[a] + 1ull;
    val[0] = 1ull;
#pragma unroll
    for (int a = 0; a < D; ++a) val[1 + a] = u[a];
    int e = 1 + D;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = a; b < D; ++b) val[e++] = u[a] * u[b];
}

// Closed-form integer moments of the r^D fine pixels of coarse pixel K.
template <int D>
__device__ __forceinline__ void block_moments(const int (&K)[3], unsigned long long r,
                                              unsigned long long (&val)[moment_width(D)]) {
    unsigned long long rD = r * r;
    if (D == 3) rD *= r;
    const unsigned long long r2 = r * r;
    const unsigned long long diag = rD * (r2 - 1ull) / 3ull;  // r^D (r - 1)(r + 1) / 3, an integer
    unsigned long long U[3];
#pragma unroll
    for (int a = 0; a < D; ++a) U[a] = 2ull * (unsigned long long)K[a] + 1ull;
    val[0] = rD;
#pragma unroll
    for (int a = 0; a < D; ++a) val[1 + a] = rD * r * U[a];
    int e = 1 + D;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = a; b < D; ++b) val[e++] = rD * r2 * U[a] * U[b] + (a == b ? diag : 0ull);
}

template <int D>
__global__ void __launch_bounds__(kMaskThreads)
    mask_kernel(const GridDev gc, const unsigned long long r, const int n, const int32_t *__restrict__ lab,
                uint32_t *__restrict__ list, DevScalars *__restrict__ sc, unsigned long long *__restrict__ gmom) {
    constexpr int K = moment_width(D);
    const int lane = threadIdx.x & 31;
    const long long Jc = gc.J;
    for (long long j0 = (long long)blockIdx.x * kMaskThreads; j0 < Jc; j0 += (long long)gridDim.x * kMaskThreads) {
        const long long j = j0 + threadIdx.x;
        const bool active = j < Jc;
        int kc[3] = {0, 0, 0};
        int L = -1;
        bool boundary = false;
        if (active) {
            long long rr = j;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                kc[a] = (int)(rr % gc.res[a]);
                rr /= gc.res[a];
            }
            L = lab[j];
            const int z0 = D == 3 ? -1 : 0, z1 = D == 3 ? 1 : 0;
            for (int dz = z0; dz <= z1; ++dz) {
                const int nz = kc[2] + dz;
                if (D == 3 && (nz < 0 || nz >= gc.res[2])) continue;
                for (int dy = -1; dy <= 1; ++dy) {
                    const int ny = kc[1] + dy;
                    if (ny < 0 || ny >= gc.res[1]) continue;
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int nx = kc[0] + dx;
                        if (nx < 0 || nx >= gc.res[0]) continue;
                        const long long nj = (long long)nx + (long long)gc.res[0] * ((long long)ny +
                                                                                      (long long)gc.res[1] * nz);
                        boundary |= lab[nj] != L;
                    }
                }
            }
        }
        const bool valid = active && L >= 0 && L < n;
        if (active && !valid) atomicOr(&sc->status, ST_BAD_LABEL);
        // boundary pixels into the list: one atomic per warp
        const bool push = valid && boundary;
        const unsigned pm = __ballot_sync(0xffffffffu, push);
        if (pm) {
            const int first = __ffs(pm) - 1;
            unsigned base = 0u;
            if (lane == first) base = atomicAdd(&sc->mask_count, (unsigned)__popc(pm));
            base = __shfl_sync(0xffffffffu, base, first);
            if (push) list[base + (unsigned)__popc(pm & ((1u << lane) - 1u))] = (uint32_t)j;
        }
        const bool interior = valid && !boundary;
        unsigned long long val[K];
        block_moments<D>(kc, r, val);
        warp_add_moments<D>(interior, L, val, gmom);
    }
}

template <int D>
__global__ void __launch_bounds__(kMaskThreads)
    refine_kernel(const GridDev gc, const GridDev gf, const int r, const int sub, const int n,
                  const double *__restrict__ x, const double *__restrict__ A, const double *__restrict__ w,
                  const SeedRec32 *__restrict__ r32, const uint32_t *__restrict__ list,
                  DevScalars *__restrict__ sc, unsigned long long *__restrict__ gmom, long long *refined) {
    constexpr int K = moment_width(D);
    __shared__ SeedRec32 sr[kMaskThreads];
    const long long total = (long long)sc->mask_count * sub;
    if (refined && blockIdx.x == 0 && threadIdx.x == 0) *refined = total;
    const double wref = dkey_inv(sc->wref_key);
    float wrh, wrl;
    split_f32(wref, wrh, wrl);
    for (long long t0 = (long long)blockIdx.x * kMaskThreads; t0 < total;
         t0 += (long long)gridDim.x * kMaskThreads) {
        const long long t = t0 + threadIdx.x;
        const bool active = t < total;
        int k[3] = {0, 0, 0};
        double yy[D];
        float yh[3] = {0.f, 0.f, 0.f}, yl[3] = {0.f, 0.f, 0.f};
        if (active) {
            const long long b = t / sub;
            int s = (int)(t - b * sub);
            long long jc = (long long)list[b];
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const int kc = (int)(jc % gc.res[a]);
                jc /= gc.res[a];
                k[a] = kc * r + s % r;
                s /= r;
            }
        }
#pragma unroll
        for (int a = 0; a < D; ++a) {
            // pixel centre of the fine grid, the reference operation order
            yy[a] = __dadd_rn(gf.lo[a], __dmul_rn((double)k[a] + 0.5, gf.h[a]));
            split_f32(yy[a], yh[a], yl[a]);
        }
        // pass 1: threshold = min_k (C_k + E_k)
        float thr = __int_as_float(0x7f800000);
        for (int c0 = 0; c0 < n; c0 += kMaskThreads) {
            const int m = min(kMaskThreads, n - c0);
            __syncthreads();
            if ((int)threadIdx.x < m) sr[threadIdx.x] = r32[c0 + threadIdx.x];
            __syncthreads();
            for (int q = 0; q < m; ++q) {
                float c, E;
                cost32_bound<D>(sr[q], yh, yl, wrh, wrl, c, E);
                thr = fminf(thr, c + E);
            }
        }
        // pass 2: FP64 reference cost of the seeds under the threshold
        double best = __longlong_as_double(0x7ff0000000000000ll);
        int bi = -1;
        for (int c0 = 0; c0 < n; c0 += kMaskThreads) {
            const int m = min(kMaskThreads, n - c0);
            __syncthreads();
            if ((int)threadIdx.x < m) sr[threadIdx.x] = r32[c0 + threadIdx.x];
            __syncthreads();
            if (!active) continue;
            for (int q = 0; q < m; ++q) {
                float c, E;
                cost32_bound<D>(sr[q], yh, yl, wrh, wrl, c, E);
                if (!(c - E <= thr)) continue;
                const int s = c0 + q;
                const double c64 = cost64<D>(yy, x + (size_t)s * D, A + (size_t)s * D * D, w[s]);
                if (bi < 0 || c64 < best) {  // seeds in increasing order: ties keep the lowest index
                    best = c64;
                    bi = s;
                }
            }
        }
        const bool valid = active && bi >= 0 && bi < n;
        if (active && !valid) atomicOr(&sc->status, ST_BAD_LABEL);
        unsigned long long val[K];
        pixel_moments<D>(k, val);
        warp_add_moments<D>(valid, bi, val, gmom);
    }
}

}  // namespace

cudaError_t launch_masked_refine(const GridDev &gc, const GridDev &gf, int r, int n, const double *x,
                                 const double *A, const double *w, const int32_t *coarse_labels,
                                 unsigned long long *mom, long long *refined, Workspace &ws, cudaStream_t st) {
    const int K = moment_width(gc.dim);
    cudaError_t e = cudaMemsetAsync(mom, 0, (size_t)n * K * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(&ws.sc->mask_count, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    const int sms = ws.sms;
    const int mblocks = (int)std::min<long long>((gc.J + kMaskThreads - 1) / kMaskThreads, (long long)sms * 8);
    if (gc.dim == 3)
        mask_kernel<3><<<mblocks, kMaskThreads, 0, st>>>(gc, (unsigned long long)r, n, coarse_labels, ws.flags,
                                                         ws.sc, mom);
    else
        mask_kernel<2><<<mblocks, kMaskThreads, 0, st>>>(gc, (unsigned long long)r, n, coarse_labels, ws.flags,
                                                         ws.sc, mom);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the number of listed pixels is known on the device only: a persistent
    // grid (8 blocks of 256 per SM) strides over r^D times that count
    const int sub = gc.dim == 3 ? r * r * r : r * r;
    const long long most = (gc.J * (long long)sub + kMaskThreads - 1) / kMaskThreads;
    const int rblocks = (int)std::max<long long>(1, std::min<long long>(most, (long long)sms * 8));
    if (gc.dim == 3)
        refine_kernel<3><<<rblocks, kMaskThreads, 0, st>>>(gc, gf, r, sub, n, x, A, w, ws.recs32, ws.flags, ws.sc,
                                                           mom, refined);
    else
        refine_kernel<2><<<rblocks, kMaskThreads, 0, st>>>(gc, gf, r, sub, n, x, A, w, ws.recs32, ws.flags, ws.sc,
                                                           mom, refined);
    return cudaGetLastError();
}

}  // namespace apd
