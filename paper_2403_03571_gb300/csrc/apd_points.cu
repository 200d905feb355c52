// Algorithm 1 on a non-uniform discretisation (Section 2.3): sample points y_j
// (loaded, not generated) with element measures |P_j|, fused with the
// measure-weighted moments m_i = sum |P_j|, S1_i = sum |P_j| y_j,
// S2_i = sum |P_j| y_j y_j^T of each cell.
//
// One thread per point.  The seeds stream through shared memory in chunks of
// 256 FP32 direct-form records (coordinates and weights split into FP32 high
// and low parts).  Pass 1 takes the smallest FP32 cost plus its rounding bound
// over all seeds as a threshold; pass 2 recomputes every seed whose FP32 cost
// minus its bound lies below it in FP64 with the reference operation order, and
// the smallest FP64 cost wins (lowest index on ties): the label equals the
// FP64 argmin over all seeds (the rescoring argument of the grid path).  The
// moments are FP64 sums accumulated with atomics (their rounding depends on
// the order of the additions).
#include <algorithm>

#include "apd_common.cuh"
#include "apd_cost.cuh"

namespace apd {

namespace {

constexpr int kPtThreads = 256;

// FP32 direct-form records and the reference weight of the seeds.
template <int D>
__global__ void points_prep_kernel(const int n, const double *__restrict__ x, const double *__restrict__ A,
                                   const double *__restrict__ w, SeedRec32 *__restrict__ r32,
                                   DevScalars *__restrict__ sc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    SeedRec r;
    SeedRec32 q;
    double wkey, frob, lam;
    int bad;
    build_seed<D>(i, n, x, A, w, r, q, wkey, frob, lam, bad);
    if (i < n) {
        r32[i] = q;
        if (bad) atomicOr(&sc->status, bad);
    }
    const double wmax = warp_max(i < n ? wkey : -DBL_MAX);
    const bool any = __any_sync(0xffffffffu, i < n);
    if ((threadIdx.x & 31) == 0 && any) atomicMax(&sc->wref_key, dkey(wmax));
}

template <int D>
__global__ void __launch_bounds__(kPtThreads)
    points_assign_kernel(const long long count, const double *__restrict__ y, const double *__restrict__ mass,
                         const int n, const double *__restrict__ x, const double *__restrict__ A,
                         const double *__restrict__ w, const SeedRec32 *__restrict__ r32,
                         DevScalars *__restrict__ sc, double *__restrict__ mom, int32_t *__restrict__ labels) {
    constexpr int K = moment_width(D);
    __shared__ SeedRec32 sr[kPtThreads];
    const double wref = dkey_inv(sc->wref_key);
    float wrh, wrl;
    split_f32(wref, wrh, wrl);
    for (long long j0 = (long long)blockIdx.x * kPtThreads; j0 < count; j0 += (long long)gridDim.x * kPtThreads) {
        const long long j = j0 + threadIdx.x;
        const bool active = j < count;
        double yy[D];
        float yh[3] = {0.f, 0.f, 0.f}, yl[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int a = 0; a < D; ++a) {
            yy[a] = active ? y[j * D + a] : 0.0;
            split_f32(yy[a], yh[a], yl[a]);
        }
        // pass 1: threshold = min_k (C_k + E_k)
        float thr = __int_as_float(0x7f800000);
        for (int c0 = 0; c0 < n; c0 += kPtThreads) {
            const int m = min(kPtThreads, n - c0);
            __syncthreads();
            if ((int)threadIdx.x < m) sr[threadIdx.x] = r32[c0 + threadIdx.x];
            __syncthreads();
            for (int k = 0; k < m; ++k) {
                float c, E;
                cost32_bound<D>(sr[k], yh, yl, wrh, wrl, c, E);
                thr = fminf(thr, c + E);
            }
        }
        // pass 2: FP64 reference cost of the candidates
        double best = __longlong_as_double(0x7ff0000000000000ll);
        int bi = 0x7fffffff;
        for (int c0 = 0; c0 < n; c0 += kPtThreads) {
            const int m = min(kPtThreads, n - c0);
            __syncthreads();
            if ((int)threadIdx.x < m) sr[threadIdx.x] = r32[c0 + threadIdx.x];
            __syncthreads();
            if (!active) continue;
            for (int k = 0; k < m; ++k) {
                float c, E;
                cost32_bound<D>(sr[k], yh, yl, wrh, wrl, c, E);
                if (!(c - E <= thr)) continue;
                const int s = c0 + k;
                const double c64 = cost64<D>(yy, x + (size_t)s * D, A + (size_t)s * D * D, w[s]);
                if (c64 < best || (c64 == best && s < bi)) {
                    best = c64;
                    bi = s;
                }
            }
        }
        if (!active) continue;
        if (bi < 0 || bi >= n) {
            atomicOr(&sc->status, ST_BAD_LABEL);
            continue;
        }
        if (labels) labels[j] = bi;
        const double mj = mass[j];
        double *o = mom + (size_t)bi * K;
        atomicAdd(&o[0], mj);
#pragma unroll
        for (int a = 0; a < D; ++a) atomicAdd(&o[1 + a], mj * yy[a]);
        int e = 1 + D;
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
            for (int b = a; b < D; ++b) atomicAdd(&o[e++], mj * yy[a] * yy[b]);
    }
}

}  // namespace

cudaError_t launch_points_assign(int dim, long long count, const double *y, const double *mass, int n,
                                 const double *x, const double *A, const double *w, double *mom,
                                 int32_t *labels, Workspace &ws, cudaStream_t st) {
    const int K = moment_width(dim);
    cudaError_t e = cudaMemsetAsync(mom, 0, (size_t)n * K * sizeof(double), st);
    if (e != cudaSuccess) return e;
    e = launch_eval_reset(ws, st, false);
    if (e != cudaSuccess) return e;
    const int pb = (n + 255) / 256;
    if (dim == 3) points_prep_kernel<3><<<pb, 256, 0, st>>>(n, x, A, w, ws.recs32, ws.sc);
    else points_prep_kernel<2><<<pb, 256, 0, st>>>(n, x, A, w, ws.recs32, ws.sc);
    const int sms = ws.sms;
    const long long want = (count + kPtThreads - 1) / kPtThreads;
    const int blocks = (int)std::min<long long>(want, (long long)sms * 8);
    if (dim == 3)
        points_assign_kernel<3><<<blocks, kPtThreads, 0, st>>>(count, y, mass, n, x, A, w, ws.recs32, ws.sc, mom,
                                                               labels);
    else
        points_assign_kernel<2><<<blocks, kPtThreads, 0, st>>>(count, y, mass, n, x, A, w, ws.recs32, ws.sc, mom,
                                                               labels);
    return cudaGetLastError();
}

}  // namespace apd
