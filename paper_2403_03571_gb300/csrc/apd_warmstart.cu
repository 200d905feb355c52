// Learned warm start of the weight solve: a per-seed MLP predicts initial
// weights from local statistics of the generators, trained on solved instances.
//
// Features of seed i of an instance with n seeds on the box [lo, hi] of
// measure |O| (F = 28 in 2D, 32 in 3D), with s = n / |O| the seed density and
// lengths in units of the mean spacing s^(-1/D):
//   [ v_i s,  the upper triangle of (A_i + A_i^T) / 2 (3 or 6 entries),
//     the distances to the 8 nearest other seeds (ascending),
//     the target volumes of those 8 seeds times s,
//     the distance to the nearer wall along each axis (D entries),
//     for the radii r = 2, 4, 8: c_r / E_r and (V_r s - c_r) / E_r, where c_r
//     counts the other seeds within r, V_r sums their target volumes and
//     E_r = w_D r^D is the expected count (w_D the unit-ball volume) ]
// The first four groups describe the seed and its nearest neighbours; the wall
// distances and the volume/count mismatch at three scales carry what a cell's
// weight needs from farther away (the solved weights vary smoothly over many
// cells, driven by the boundary and by the local excess of target volume).
// Network: F -> 64 -> 64 -> 64 -> 1, ReLU on the hidden layers, inputs
// standardised by a stored mean / standard deviation.  The output y_i is a
// weight in units of the mean cell size squared: w_i = y_i s^(-2/D).
// Weights are determined only up to a common constant (the gauge of the
// dual); training targets are therefore centred per instance.
//
// Kernels: brute-force k-nearest-neighbour features, inference, a training
// step (forward, backward by hand, per-CTA gradient partials summed in a fixed
// order by the Adam kernel), and the input statistics.  All FP32 except the
// neighbour distances (FP64) and the statistic sums (FP64).
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "apd_common.cuh"

namespace apd {
namespace {

constexpr int kH = 64;       // hidden width
constexpr int kNN = 8;       // neighbours per seed
constexpr int kTrainB = 128; // samples (threads) per CTA of the network kernels

constexpr int kRadii = 3;    // neighbourhood radii 2, 4, 8 (mean spacings)
__host__ __device__ constexpr int feat_dim(int D) { return 1 + D * (D + 1) / 2 + 2 * kNN + D + 2 * kRadii; }
static_assert(feat_dim(3) == kWarmFeatMax, "workspace feature scratch");
constexpr int F2 = feat_dim(2), F3 = feat_dim(3);
__host__ __device__ constexpr int param_count(int F) { return kH * F + kH + 2 * (kH * kH + kH) + kH + 1; }

// parameter offsets in the flat FP32 array: W1 [64][F], b1, W2 [64][64], b2, W3, b3, W4 [64], b4
struct Layout {
    int F, w1, b1, w2, b2, w3, b3, w4, b4, P;
    __host__ __device__ constexpr Layout(int f)
        : F(f), w1(0), b1(kH * f), w2(kH * f + kH), b2(kH * f + kH + kH * kH), w3(kH * f + 2 * kH + kH * kH),
          b3(kH * f + 2 * kH + 2 * kH * kH), w4(kH * f + 3 * kH + 2 * kH * kH), b4(kH * f + 4 * kH + 2 * kH * kH),
          P(param_count(f)) {}
};

// ---------------------------------------------------------------------------
// features: one thread per seed, brute-force 8 nearest neighbours
// ---------------------------------------------------------------------------
// One warp per seed: the lanes scan the other seeds of the instance (FP64
// distances), each keeping its 8 nearest in order and its partial ball counts;
// the 8 nearest of the seed are then drawn from the lanes' lists in the order
// (distance, index), which is also the order of the sequential scan (ties keep
// the lower index first).
template <int D>
__global__ void __launch_bounds__(256)
    features_kernel(const int count, const long long *__restrict__ offs, const double *__restrict__ box,
                    const double *__restrict__ x, const double *__restrict__ A, const double *__restrict__ v,
                    float *__restrict__ feat, int32_t *__restrict__ knn) {
    constexpr int F = feat_dim(D);
    const long long total = offs[count];
    const long long gi = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gi >= total) return;  // whole warps leave together
    int lo = 0, hi = count - 1;  // instance: last b with offs[b] <= gi
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (offs[mid] <= gi) lo = mid;
        else hi = mid - 1;
    }
    const long long o = offs[lo];
    const int n = (int)(offs[lo + 1] - o);
    const double *bx = box + (size_t)lo * 6;  // lo[3], hi[3]
    double meas = 1.0;
#pragma unroll
    for (int a = 0; a < D; ++a) meas *= bx[3 + a] - bx[a];
    const double dens = (double)n / meas;
    const double ls = pow(dens, 1.0 / D);      // 1 / mean spacing
    double xi[D];
#pragma unroll
    for (int a = 0; a < D; ++a) xi[a] = x[gi * D + a];
    double rad2[kRadii], cnt[kRadii], vsum[kRadii];
#pragma unroll
    for (int r = 0; r < kRadii; ++r) {
        const double rr = (double)(2 << r) / ls;
        rad2[r] = rr * rr;
        cnt[r] = 0.0;
        vsum[r] = 0.0;
    }
    double bd[kNN];
    int bj[kNN];
#pragma unroll
    for (int k = 0; k < kNN; ++k) {
        bd[k] = 1e300;
        bj[k] = -1;
    }
    for (int j = lane; j < n; j += 32) {
        if (o + j == gi) continue;
        double d2 = 0.0;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const double t = x[(o + j) * D + a] - xi[a];
            d2 += t * t;
        }
#pragma unroll
        for (int r = 0; r < kRadii; ++r)
            if (d2 < rad2[r]) {
                cnt[r] += 1.0;
                vsum[r] += v[o + j];
            }
        if (d2 < bd[kNN - 1]) {  // insertion into the lane's sorted list (j increases along the scan)
#pragma unroll
            for (int p = kNN - 1; p > 0; --p) {
                const bool shift = bd[p - 1] > d2;
                const bool here = !shift && bd[p] > d2;
                bd[p] = shift ? bd[p - 1] : (here ? d2 : bd[p]);
                bj[p] = shift ? bj[p - 1] : (here ? j : bj[p]);
            }
            if (bd[0] > d2) {
                bd[0] = d2;
                bj[0] = j;
            }
        }
    }
#pragma unroll
    for (int r = 0; r < kRadii; ++r) {
        cnt[r] = warp_sum(cnt[r]);
        vsum[r] = warp_sum(vsum[r]);
    }
    // merge: 8 rounds of the smallest (distance, index) head over the lanes
    double fd[kNN];
    int fj[kNN];
#pragma unroll
    for (int k = 0; k < kNN; ++k) {
        double md = bd[0];
        int mj = bj[0] < 0 ? 0x7fffffff : bj[0];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const double od = __shfl_xor_sync(0xffffffffu, md, off);
            const int oj = __shfl_xor_sync(0xffffffffu, mj, off);
            if (od < md || (od == md && oj < mj)) {
                md = od;
                mj = oj;
            }
        }
        const bool mine = (bd[0] == md) && ((bj[0] < 0 ? 0x7fffffff : bj[0]) == mj);
        fd[k] = md;
        fj[k] = mj == 0x7fffffff ? -1 : mj;
        if (mine && mj != 0x7fffffff) {  // pop the head
#pragma unroll
            for (int p = 0; p < kNN - 1; ++p) {
                bd[p] = bd[p + 1];
                bj[p] = bj[p + 1];
            }
            bd[kNN - 1] = 1e300;
            bj[kNN - 1] = -1;
        }
    }
    if (lane != 0) return;
    if (knn) {
#pragma unroll
        for (int k = 0; k < kNN; ++k) knn[gi * kNN + k] = fj[k] >= 0 ? (int32_t)(o + fj[k]) : -1;
    }
    float *f = feat + gi * F;
    int c = 0;
    f[c++] = (float)(v[gi] * dens);
    const double *Ai = A + gi * D * D;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = a; b < D; ++b) f[c++] = (float)(0.5 * (Ai[a * D + b] + Ai[b * D + a]));
#pragma unroll
    for (int k = 0; k < kNN; ++k) f[c + k] = fj[k] >= 0 ? (float)(sqrt(fd[k]) * ls) : 4.f;
#pragma unroll
    for (int k = 0; k < kNN; ++k) f[c + kNN + k] = fj[k] >= 0 ? (float)(v[o + fj[k]] * dens) : 0.f;
    c += 2 * kNN;
#pragma unroll
    for (int a = 0; a < D; ++a) f[c++] = (float)(fmin(xi[a] - bx[a], bx[3 + a] - xi[a]) * ls);
    const double wD = D == 2 ? 3.14159265358979323846 : 4.18879020478639098461;  // unit-ball volume
#pragma unroll
    for (int r = 0; r < kRadii; ++r) {
        const double e = wD * (double)((2 << r) * (2 << r) * (D == 3 ? (2 << r) : 1));
        f[c++] = (float)(cnt[r] / e);
        f[c++] = (float)((vsum[r] * dens - cnt[r]) / e);
    }
}

// ---------------------------------------------------------------------------
// network evaluation (one sample per thread; weights and the thread's
// activation rows in shared memory, rows padded to avoid bank conflicts)
// ---------------------------------------------------------------------------
constexpr int kRow = kH + 1;

template <int F>
struct Rows {
    float x[kTrainB][F + 1];
    float h1[kTrainB][kRow];
    float h2[kTrainB][kRow];
    float h3[kTrainB][kRow];
    float d[kTrainB][kRow];   // delta of the layer being back-propagated
    float dy[kTrainB];
    float loss[kTrainB];
};

template <int F>
constexpr size_t rows_offset() {  // floats before the rows: parameters, then mean / inverse std
    return ((size_t)param_count(F) + 2 * F + 3) & ~(size_t)3;
}
template <int F>
constexpr size_t net_smem() {
    return rows_offset<F>() * sizeof(float) + sizeof(Rows<F>);
}

template <int F>
__device__ __forceinline__ void load_net(float *sp, const float *__restrict__ params, const float *__restrict__ norm) {
    constexpr int P = param_count(F);
    for (int k = threadIdx.x; k < P; k += blockDim.x) sp[k] = params[k];
    for (int k = threadIdx.x; k < 2 * F; k += blockDim.x) sp[P + k] = norm[k];
}

// out[j] = relu(b[j] + sum_k W[j][k] in[k]) for the calling thread's rows
__device__ __forceinline__ void dense_relu(const float *sp, int w, int bo, int in_dim, const float *in, float *out) {
    for (int j = 0; j < kH; ++j) {
        float acc = sp[bo + j];
        const float *wr = sp + w + j * in_dim;
#pragma unroll 8
        for (int k = 0; k < in_dim; ++k) acc = fmaf(wr[k], in[k], acc);
        out[j] = fmaxf(acc, 0.f);
    }
}

// standardised input of sample s into the thread's x row, then the forward pass
template <int F>
__device__ __forceinline__ float forward(const float *sp, Rows<F> &R, int t, const float *__restrict__ feat,
                                         long long s) {
    constexpr Layout L(F);
    const float *mean = sp + L.P, *istd = sp + L.P + F;
#pragma unroll
    for (int k = 0; k < F; ++k) R.x[t][k] = (feat[s * F + k] - mean[k]) * istd[k];
    dense_relu(sp, L.w1, L.b1, F, R.x[t], R.h1[t]);
    dense_relu(sp, L.w2, L.b2, kH, R.h1[t], R.h2[t]);
    dense_relu(sp, L.w3, L.b3, kH, R.h2[t], R.h3[t]);
    float y = sp[L.b4];
    for (int k = 0; k < kH; ++k) y = fmaf(sp[L.w4 + k], R.h3[t][k], y);
    return y;
}

// W_pred of every seed: y_i s^(-2/D), s = n_b / |O_b|
template <int D>
__global__ void __launch_bounds__(kTrainB)
    predict_kernel(const int count, const long long *__restrict__ offs, const double *__restrict__ box,
                   const float *__restrict__ params, const float *__restrict__ norm, const float *__restrict__ feat,
                   double *__restrict__ w_out) {
    constexpr int F = feat_dim(D);
    extern __shared__ float sp[];
    Rows<F> &R = *reinterpret_cast<Rows<F> *>(sp + rows_offset<F>());
    load_net<F>(sp, params, norm);
    __syncthreads();
    const long long total = offs[count];
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= total) return;
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (offs[mid] <= s) lo = mid;
        else hi = mid - 1;
    }
    const int n = (int)(offs[lo + 1] - offs[lo]);
    double meas = 1.0;
#pragma unroll
    for (int a = 0; a < D; ++a) meas *= box[(size_t)lo * 6 + 3 + a] - box[(size_t)lo * 6 + a];
    const float y = forward<F>(sp, R, threadIdx.x, feat, s);
    w_out[s] = (double)y * pow((double)n / meas, -2.0 / D);
}

// ---------------------------------------------------------------------------
// training: loss = (1/B) sum_s (y_s - t_s)^2 over the batch idx[0 .. B)
// ---------------------------------------------------------------------------
// One CTA = kTrainB samples, forward as above, then backward layer by layer:
//   dy = 2 (y - t) / B;  gW4 = sum dy h3, gb4 = sum dy
//   d3 = dy W4 . [h3 > 0];  gW3 = sum d3 h2^T, gb3 = sum d3
//   d2 = W3^T d3 . [h2 > 0];  gW2 = sum d2 h1^T, gb2 = sum d2
//   d1 = W2^T d2 . [h1 > 0];  gW1 = sum d1 x^T,  gb1 = sum d1
// The CTA's gradient goes to part[blockIdx.x][P]; the Adam kernel sums the
// partials in CTA order (deterministic).
__device__ __forceinline__ void grad_outer(const float (*dl)[kRow], const float *hin, int hstride, int in_dim,
                                           int nvalid, float *gw, float *gb) {
    // gW[j][k] = sum_s d[s][j] hin[s][k]; thread t takes entries t, t + blockDim, ...
    for (int e = threadIdx.x; e < kH * in_dim; e += blockDim.x) {
        const int j = e / in_dim, k = e % in_dim;
        float acc = 0.f;
        for (int s = 0; s < nvalid; ++s) acc = fmaf(dl[s][j], hin[s * hstride + k], acc);
        gw[e] = acc;
    }
    for (int j = threadIdx.x; j < kH; j += blockDim.x) {
        float acc = 0.f;
        for (int s = 0; s < nvalid; ++s) acc += dl[s][j];
        gb[j] = acc;
    }
}

// d_new[k] = [h[k] > 0] sum_j W[j][k] d[j] for the calling thread's row (W [64][64])
__device__ __forceinline__ void back_hidden(const float *sp, int w, const float *h, float *d) {
    float nd[kH];
    for (int k = 0; k < kH; ++k) {
        float acc = 0.f;
#pragma unroll 8
        for (int j = 0; j < kH; ++j) acc = fmaf(sp[w + j * kH + k], d[j], acc);
        nd[k] = h[k] > 0.f ? acc : 0.f;
    }
#pragma unroll
    for (int k = 0; k < kH; ++k) d[k] = nd[k];
}

template <int F>
__global__ void __launch_bounds__(kTrainB)
    train_grad_kernel(const int B, const int *__restrict__ idx, const float *__restrict__ params,
                      const float *__restrict__ norm, const float *__restrict__ feat, const float *__restrict__ target,
                      const float *__restrict__ dy_in, float *__restrict__ part, float *__restrict__ loss_part) {
    constexpr Layout L(F);
    extern __shared__ float sp[];
    Rows<F> &R = *reinterpret_cast<Rows<F> *>(sp + rows_offset<F>());
    load_net<F>(sp, params, norm);
    __syncthreads();
    const int t = threadIdx.x;
    const int s0 = blockIdx.x * kTrainB;
    const int nvalid = min(kTrainB, B - s0);
    float *gp = part + (size_t)blockIdx.x * L.P;
    if (t < nvalid) {
        const long long s = idx[s0 + t];
        const float y = forward<F>(sp, R, t, feat, s);
        if (dy_in) {  // loss gradient supplied (neighbour-difference loss)
            R.dy[t] = dy_in[s];
            R.loss[t] = 0.f;
        } else {
            const float r = y - target[s];
            R.dy[t] = 2.f * r / (float)B;
            R.loss[t] = r * r;
        }
    } else {  // rows of absent samples contribute nothing
        for (int k = 0; k <= F; ++k) R.x[t][k] = 0.f;
        for (int k = 0; k < kRow; ++k) R.h1[t][k] = R.h2[t][k] = R.h3[t][k] = 0.f;
        R.dy[t] = 0.f;
        R.loss[t] = 0.f;
    }
    // d3 = dy W4 . [h3 > 0]
    for (int j = 0; j < kH; ++j) R.d[t][j] = R.h3[t][j] > 0.f ? R.dy[t] * sp[L.w4 + j] : 0.f;
    __syncthreads();
    for (int k = t; k < kH; k += blockDim.x) {
        float acc = 0.f;
        for (int s = 0; s < nvalid; ++s) acc = fmaf(R.dy[s], R.h3[s][k], acc);
        gp[L.w4 + k] = acc;
    }
    if (t == 0) {
        float acc = 0.f, la = 0.f;
        for (int s = 0; s < nvalid; ++s) {
            acc += R.dy[s];
            la += R.loss[s];
        }
        gp[L.b4] = acc;
        loss_part[blockIdx.x] = la;
    }
    grad_outer(R.d, &R.h2[0][0], kRow, kH, nvalid, gp + L.w3, gp + L.b3);
    __syncthreads();
    back_hidden(sp, L.w3, R.h2[t], R.d[t]);
    __syncthreads();
    grad_outer(R.d, &R.h1[0][0], kRow, kH, nvalid, gp + L.w2, gp + L.b2);
    __syncthreads();
    back_hidden(sp, L.w2, R.h1[t], R.d[t]);
    __syncthreads();
    grad_outer(R.d, &R.x[0][0], F + 1, F, nvalid, gp + L.w1, gp + L.b1);
}

// Network outputs of the batch samples into y[s] (global sample index), and a
// zeroed loss gradient dy[s] for the pair kernel.
template <int F>
__global__ void __launch_bounds__(kTrainB)
    forward_batch_kernel(const int B, const int *__restrict__ idx, const float *__restrict__ params,
                         const float *__restrict__ norm, const float *__restrict__ feat, float *__restrict__ y,
                         float *__restrict__ dy) {
    extern __shared__ float sp[];
    Rows<F> &R = *reinterpret_cast<Rows<F> *>(sp + rows_offset<F>());
    load_net<F>(sp, params, norm);
    __syncthreads();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const long long s = idx[b];
    y[s] = forward<F>(sp, R, threadIdx.x, feat, s);
    dy[s] = 0.f;
}

// Neighbour-difference loss over the batch's (i, j in kNN(i)) pairs plus a
// small squared-error anchor,
//   L = (1/(8B)) sum ((y_i - y_j) - (t_i - t_j))^2 + (mu/B) sum (y_i - t_i)^2,
// and its gradient with respect to the outputs (scattered with atomics; every
// neighbour of a batch sample must be in the batch, e.g. whole instances).
__global__ void pair_loss_kernel(const int B, const int *__restrict__ idx, const int32_t *__restrict__ knn,
                                 const float *__restrict__ y, const float *__restrict__ target, const float inv_pairs,
                                 const float mu, float *__restrict__ dy, float *__restrict__ loss) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.f;
    if (b < B) {
        const long long i = idx[b];
        const float e = y[i] - target[i];
        float gi = 2.f * mu * e / (float)B;
        l = mu * e * e * (float)kNN;  // scaled back by inv_pairs below
#pragma unroll
        for (int k = 0; k < kNN; ++k) {
            const int j = knn[i * kNN + k];
            if (j < 0) continue;
            const float r = (y[i] - y[j]) - (target[i] - target[j]);
            l += r * r;
            gi += 2.f * r * inv_pairs;
            atomicAdd(&dy[j], -2.f * r * inv_pairs);
        }
        atomicAdd(&dy[i], gi);
    }
    l *= inv_pairs;
    // block sum of the loss, one atomic per block
    __shared__ float sh[32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) l += __shfl_xor_sync(0xffffffffu, l, off);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        atomicAdd(loss, t);
    }
}

// Sum of the CTA partials (fixed order) -> grad (optional) and an Adam step
// (optional, lr > 0): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
// p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + 1e-8).
__global__ void adam_kernel(const int P, const int nparts, const float *__restrict__ part,
                            const float *__restrict__ loss_part, float *__restrict__ params, float *__restrict__ m,
                            float *__restrict__ v, const float lr, const float bc1, const float bc2,
                            float *__restrict__ grad_out, float *__restrict__ loss_out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0 && loss_out) {
        double l = 0.0;
        for (int b = 0; b < nparts; ++b) l += (double)loss_part[b];
        *loss_out = (float)l;
    }
    if (p >= P) return;
    float g = 0.f;
    for (int b = 0; b < nparts; ++b) g += part[(size_t)b * P + p];
    if (grad_out) grad_out[p] = g;
    if (lr > 0.f) {
        const float mm = 0.9f * m[p] + 0.1f * g;
        const float vv = 0.999f * v[p] + 0.001f * g * g;
        m[p] = mm;
        v[p] = vv;
        params[p] -= lr * (mm / bc1) / (sqrtf(vv / bc2) + 1e-8f);
    }
}

// per-feature mean and 1 / std over S samples (FP64 sums, one CTA per feature)
__global__ void __launch_bounds__(256)
    norm_kernel(const long long S, const int F, const float *__restrict__ feat, float *__restrict__ norm) {
    __shared__ double sh[33];
    const int k = blockIdx.x;
    double s1 = 0.0, s2 = 0.0;
    for (long long s = threadIdx.x; s < S; s += blockDim.x) {
        const double f = feat[s * F + k];
        s1 += f;
        s2 += f * f;
    }
    s1 = block_sum(s1, sh);
    s2 = block_sum(s2, sh);
    if (threadIdx.x == 0) {
        const double mean = s1 / (double)S;
        const double var = fmax(s2 / (double)S - mean * mean, 0.0);
        norm[k] = (float)mean;
        norm[F + k] = (float)(1.0 / sqrt(var + 1e-12));
    }
}

}  // namespace
}  // namespace apd

using namespace apd;

struct apd_mlp {
    int dim = 0, F = 0, P = 0;
    float *params = nullptr, *m = nullptr, *v = nullptr, *norm = nullptr;
    float *part = nullptr, *loss_part = nullptr;
    int part_cap = 0;  // CTAs the partial buffer holds
    long long *offs = nullptr;
    double *box = nullptr;   // [inst_cap][6] instance boxes (lo, hi)
    float *pair_loss = nullptr;  // loss sink of the pair kernel when the caller wants none
    int inst_cap = 0;
    int step = 0;
};

namespace apd {
int warmstart_dim(const apd_mlp *net) { return net ? net->dim : 0; }
}  // namespace apd

namespace {

int ws_rc(cudaError_t e) { return e == cudaSuccess ? APD_OK : APD_ERR_CUDA; }

int ensure_instances(apd_mlp *net, int count, const int64_t *offsets, const double *box, cudaStream_t st) {
    if (count > net->inst_cap) {
        if (net->offs) cudaFree(net->offs);
        if (net->box) cudaFree(net->box);
        net->offs = nullptr;
        net->box = nullptr;
        net->inst_cap = 0;
        if (cudaMalloc((void **)&net->offs, (size_t)(count + 1) * sizeof(long long)) != cudaSuccess ||
            cudaMalloc((void **)&net->box, (size_t)count * 6 * sizeof(double)) != cudaSuccess)
            return APD_ERR_CUDA;
        net->inst_cap = count;
    }
    // host arrays -> device (pageable copies are synchronous with respect to the host)
    if (cudaMemcpyAsync(net->offs, offsets, (size_t)(count + 1) * sizeof(long long), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(net->box, box, (size_t)count * 6 * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return APD_ERR_CUDA;
    return APD_OK;
}

int check_offsets(int dim, int count, const int64_t *offsets, const double *box) {
    if (count < 1 || !offsets || !box || offsets[0] != 0) return APD_ERR_ARG;
    for (int b = 0; b < count; ++b) {
        if (offsets[b + 1] <= offsets[b]) return APD_ERR_ARG;
        for (int a = 0; a < dim; ++a)
            if (!(box[6 * b + 3 + a] > box[6 * b + a]) || !std::isfinite(box[6 * b + a]) ||
                !std::isfinite(box[6 * b + 3 + a]))
                return APD_ERR_ARG;
    }
    return APD_OK;
}

}  // namespace

extern "C" {

int apd_warmstart_create(apd_mlp **out, int32_t dim, const float *params, const float *norm) {
    if (!out) return APD_ERR_ARG;
    *out = nullptr;
    if ((dim != 2 && dim != 3) || !params) return APD_ERR_ARG;
    apd_mlp *net = new (std::nothrow) apd_mlp();
    if (!net) return APD_ERR_CUDA;
    net->dim = dim;
    net->F = feat_dim(dim);
    net->P = param_count(net->F);
    const size_t P = (size_t)net->P, F = (size_t)net->F;
    bool ok = cudaMalloc((void **)&net->params, P * sizeof(float)) == cudaSuccess &&
              cudaMalloc((void **)&net->m, P * sizeof(float)) == cudaSuccess &&
              cudaMalloc((void **)&net->v, P * sizeof(float)) == cudaSuccess &&
              cudaMalloc((void **)&net->norm, 2 * F * sizeof(float)) == cudaSuccess;
    std::vector<float> nz(2 * F);
    for (size_t k = 0; k < F; ++k) {
        nz[k] = norm ? norm[k] : 0.f;
        nz[F + k] = norm ? norm[F + k] : 1.f;
    }
    ok = ok && cudaMemcpy(net->params, params, P * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(net->norm, nz.data(), 2 * F * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemset(net->m, 0, P * sizeof(float)) == cudaSuccess &&
         cudaMemset(net->v, 0, P * sizeof(float)) == cudaSuccess;
    if (ok && dim == 2)
        ok = cudaFuncSetAttribute(predict_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)net_smem<F2>()) == cudaSuccess &&
             cudaFuncSetAttribute(forward_batch_kernel<F2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)net_smem<F2>()) == cudaSuccess &&
             cudaFuncSetAttribute(train_grad_kernel<F2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)net_smem<F2>()) == cudaSuccess;
    if (ok && dim == 3)
        ok = cudaFuncSetAttribute(predict_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)net_smem<F3>()) == cudaSuccess &&
             cudaFuncSetAttribute(forward_batch_kernel<F3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)net_smem<F3>()) == cudaSuccess &&
             cudaFuncSetAttribute(train_grad_kernel<F3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)net_smem<F3>()) == cudaSuccess;
    if (!ok) {
        apd_warmstart_destroy(net);
        return APD_ERR_CUDA;
    }
    *out = net;
    return APD_OK;
}

void apd_warmstart_destroy(apd_mlp *net) {
    if (!net) return;
    void *ptrs[] = {net->params, net->m, net->v, net->norm, net->part, net->loss_part, net->offs, net->box,
                    net->pair_loss};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete net;
}

int32_t apd_warmstart_sizes(int32_t dim, int32_t *n_features, int32_t *n_params) {
    if (dim != 2 && dim != 3) return APD_ERR_ARG;
    if (n_features) *n_features = feat_dim(dim);
    if (n_params) *n_params = param_count(feat_dim(dim));
    return APD_OK;
}

int apd_warmstart_get(apd_mlp *net, float *params, float *norm) {
    if (!net) return APD_ERR_ARG;
    if (params && cudaMemcpy(params, net->params, (size_t)net->P * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
        return APD_ERR_CUDA;
    if (norm && cudaMemcpy(norm, net->norm, 2 * (size_t)net->F * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
        return APD_ERR_CUDA;
    return APD_OK;
}

int apd_warmstart_features(apd_mlp *net, int32_t count, const int64_t *offsets, const double *box,
                           const double *x, const double *A, const double *v, float *features, int32_t *knn,
                           apd_stream_t stream) {
    if (!net || !x || !A || !v || !features) return APD_ERR_ARG;
    int rc = check_offsets(net->dim, count, offsets, box);
    if (rc != APD_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    rc = ensure_instances(net, count, offsets, box, st);
    if (rc != APD_OK) return rc;
    const long long total = offsets[count];
    const int blocks = (int)((total + 7) / 8);  // one warp per seed
    if (net->dim == 2)
        features_kernel<2><<<blocks, 256, 0, st>>>(count, net->offs, net->box, x, A, v, features, knn);
    else
        features_kernel<3><<<blocks, 256, 0, st>>>(count, net->offs, net->box, x, A, v, features, knn);
    return ws_rc(cudaGetLastError());
}

int apd_warmstart_fit_norm(apd_mlp *net, int64_t samples, const float *features, apd_stream_t stream) {
    if (!net || samples < 2 || !features) return APD_ERR_ARG;
    norm_kernel<<<net->F, 256, 0, (cudaStream_t)stream>>>(samples, net->F, features, net->norm);
    return ws_rc(cudaGetLastError());
}

int apd_warmstart_predict(apd_mlp *net, int32_t count, const int64_t *offsets, const double *box,
                          const float *features, double *w_out, apd_stream_t stream) {
    if (!net || !features || !w_out) return APD_ERR_ARG;
    int rc = check_offsets(net->dim, count, offsets, box);
    if (rc != APD_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    rc = ensure_instances(net, count, offsets, box, st);
    if (rc != APD_OK) return rc;
    const long long total = offsets[count];
    const int blocks = (int)((total + kTrainB - 1) / kTrainB);
    if (net->dim == 2)
        predict_kernel<2><<<blocks, kTrainB, net_smem<F2>(), st>>>(count, net->offs, net->box, net->params,
                                                                    net->norm, features, w_out);
    else
        predict_kernel<3><<<blocks, kTrainB, net_smem<F3>(), st>>>(count, net->offs, net->box, net->params,
                                                                    net->norm, features, w_out);
    return ws_rc(cudaGetLastError());
}

static int train_step_impl(apd_mlp *net, int32_t batch, const int32_t *idx, const float *features,
                           const float *targets, const float *dy_in, float lr, float *grad_out, float *loss_out,
                           cudaStream_t st) {
    const int nparts = (batch + kTrainB - 1) / kTrainB;
    if (nparts > net->part_cap) {
        if (net->part) cudaFree(net->part);
        if (net->loss_part) cudaFree(net->loss_part);
        net->part = nullptr;
        net->loss_part = nullptr;
        net->part_cap = 0;
        if (cudaMalloc((void **)&net->part, (size_t)nparts * net->P * sizeof(float)) != cudaSuccess ||
            cudaMalloc((void **)&net->loss_part, (size_t)nparts * sizeof(float)) != cudaSuccess)
            return APD_ERR_CUDA;
        net->part_cap = nparts;
    }
    const size_t smem = net->F == F2 ? net_smem<F2>() : net_smem<F3>();
    if (net->F == F2)
        train_grad_kernel<F2><<<nparts, kTrainB, smem, st>>>(batch, idx, net->params, net->norm, features, targets,
                                                             dy_in, net->part, net->loss_part);
    else
        train_grad_kernel<F3><<<nparts, kTrainB, smem, st>>>(batch, idx, net->params, net->norm, features, targets,
                                                             dy_in, net->part, net->loss_part);
    float bc1 = 1.f, bc2 = 1.f;
    if (lr > 0.f) {
        net->step += 1;
        bc1 = 1.f - powf(0.9f, (float)net->step);
        bc2 = 1.f - powf(0.999f, (float)net->step);
    }
    adam_kernel<<<(net->P + 255) / 256, 256, 0, st>>>(net->P, nparts, net->part, net->loss_part, net->params, net->m,
                                                      net->v, lr, bc1, bc2, grad_out, loss_out);
    return ws_rc(cudaGetLastError());
}

int apd_warmstart_train_step(apd_mlp *net, int32_t batch, const int32_t *idx, const float *features,
                             const float *targets, float lr, float *grad_out, float *loss_out, apd_stream_t stream) {
    if (!net || batch < 1 || !idx || !features || !targets || !(lr >= 0.f)) return APD_ERR_ARG;
    return train_step_impl(net, batch, idx, features, targets, nullptr, lr, grad_out, loss_out, (cudaStream_t)stream);
}

int apd_warmstart_train_step_pairs(apd_mlp *net, int32_t batch, const int32_t *idx, const float *features,
                                   const float *targets, const int32_t *knn, float *y_buf, float *dy_buf, float mu,
                                   float lr, float *grad_out, float *loss_out, apd_stream_t stream) {
    if (!net || batch < 1 || !idx || !features || !targets || !knn || !y_buf || !dy_buf || !(lr >= 0.f) ||
        !(mu >= 0.f))
        return APD_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int blocks = (batch + kTrainB - 1) / kTrainB;
    if (net->F == F2)
        forward_batch_kernel<F2><<<blocks, kTrainB, net_smem<F2>(), st>>>(batch, idx, net->params, net->norm,
                                                                           features, y_buf, dy_buf);
    else
        forward_batch_kernel<F3><<<blocks, kTrainB, net_smem<F3>(), st>>>(batch, idx, net->params, net->norm,
                                                                           features, y_buf, dy_buf);
    if (loss_out && cudaMemsetAsync(loss_out, 0, sizeof(float), st) != cudaSuccess) return APD_ERR_CUDA;
    if (!net->pair_loss && cudaMalloc((void **)&net->pair_loss, sizeof(float)) != cudaSuccess) return APD_ERR_CUDA;
    pair_loss_kernel<<<(batch + 255) / 256, 256, 0, st>>>(batch, idx, knn, y_buf, targets,
                                                          1.f / ((float)batch * (float)kNN), mu, dy_buf,
                                                          loss_out ? loss_out : net->pair_loss);
    const int rc = ws_rc(cudaGetLastError());
    if (rc != APD_OK) return rc;
    return train_step_impl(net, batch, idx, features, targets, dy_buf, lr, grad_out, nullptr, st);
}

}  // extern "C"
