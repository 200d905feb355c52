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
// Moments.  Each thread run-length encodes its row (neighbouring pixels share a
// label), accumulates count, sum u and sum u u^T (u = 2k + 1) per run, and adds
// runs into a per-CTA shared-memory hash table keyed by label; the table is
// flushed to the global int64 moments with one atomic per (cell, word).
#include <float.h>

#include "apd_internal.cuh"
#include "apd_cost.cuh"

namespace apd {

namespace {

constexpr float kUnit = 5.9604644775390625e-8f;  // 2^-24, unit roundoff of FP32
// Rounding-bound multiplier: about 24 roundings of size <= u T in the cost
// chain plus <= 62 u |C| from the packed 5-bit index, with a 1.8x margin.
constexpr float kKappa = 160.f;
constexpr int kTable = 128;  // shared-memory hash slots per CTA

template <int D>
struct Cfg;
template <>
struct Cfg<3> {
    static constexpr int P = 16, TY = 16, TZ = 16, NV = 3;
};
template <>
struct Cfg<2> {
    static constexpr int P = 16, TY = 256, TZ = 1, NV = 2;
};

__device__ __forceinline__ unsigned long long f2_bits(float2 v) {
    return (unsigned long long)__float_as_uint(v.x) | ((unsigned long long)__float_as_uint(v.y) << 32);
}
__device__ __forceinline__ float2 bits_f2(unsigned long long b) {
    return make_float2(__uint_as_float((unsigned)(b & 0xffffffffu)), __uint_as_float((unsigned)(b >> 32)));
}
// packed FP32x2 fused multiply-add: (a * b + c) elementwise
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)), "l"(f2_bits(c)));
    return bits_f2(r);
}
__device__ __forceinline__ float fmin3(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
// cost with the local seed index in the 5 low mantissa bits
__device__ __forceinline__ float pack(float c, unsigned idx) {
    return __uint_as_float((__float_as_uint(c) & ~31u) | idx);
}

// Row coefficients of two consecutive seeds (see the file comment), returned as
// duplicated pairs for the packed pixel-pair FMAs.  Every multiply is rounded on
// its own (no contraction), so the fast and update passes compute identical bits.
template <int D>
__device__ __forceinline__ void seed_pair_coeffs(const float4 (*phi)[kChunk], int s0, float f1, float f2,
                                                 float2 &qa, float2 &qb, float2 &ba, float2 &bbb,
                                                 float2 &aa2, float2 &ab2) {
    float a[2], bb[2], q00[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const float4 v0 = phi[0][s0 + e];
        const float4 v1 = phi[1][s0 + e];
        if (D == 3) {
            const float4 v2 = phi[2][s0 + e];
            const float d1 = __fsub_rn(f1, v0.x);
            const float d2 = __fsub_rn(f2, v0.y);
            const float e0 = fmaf(v1.z, d2, __fmul_rn(v1.y, d1));
            bb[e] = fmaf(2.f, e0, v1.w);
            const float t = fmaf(v0.w, d2, __fmul_rn(v0.z, d1));
            float aa = fmaf(d1, t, v2.x);
            aa = fmaf(v2.y, e0, aa);
            a[e] = fmaf(__fmul_rn(v1.x, d2), d2, aa);
            q00[e] = v2.z;
        } else {
            const float d1 = __fsub_rn(f1, v0.x);
            const float u1 = fmaf(v0.y, d1, v0.z);
            a[e] = fmaf(d1, u1, v0.w);
            bb[e] = fmaf(v1.y, d1, v1.x);
            q00[e] = v1.z;
        }
    }
    qa = make_float2(q00[0], q00[0]);
    qb = make_float2(q00[1], q00[1]);
    ba = make_float2(bb[0], bb[0]);
    bbb = make_float2(bb[1], bb[1]);
    aa2 = make_float2(a[0], a[0]);
    ab2 = make_float2(a[1], a[1]);
}

// Two new packed keys into the top-2 (b1 <= b2) of one pixel; gi follows b1.
__device__ __forceinline__ void top2_update(float &b1, float &b2, int &gi, float ka, float kb, int gbase) {
    const float mn = fminf(ka, kb), mx = fmaxf(ka, kb);
    const bool lt = mn < b1;
    b2 = fmin3(b2, fmaxf(b1, mn), mx);
    b1 = fminf(b1, mn);
    gi = lt ? (gbase | (int)(__float_as_uint(mn) & 31u)) : gi;
}

template <int D>
struct SharedLayout {
    static constexpr int K = moment_width(D);
    SeedRec raw[2][kChunk];
    float4 phi[Cfg<D>::NV][kChunk];
    unsigned long long tval[kTable][K];
    int tkey[kTable];
    uint64_t bar[2];
    int start_chunk;
};

template <int D>
__device__ __forceinline__ void table_add(SharedLayout<D> &sm, unsigned long long *gmom, int label,
                                          const unsigned long long (&val)[moment_width(D)]) {
    constexpr int K = moment_width(D);
    int slot = label & (kTable - 1);
    for (int probe = 0; probe < kTable; ++probe) {
        int k = atomicCAS(&sm.tkey[slot], -1, label);
        if (k == -1 || k == label) {
#pragma unroll
            for (int v = 0; v < K; ++v)
                if (val[v]) atomicAdd(&sm.tval[slot][v], val[v]);
            return;
        }
        slot = (slot + 1) & (kTable - 1);
    }
#pragma unroll
    for (int v = 0; v < K; ++v)
        if (val[v]) atomicAdd(&gmom[(size_t)label * K + v], val[v]);
}

template <int D>
__device__ __forceinline__ void flush_run(SharedLayout<D> &sm, unsigned long long *gmom, int label,
                                          unsigned long long cnt, unsigned long long s0,
                                          unsigned long long s00, unsigned long long u1,
                                          unsigned long long u2) {
    unsigned long long val[moment_width(D)];
    if (D == 3) {
        val[0] = cnt;
        val[1] = s0;
        val[2] = cnt * u1;
        val[3] = cnt * u2;
        val[4] = s00;
        val[5] = s0 * u1;
        val[6] = s0 * u2;
        val[7] = cnt * u1 * u1;
        val[8] = cnt * u1 * u2;
        val[9] = cnt * u2 * u2;
    } else {
        val[0] = cnt;
        val[1] = s0;
        val[2] = cnt * u1;
        val[3] = s00;
        val[4] = s0 * u1;
        val[5] = cnt * u1 * u1;
    }
    table_add<D>(sm, gmom, label, val);
}

template <int D>
__global__ void __launch_bounds__(256, 2)
    assign_fp32_kernel(const GridDev g, const int n, const int n_chunks, const float R_tile,
                       const SeedRec *__restrict__ recs, const uint32_t *__restrict__ scodes,
                       const int32_t *__restrict__ perm, unsigned long long *__restrict__ gmom,
                       uint32_t *__restrict__ flags, int32_t *__restrict__ labels,
                       DevScalars *__restrict__ sc) {
    using C = Cfg<D>;
    constexpr int P = C::P;
    constexpr int TY = C::TY;
    constexpr int K = moment_width(D);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    SharedLayout<D> &sm = *reinterpret_cast<SharedLayout<D> *>(smem_raw);

    const int tid = threadIdx.x;
    const int ty = tid % TY;
    const int tz = tid / TY;
    const int k0b = blockIdx.x * P;
    const int k1b = blockIdx.y * TY;
    const int k2b = (D == 3) ? blockIdx.z * C::TZ : 0;
    const int k1 = k1b + ty;
    const int k2 = k2b + tz;
    const bool row_valid = (k1 < g.res[1]) && (D == 2 || k2 < g.res[2]);

    // CTA reference point (FP64): row centre along axis 0, tile centre along 1, 2
    const double c0 = g.lo[0] + (double)(k0b + P / 2) * g.h[0];
    const double c1 = g.lo[1] + (double)(k1b + TY / 2) * g.h[1];
    const double c2 = (D == 3) ? g.lo[2] + (double)(k2b + C::TZ / 2) * g.h[2] : 0.0;
    const float f1 = ((float)(ty - TY / 2) + 0.5f) * g.h32[1];
    const float f2 = (D == 3) ? ((float)(tz - C::TZ / 2) + 0.5f) * g.h32[2] : 0.f;
    float2 y2[P / 2];
#pragma unroll
    for (int q = 0; q < P / 2; ++q)
        y2[q] = make_float2(((float)(2 * q - P / 2) + 0.5f) * g.h32[0],
                            ((float)(2 * q + 1 - P / 2) + 0.5f) * g.h32[0]);

    for (int t = tid; t < kTable; t += blockDim.x) {
        sm.tkey[t] = -1;
#pragma unroll
        for (int v = 0; v < K; ++v) sm.tval[t][v] = 0ull;
    }
    if (tid == 0) {
        mbar_init(&sm.bar[0], 1);
        mbar_init(&sm.bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    // Scan order of the seed chunks: with Morton-sorted seeds, start at the chunk
    // holding this tile's Morton position and zig-zag outwards, so that the near
    // seeds (the likely winners) come first and later groups are mostly skipped.
    if (tid == 0) {
        int start = 0;
        if (scodes) {
            double frac[3] = {0.0, 0.0, 0.0};
            const int kc[3] = {k0b + P / 2, k1b + TY / 2, k2b + C::TZ / 2};
#pragma unroll
            for (int a = 0; a < D; ++a) frac[a] = ((double)kc[a] + 0.5) / (double)g.res[a];
            const uint32_t code = morton_code(D, frac);
            int lo = 0, hi = n;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (scodes[mid] < code) lo = mid + 1;
                else hi = mid;
            }
            start = min(lo / kChunk, n_chunks - 1);
        }
        sm.start_chunk = start;
    }
    __syncthreads();
    const int start_chunk = sm.start_chunk;
    auto chunk_at = [&](int k) {
        const int off = (k & 1) ? ((k + 1) >> 1) : -(k >> 1);
        int c = (start_chunk + off) % n_chunks;
        return c < 0 ? c + n_chunks : c;
    };
    const double wref = dkey_inv(sc->wref_key);
    if (tid == 0) {
        for (int k = 0; k < 2 && k < n_chunks; ++k) {
            mbar_expect_tx(&sm.bar[k], kChunk * sizeof(SeedRec));
            bulk_g2s(&sm.raw[k][0], recs + (size_t)chunk_at(k) * kChunk, kChunk * sizeof(SeedRec),
                     &sm.bar[k]);
        }
    }

    // per pixel: two smallest packed costs (b1 <= b2) and the scan position of the best
    float b1[P], b2[P];
    int GI[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        b1[p] = FLT_MAX;
        b2[p] = FLT_MAX;
        GI[p] = 0;
    }
    bool ok = true;

    for (int k = 0; k < n_chunks; ++k) {
        const int b = k & 1;
        const int c = chunk_at(k);
        if (!mbar_wait_bounded(&sm.bar[b], (uint32_t)((k >> 1) & 1), &sc->status)) ok = false;
        // transform this chunk: one seed per thread
        {
            const int s = c * kChunk + tid;
            float4 v0, v1, v2;
            if (ok && s < n) {
                const SeedRec &r = sm.raw[b][tid];
                const float d0 = (float)(c0 - r.x[0]);
                const float x1p = (float)(r.x[1] - c1);
                const float wp = (float)(r.w - wref);  // <= 0
                if (D == 3) {
                    const float x2p = (float)(r.x[2] - c2);
                    const float A00 = r.a[0], A01 = r.a[1], A02 = r.a[2], A11 = r.a[3],
                                A12 = r.a[4], A22 = r.a[5];
                    v0 = make_float4(x1p, x2p, A11, 2.f * A12);
                    v1 = make_float4(A22, A01, A02, 2.f * A00 * d0);
                    v2 = make_float4(A00 * d0 * d0 - wp, 2.f * d0, A00, 0.f);
                } else {
                    const float A00 = r.a[0], A01 = r.a[1], A11 = r.a[2];
                    v0 = make_float4(x1p, A11, 2.f * A01 * d0, A00 * d0 * d0 - wp);
                    v1 = make_float4(2.f * A00 * d0, 2.f * A01, A00, 0.f);
                    v2 = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            } else {  // padding seed: constant huge cost
                if (D == 3) {
                    v0 = make_float4(0.f, 0.f, 0.f, 0.f);
                    v1 = make_float4(0.f, 0.f, 0.f, 0.f);
                    v2 = make_float4(1e30f, 0.f, 0.f, 0.f);
                } else {
                    v0 = make_float4(0.f, 0.f, 0.f, 1e30f);
                    v1 = make_float4(0.f, 0.f, 0.f, 0.f);
                    v2 = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
            sm.phi[0][tid] = v0;
            sm.phi[1][tid] = v1;
            if (D == 3) sm.phi[2][tid] = v2;
        }
        __syncthreads();
        if (tid == 0 && ok && k + 2 < n_chunks) {
            mbar_expect_tx(&sm.bar[b], kChunk * sizeof(SeedRec));
            bulk_g2s(&sm.raw[b][0], recs + (size_t)chunk_at(k + 2) * kChunk, kChunk * sizeof(SeedRec),
                     &sm.bar[b]);
        }
        if (ok) {
            const int valid_in_chunk = min(kChunk, n - c * kChunk);
            const int groups = (valid_in_chunk + kGroup - 1) / kGroup;
            for (int gr = 0; gr < groups; ++gr) {
                // fast pass: smallest cost of this group per pixel (one 3-input min per two pairs)
                float gm[P];
#pragma unroll
                for (int p = 0; p < P; ++p) gm[p] = FLT_MAX;
#pragma unroll 2
                for (int l = 0; l < kGroup; l += 2) {
                    float2 qa, qb, ba, bbb, aa2, ab2;
                    seed_pair_coeffs<D>(sm.phi, gr * kGroup + l, f1, f2, qa, qb, ba, bbb, aa2, ab2);
#pragma unroll
                    for (int q = 0; q < P / 2; ++q) {
                        const float2 ca = ffma2(ffma2(qa, y2[q], ba), y2[q], aa2);
                        const float2 cb = ffma2(ffma2(qb, y2[q], bbb), y2[q], ab2);
                        gm[2 * q] = fmin3(gm[2 * q], ca.x, cb.x);
                        gm[2 * q + 1] = fmin3(gm[2 * q + 1], ca.y, cb.y);
                    }
                }
                // a packed key differs from its cost by < 32 ulp: a group whose smallest
                // cost exceeds b2 by the margin cannot change b1 or b2 and is skipped
                bool need = false;
#pragma unroll
                for (int p = 0; p < P; ++p) need |= gm[p] < fmaf(fabsf(b2[p]), 0x1p-15f, b2[p]);
                if (!__any_sync(0xffffffffu, need)) continue;
                // update pass: recompute the same costs, packed top-2 with the index
                const int gbase = c * kChunk + gr * kGroup;
#pragma unroll 2
                for (int l = 0; l < kGroup; l += 2) {
                    float2 qa, qb, ba, bbb, aa2, ab2;
                    seed_pair_coeffs<D>(sm.phi, gr * kGroup + l, f1, f2, qa, qb, ba, bbb, aa2, ab2);
                    const unsigned la = (unsigned)l, lb = (unsigned)(l + 1);
#pragma unroll
                    for (int q = 0; q < P / 2; ++q) {
                        const float2 ca = ffma2(ffma2(qa, y2[q], ba), y2[q], aa2);
                        const float2 cb = ffma2(ffma2(qb, y2[q], bbb), y2[q], ab2);
                        top2_update(b1[2 * q], b2[2 * q], GI[2 * q], pack(ca.x, la), pack(cb.x, lb), gbase);
                        top2_update(b1[2 * q + 1], b2[2 * q + 1], GI[2 * q + 1], pack(ca.y, la),
                                    pack(cb.y, lb), gbase);
                    }
                }
            }
        }
        __syncthreads();
    }
    // scan position -> seed index
    if (perm && ok) {
#pragma unroll
        for (int p = 0; p < P; ++p) GI[p] = GI[p] < n ? perm[GI[p]] : GI[p];
    }

    // flag near ties, write labels, accumulate moments
    const float lam_abs = (float)__longlong_as_double((long long)sc->lam_abs_bits);
    const float lam_min = (float)__longlong_as_double((long long)sc->lam_min_bits);
    const float inv_lam = 1.f / fmaxf(lam_min, 1e-30f);
    const long long rowbase = (long long)g.res[0] * ((long long)k1 + (long long)g.res[1] * (long long)k2);
    const unsigned long long u1 = 2ull * (unsigned long long)k1 + 1ull;
    const unsigned long long u2 = 2ull * (unsigned long long)k2 + 1ull;
    int cur = -1;
    unsigned long long cnt = 0, s0 = 0, s00 = 0;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int k0 = k0b + p;
        const bool valid = ok && row_valid && (k0 < g.res[0]);
        bool flagged = false;
        if (valid) {
            const float cs = fabsf(b1[p]) * 1.0078125f + 1e-30f;
            const float rr = R_tile + sqrtf(cs * inv_lam);
            const float T = lam_abs * rr * rr + cs;
            const float E = kKappa * kUnit * T;
            // GI >= n only if a padding seed won (all real costs non-finite or huge)
            flagged = !(b2[p] - b1[p] > 2.f * E) || GI[p] >= n;
            const long long j = rowbase + k0;
            if (flagged) {
                const unsigned slot = atomicAdd(&sc->flag_count, 1u);
                flags[slot] = (uint32_t)j;
            }
            if (labels) labels[j] = GI[p];
        }
        const int L = (valid && !flagged) ? GI[p] : -1;
        if (L != cur) {
            if (cur >= 0) flush_run<D>(sm, gmom, cur, cnt, s0, s00, u1, u2);
            cur = L;
            cnt = s0 = s00 = 0;
        }
        if (L >= 0) {
            const unsigned long long u0 = 2ull * (unsigned long long)k0 + 1ull;
            cnt += 1;
            s0 += u0;
            s00 += u0 * u0;
        }
    }
    if (cur >= 0) flush_run<D>(sm, gmom, cur, cnt, s0, s00, u1, u2);
    __syncthreads();
    for (int t = tid; t < kTable; t += blockDim.x) {
        const int key = sm.tkey[t];
        if (key >= 0) {
#pragma unroll
            for (int v = 0; v < K; ++v) {
                const unsigned long long val = sm.tval[t][v];
                if (val) atomicAdd(&gmom[(size_t)key * K + v], val);
            }
        }
    }
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
template <int D>
__global__ void __launch_bounds__(256)
    rescore_kernel(const GridDev g, const int n, const double *__restrict__ x,
                   const double *__restrict__ A, const double *__restrict__ w,
                   const SeedRec32 *__restrict__ r32, const uint32_t *__restrict__ flags,
                   DevScalars *__restrict__ sc, unsigned long long *__restrict__ gmom,
                   int32_t *__restrict__ labels) {
    constexpr int K = moment_width(D);
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const unsigned count = sc->flag_count;
    if (warp == 0 && lane == 0 && count)
        atomicAdd((unsigned long long *)&sc->rescored_total, (unsigned long long)count);
    const double wref = dkey_inv(sc->wref_key);
    float wrh, wrl;
    wrh = (float)wref;
    wrl = (float)(wref - (double)wrh);
    for (unsigned it = warp; it < count; it += nwarps) {
        const long long j = (long long)flags[it];
        int k[3] = {0, 0, 0};
        long long rr = j;
        double y[D];
        float yh[3] = {0.f, 0.f, 0.f}, yl[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int a = 0; a < D; ++a) {
            k[a] = (int)(rr % g.res[a]);
            rr /= g.res[a];
            y[a] = __dadd_rn(g.lo[a], __dmul_rn((double)k[a] + 0.5, g.h[a]));
            yh[a] = (float)y[a];
            yl[a] = (float)(y[a] - (double)yh[a]);
        }
        // pass 1: threshold = min over seeds of (C + E)
        float thr = __int_as_float(0x7f800000);
        for (int s = lane; s < n; s += 32) {
            float c, E;
            cost32_bound<D>(r32[s], yh, yl, wrh, wrl, c, E);
            thr = fminf(thr, c + E);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) thr = fminf(thr, __shfl_xor_sync(0xffffffffu, thr, off));
        // pass 2: FP64 reference cost of the candidates
        double best = __longlong_as_double(0x7ff0000000000000ll);
        int bi = 0x7fffffff;
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
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, off);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
            if (ob < best || (ob == best && oi < bi)) {
                best = ob;
                bi = oi;
            }
        }
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
}

template <int D>
cudaError_t launch_assign_fp32_t(const GridDev &g, int n, Workspace &ws, int32_t *labels,
                                 unsigned long long *gmom, cudaStream_t st) {
    using C = Cfg<D>;
    const size_t smem = sizeof(SharedLayout<D>);
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(assign_fp32_kernel<D>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    dim3 grid((g.res[0] + C::P - 1) / C::P, (g.res[1] + C::TY - 1) / C::TY,
              D == 3 ? (g.res[2] + C::TZ - 1) / C::TZ : 1);
    const int n_chunks = (n + kChunk - 1) / kChunk;
    double hx = 0.5 * C::P * g.h[0], hy = 0.5 * C::TY * g.h[1], hz = D == 3 ? 0.5 * C::TZ * g.h[2] : 0.0;
    const float R = (float)(sqrt(hx * hx + hy * hy + hz * hz) * (1.0 + 1e-6));
    assign_fp32_kernel<D><<<grid, C::TY * C::TZ, smem, st>>>(
        g, n, n_chunks, R, ws.recs, ws.sorted ? ws.scodes : nullptr, ws.sorted ? ws.perm : nullptr, gmom,
        ws.flags, labels, ws.sc);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_assign_fp32(const GridDev &g, int n, Workspace &ws, int32_t *labels,
                               unsigned long long *moments, cudaStream_t st) {
    return g.dim == 3 ? launch_assign_fp32_t<3>(g, n, ws, labels, moments, st)
                      : launch_assign_fp32_t<2>(g, n, ws, labels, moments, st);
}

cudaError_t launch_rescore_fp64(const GridDev &g, int n, const double *x, const double *A,
                                const double *w, Workspace &ws, int32_t *labels,
                                unsigned long long *moments, cudaStream_t st) {
    int dev_sms = 152;
    cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, ws.device);
    const int blocks = dev_sms * 2;
    if (g.dim == 3)
        rescore_kernel<3><<<blocks, 256, 0, st>>>(g, n, x, A, w, ws.recs32, ws.flags, ws.sc, moments, labels);
    else
        rescore_kernel<2><<<blocks, 256, 0, st>>>(g, n, x, A, w, ws.recs32, ws.flags, ws.sc, moments, labels);
    return cudaGetLastError();
}

}  // namespace apd
