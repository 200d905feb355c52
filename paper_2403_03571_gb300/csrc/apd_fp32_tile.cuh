// FP32 scoring of one pixel tile (Algorithm 1 fused with the moment
// reduction), shared by the one-instance kernel and the batched persistent
// kernel.  The method and its rounding bound are described in
// apd_assign_fp32.cu.
#pragma once

#include <float.h>

#include "apd_internal.cuh"

namespace apd {
namespace fp32 {

constexpr float kUnit = 5.9604644775390625e-8f;  // 2^-24, unit roundoff of FP32
// Rounding-bound multiplier: about 24 roundings of size <= u T in the cost
// chain plus <= 62 u |C| from the packed 5-bit index, with a 1.8x margin.
constexpr float kKappa = 160.f;
constexpr int kTable = 128;  // shared-memory hash slots per CTA

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

// Two new packed keys of the group at scan position gbase into the top-2
// (b1 <= b2) of one pixel; gi follows b1's group (the index inside the group is
// in b1's low bits and is added once, after the scan).
__device__ __forceinline__ void top2_update(float &b1, float &b2, int &gi, float ka, float kb, int gbase) {
    const float mn = fminf(ka, kb), mx = fmaxf(ka, kb);
    const bool lt = mn < b1;
    b2 = fmin3(b2, fmaxf(b1, mn), mx);
    b1 = fminf(b1, mn);
    gi = lt ? gbase : gi;
}

// Largest second-best key over the warp's pixels.
template <int P>
__device__ __forceinline__ float warp_max_b2(const float (&b2)[P]) {
    float m = b2[0];
#pragma unroll
    for (int p = 1; p < P; ++p) m = fmaxf(m, b2[p]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    return m;
}
// True when a group whose cost lower bound is lb (wpart: its weight part) lies
// above the largest second-best key bmax by more than the rounding margin, so
// that none of its seeds can change a top-2 of the warp's pixels.
__device__ __forceinline__ bool group_beyond(float lb, float wpart, float bmax) {
    return bmax < FLT_MAX && lb > bmax + 1e-6f * (fabsf(bmax) + fabsf(lb) + fabsf(wpart)) + 1e-30f;
}
// Order-preserving map of a float to an unsigned key.
__device__ __forceinline__ unsigned sortable_key(float v) {
    const unsigned u = __float_as_uint(v);
    return u ^ ((u >> 31) ? 0xffffffffu : 0x80000000u);
}

template <int D>
struct SharedLayout {
    static constexpr int K = moment_width(D);
    SeedRec raw[2][kChunk];
    float4 phi[D][kChunk];
    float4 sbd[kChunk];  // per seed of the chunk: offset from the tile centre, lambda_min lower bound
    float swp[kChunk];   // per seed: a lower bound of wref - w (the weight part of its cost bound)
    unsigned long long tval[kTable][K];
    int tkey[kTable];
    uint64_t bar[2];
    int start_chunk;
    float wbox[16][6];  // per warp: pixel box lo[3], hi[3], absolute (pruning)
    float wrel[16][6];  // per warp: the same box relative to the tile centre
    float glb[16][kChunk / kGroup];  // per warp: cost lower bound of each group of the chunk
    float gwp[16][kChunk / kGroup];  // per warp: the weight part of that bound
    double cref[4];  // tile centre (FP64) and the reference weight wref
    unsigned long long scored;  // pixel-seed pairs the CTA's scoring evaluated in this tile
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

// Integer moments of a run of cnt pixels along the first axis (sum of the
// doubled first coordinate s0, of its square s00) on the row (u1, u2).
template <int D>
__device__ __forceinline__ void run_moments(unsigned long long cnt, unsigned long long s0, unsigned long long s00,
                                            unsigned long long u1, unsigned long long u2,
                                            unsigned long long (&val)[moment_width(D)]) {
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
}

template <int D>
__device__ __forceinline__ void flush_run(SharedLayout<D> &sm, unsigned long long *gmom, int label,
                                          unsigned long long cnt, unsigned long long s0,
                                          unsigned long long s00, unsigned long long u1,
                                          unsigned long long u2) {
    unsigned long long val[moment_width(D)];
    run_moments<D>(cnt, s0, s00, u1, u2, val);
    table_add<D>(sm, gmom, label, val);
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}


// One scoring problem: an instance's grid, seeds in scan order and outputs.
struct TileSrc {
    GridDev g;
    int n;
    int n_chunks;
    float R_tile;                 // tile half-diagonal bound
    const SeedRec *recs;          // [n_chunks * kChunk] scan order
    const uint32_t *scodes;       // sorted Morton codes (null: natural order)
    const int32_t *perm;          // scan position -> seed index (null: identity)
    unsigned long long *gmom;     // [n][K]
    uint32_t *flags;              // queue of pixels for FP64 rescoring
    int32_t *flag_gi;             // FP32 best seed of each queued pixel (or null)
    int32_t *labels;              // [J] or null
    DevScalars *sc;
    const GroupBound *groups;     // bounds of the scan-order 32-seed groups: pruning (null: dense)
    unsigned long long *pairs_scored;  // pixel-seed pairs the scoring evaluated (or null)
    uint32_t wait_limit;          // polls of each chunk wait (kDefaultWaitPolls normally)
};

// Scores the (TX P) x TY x TZ tile (bx, by, bz) of `s` with NT = TX TY TZ
// threads; thread (seg, ty, tz) owns the row segment of P pixels starting at
// first-axis offset seg P inside the tile.
// `uses[b]` counts the phases of chunk barrier b this thread has waited for,
// `uses[2 + b]` the copies issued into buffer b (thread 0), across the tiles a
// CTA has scored; the shared-memory table must be empty on entry and is empty
// again on return.  Returns false if a chunk wait timed out: thread 0 has then
// waited (with the default limit) for every copy still in flight, and the CTA
// must stop.
template <int D, int TX, int P, int TY, int TZ>
__device__ __forceinline__ bool score_tile(SharedLayout<D> &sm, const TileSrc &s, const int bx, const int by,
                                           const int bz, uint32_t (&uses)[4]) {
    constexpr int K = moment_width(D);
    constexpr int NT = TX * TY * TZ;
    constexpr int W0 = TX * P;  // tile width along the first axis
    const GridDev &g = s.g;
    const int n = s.n, n_chunks = s.n_chunks;

    const int tid = threadIdx.x;
    const int seg = tid % TX;
    // 3D tiles of 16 x 16 rows: each warp takes an 8 x 4 block of rows, a more
    // compact pixel box than 16 x 2 for the pruning bounds
    constexpr bool kBlockRows = D == 3 && TX == 1 && TY == 16 && TZ == 16;
    const int ty = kBlockRows ? ((tid & 7) + 8 * ((tid >> 5) & 1)) : (tid / TX) % TY;
    const int tz = kBlockRows ? (((tid >> 3) & 3) + 4 * (tid >> 6)) : tid / (TX * TY);
    const int k0t = bx * W0;       // first pixel of the tile along axis 0
    const int k0b = k0t + seg * P;  // first pixel of this thread's row segment
    const int k1b = by * TY;
    const int k2b = (D == 3) ? bz * TZ : 0;
    const int k1 = k1b + ty;
    const int k2 = k2b + tz;
    const int klast = D == 3 ? k2 : k1;  // the windowed axis
    const bool row_valid = (k1 < g.res[1]) && (D == 2 || k2 < g.res[2]) && klast >= win_lo(g) && klast < win_hi(g);

    const int lane = tid & 31;
    const int wid = tid >> 5;
    const int kc0 = k0t + W0 / 2, kc1 = k1b + TY / 2, kc2 = k2b + TZ / 2;  // tile centre pixel
    // CTA-uniform values, computed by one thread and kept in shared memory: the
    // tile centre (FP64, the reference point of the row form), the reference
    // weight, and the first chunk of the scan.  With Morton-sorted seeds the scan
    // starts at the chunk holding this tile's Morton position and zig-zags
    // outwards, so that the near seeds (the likely winners) come first.
    auto chunk_from = [n_chunks](int start, int k) {
        const int off = (k & 1) ? ((k + 1) >> 1) : -(k >> 1);
        int c = (start + off) % n_chunks;
        return c < 0 ? c + n_chunks : c;
    };
    if (tid == 0) {
        sm.cref[0] = g.lo[0] + (double)kc0 * g.h[0];
        sm.cref[1] = g.lo[1] + (double)kc1 * g.h[1];
        sm.cref[2] = (D == 3) ? g.lo[2] + (double)kc2 * g.h[2] : 0.0;
        sm.cref[3] = dkey_inv(s.sc->wref_key);
        int start = 0;
        if (s.scodes) {
            double frac[3] = {0.0, 0.0, 0.0};
            const int kc[3] = {kc0, kc1, kc2};
#pragma unroll
            for (int a = 0; a < D; ++a) frac[a] = ((double)kc[a] + 0.5) / (double)g.res[a];
            const uint32_t code = morton_code(D, frac);
            int lo = 0, hi = n;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (s.scodes[mid] < code) lo = mid + 1;
                else hi = mid;
            }
            start = min(lo / kChunk, n_chunks - 1);
        }
        sm.start_chunk = start;
        for (int k = 0; k < 2 && k < n_chunks; ++k) {
            mbar_expect_tx(&sm.bar[k], kChunk * sizeof(SeedRec));
            bulk_g2s(&sm.raw[k][0], s.recs + (size_t)chunk_from(start, k) * kChunk, kChunk * sizeof(SeedRec),
                     &sm.bar[k]);
            ++uses[2 + k];
        }
    }
    const float f1 = ((float)(ty - TY / 2) + 0.5f) * g.h32[1];
    const float f2 = (D == 3) ? ((float)(tz - TZ / 2) + 0.5f) * g.h32[2] : 0.f;
    float2 y2[P / 2];
#pragma unroll
    for (int q = 0; q < P / 2; ++q)
        y2[q] = make_float2(((float)(seg * P + 2 * q - W0 / 2) + 0.5f) * g.h32[0],
                            ((float)(seg * P + 2 * q + 1 - W0 / 2) + 0.5f) * g.h32[0]);

    // Pruning (optional): the box of this warp's pixel centres, in absolute FP32
    // coordinates rounded outwards (against the seed-group boxes) and relative to
    // the tile centre (against the seeds' own offsets from it); a seed or group
    // whose cost lower bound over the box exceeds every pixel's second-best cost
    // cannot change any label or queue decision and is skipped.
    if (s.groups) {
        const int klo[3] = {__reduce_min_sync(0xffffffffu, k0b), __reduce_min_sync(0xffffffffu, k1),
                            __reduce_min_sync(0xffffffffu, k2)};
        const int khi[3] = {__reduce_max_sync(0xffffffffu, k0b + P - 1), __reduce_max_sync(0xffffffffu, k1),
                            __reduce_max_sync(0xffffffffu, k2)};
        if (lane == 0) {
            const int kc[3] = {kc0, kc1, kc2};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const bool ax = a < D;
                sm.wbox[wid][a] = ax ? __double2float_rd(g.lo[a] + ((double)klo[a] + 0.5) * g.h[a]) : 0.f;
                sm.wbox[wid][3 + a] = ax ? __double2float_ru(g.lo[a] + ((double)khi[a] + 0.5) * g.h[a]) : 0.f;
                sm.wrel[wid][a] = ax ? ((float)(klo[a] - kc[a]) + 0.5f) * g.h32[a] : 0.f;
                sm.wrel[wid][3 + a] = ax ? ((float)(khi[a] - kc[a]) + 0.5f) * g.h32[a] : 0.f;
            }
        }
    }
    __syncthreads();  // sm.cref, sm.start_chunk, sm.wbox, sm.wrel
    const int start_chunk = sm.start_chunk;
    auto chunk_at = [&](int k) { return chunk_from(start_chunk, k); };

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
        if (ok) {
            if (mbar_wait_bounded(&sm.bar[b], uses[b] & 1u, &s.sc->status, s.wait_limit)) ++uses[b];
            else ok = false;
        }
        // Group bounds of this chunk (lane = group): the cost lower bound over the
        // warp's pixel box, used to order the groups (nearest first) and to skip
        // those above every pixel's second-best cost.  The dense sweep takes the
        // groups in index order.
        const int valid_in_chunk = min(kChunk, n - c * kChunk);
        const int groups = (valid_in_chunk + kGroup - 1) / kGroup;
        unsigned live = (1u << groups) - 1u;  // groups of this chunk the warp may score
        if (s.groups) {
            const float bmax = warp_max_b2<P>(b2);  // all lanes: it shuffles across the warp
            bool drop = false;
            if (lane < groups) {
                const GroupBound gb = s.groups[c * (kChunk / kGroup) + lane];
                float d2 = 0.f;
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    const float lo = sm.wbox[tid >> 5][a], hi = sm.wbox[tid >> 5][3 + a];
                    const float slack = 1e-6f * (fabsf(lo) + fabsf(hi) + fabsf(gb.lo[a]) + fabsf(gb.hi[a]));
                    const float t = fmaxf(fmaxf(gb.lo[a] - hi, lo - gb.hi[a]) - slack, 0.f);
                    d2 = fmaf(t, t, d2);
                }
                const float wp = gb.wgap;
                const float lb = __fmul_rd(__fmul_rd(gb.lam, d2), 1.f - 1e-5f) + wp;
                sm.glb[wid][lane] = lb;
                sm.gwp[wid][lane] = wp;
                drop = group_beyond(lb, wp, bmax);
            }
            live &= ~__ballot_sync(0xffffffffu, drop);
            __syncwarp();
        }
        const bool need_chunk = s.groups ? (__syncthreads_or(live != 0u) != 0) : true;
        // transform this chunk into the row-form coefficients
        for (int sl = need_chunk ? tid : kChunk; sl < kChunk; sl += NT) {
            const int si = c * kChunk + sl;
            float4 v0, v1, v2;
            // pruning data: the seed's offset from the tile centre (FP32 of the FP64
            // difference), its lambda_min lower bound, and a lower bound of wref - w
            float4 bd = make_float4(0.f, 0.f, 0.f, 0.f);
            float bw = 0.f;
            if (ok && si < n) {
                const SeedRec &r = sm.raw[b][sl];
                const float d0 = (float)(sm.cref[0] - r.x[0]);
                const float x1p = (float)(r.x[1] - sm.cref[1]);
                const float x2p = (D == 3) ? (float)(r.x[2] - sm.cref[2]) : 0.f;
                const float wp = (float)(r.w - sm.cref[3]);  // <= 0
                bd = make_float4(-d0, x1p, x2p, r.pad[0]);
                bw = __fmul_rd(-wp, 1.f - 0x1p-23f);  // rounding of wp is below 2^-24 relative
                if (D == 3) {
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
            sm.phi[0][sl] = v0;
            sm.phi[1][sl] = v1;
            if (D == 3) sm.phi[2][sl] = v2;
            if (s.groups) {
                sm.sbd[sl] = bd;
                sm.swp[sl] = bw;
            }
        }
        // a timed-out wait in any thread stops the whole CTA
        ok = __syncthreads_and(ok);
        if (tid == 0 && ok && k + 2 < n_chunks) {
            mbar_expect_tx(&sm.bar[b], kChunk * sizeof(SeedRec));
            bulk_g2s(&sm.raw[b][0], s.recs + (size_t)chunk_at(k + 2) * kChunk, kChunk * sizeof(SeedRec),
                     &sm.bar[b]);
            ++uses[2 + b];
        }
        if (ok && need_chunk) {
            while (true) {
                // drop the groups that the current second-best costs rule out,
                // then take the remaining one with the smallest bound
                const bool mine = (live >> lane) & 1u;
                float bmax = FLT_MAX;
                if (s.groups) {
                    bmax = warp_max_b2<P>(b2);
                    live &= ~__ballot_sync(0xffffffffu,
                                           mine && group_beyond(sm.glb[wid][lane], sm.gwp[wid][lane], bmax));
                }
                if (!live) break;
                unsigned pick = live;  // dense: index order
                if (s.groups) {
                    const bool cand = (live >> lane) & 1u;
                    const unsigned key = cand ? sortable_key(sm.glb[wid][lane]) : 0xffffffffu;
                    const unsigned kmin = __reduce_min_sync(0xffffffffu, key);
                    pick = __ballot_sync(0xffffffffu, cand && key == kmin);
                    if (!pick) break;  // cannot happen: kmin is a candidate's key
                }
                const int gr = __ffs(pick) - 1;
                live &= ~(1u << gr);
                const int gbase = c * kChunk + gr * kGroup;
                // exact top-2 update of every pixel with the seed pair (l, l+1)
                auto update_pair = [&](const int l) {
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
                };
                if (s.groups) {
                    // Pruned: the seeds of the group whose own bound (lambda_i times the
                    // squared distance from x_i to the warp's pixel box, plus wref - w_i)
                    // is not above every pixel's second-best cost, scored in pairs
                    // (l, l+1) (marked at the even bit l) by the exact update directly:
                    // nearly every such pair changes some pixel's top-2.
                    const int sl = gr * kGroup + lane;
                    const bool real = sl < valid_in_chunk;
                    float slb = FLT_MAX, swp = 0.f;
                    if (real) {
                        const float4 sb = sm.sbd[sl];
                        swp = sm.swp[sl];
                        const float xs[3] = {sb.x, sb.y, sb.z};
                        float d2 = 0.f;
#pragma unroll
                        for (int a = 0; a < D; ++a) {
                            const float lo = sm.wrel[wid][a], hi = sm.wrel[wid][3 + a];
                            const float slack = 1e-6f * (fabsf(lo) + fabsf(hi) + 2.f * fabsf(xs[a]));
                            const float t = fmaxf(fmaxf(xs[a] - hi, lo - xs[a]) - slack, 0.f);
                            d2 = fmaf(t, t, d2);
                        }
                        slb = __fmul_rd(__fmul_rd(sb.w, d2), 1.f - 1e-5f) + swp;
                    }
                    unsigned done = 0u;
                    if (!(bmax < FLT_MAX)) {
                        // first group of the tile: the pair holding the seed of smallest
                        // bound goes first, so that the rest is tested against real costs
                        const unsigned key = real ? sortable_key(slb) : 0xffffffffu;
                        const unsigned kmin = __reduce_min_sync(0xffffffffu, key);
                        const int j = (__ffs(__ballot_sync(0xffffffffu, key == kmin)) - 1) & ~1;
                        update_pair(j);
                        done = 1u << j;
                        bmax = warp_max_b2<P>(b2);
                    }
                    const unsigned sv = __ballot_sync(0xffffffffu, real && !group_beyond(slb, swp, bmax));
                    const unsigned pm = (sv | (sv >> 1)) & 0x55555555u & ~done;
                    if (s.pairs_scored && lane == 0)
                        atomicAdd(&sm.scored, (unsigned long long)(2 * __popc(pm | done)) *
                                                  (unsigned long long)(32 * P));
                    for (unsigned m = pm; m; m &= m - 1u) update_pair(__ffs(m) - 1);
                    continue;
                }
                if (s.pairs_scored && lane == 0)
                    atomicAdd(&sm.scored, (unsigned long long)min(kGroup, valid_in_chunk - gr * kGroup) *
                                              (unsigned long long)(32 * P));
                // dense: fast pass (smallest cost of this group per pixel, one 3-input
                // min per two pairs), then the update pass only where it can matter
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
#pragma unroll 2
                for (int l = 0; l < kGroup; l += 2) update_pair(l);
            }
        }
        __syncthreads();
    }
    if (!ok && tid == 0) {
        // a wait gave up: let the copies still in flight land before the CTA stops
#pragma unroll
        for (int b = 0; b < 2; ++b)
            while (uses[b] < uses[2 + b] && mbar_wait_bounded(&sm.bar[b], uses[b] & 1u, &s.sc->status)) ++uses[b];
    }
    // scan position of the best: its group base and the index bits of its key
#pragma unroll
    for (int p = 0; p < P; ++p) GI[p] |= (int)(__float_as_uint(b1[p]) & 31u);
    // scan position -> seed index
    if (s.perm && ok) {
#pragma unroll
        for (int p = 0; p < P; ++p) GI[p] = GI[p] < n ? s.perm[GI[p]] : GI[p];
    }

    // flag near ties, write labels, accumulate moments
    const float lam_abs = (float)__longlong_as_double((long long)s.sc->lam_abs_bits);
    const float lam_min = (float)__longlong_as_double((long long)s.sc->lam_min_bits);
    const float inv_lam = 1.f / fmaxf(lam_min, 1e-30f);
    const long long rowbase = (long long)g.res[0] * ((long long)k1 + (long long)g.res[1] * (long long)k2);
    const unsigned long long u1 = 2ull * (unsigned long long)k1 + 1ull;
    const unsigned long long u2 = 2ull * (unsigned long long)k2 + 1ull;
    // Runs of equal labels along the thread's row: the first kRuns are kept for
    // the warp-level aggregation below, any further ones go to the table at once.
    constexpr int kRuns = 4;
    int rlab[kRuns];
    unsigned long long rcnt[kRuns], rs0[kRuns], rs00[kRuns];
#pragma unroll
    for (int q = 0; q < kRuns; ++q) {
        rlab[q] = -1;
        rcnt[q] = rs0[q] = rs00[q] = 0ull;
    }
    int nr = 0;
    auto end_run = [&](int lab, unsigned long long c_, unsigned long long a_, unsigned long long b_) {
        if (nr < kRuns) {
#pragma unroll
            for (int q = 0; q < kRuns; ++q)
                if (q == nr) {
                    rlab[q] = lab;
                    rcnt[q] = c_;
                    rs0[q] = a_;
                    rs00[q] = b_;
                }
            ++nr;
        } else {
            flush_run<D>(sm, s.gmom, lab, c_, a_, b_, u1, u2);
        }
    };
    int cur = -1;
    unsigned long long cnt = 0, s0 = 0, s00 = 0;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int k0 = k0b + p;
        const bool valid = ok && row_valid && (k0 < g.res[0]);
        bool flagged = false;
        if (valid) {
            const float cs = fabsf(b1[p]) * 1.0078125f + 1e-30f;
            const float rr = s.R_tile + sqrtf(cs * inv_lam);
            const float T = lam_abs * rr * rr + cs;
            const float E = kKappa * kUnit * T;
            // GI >= n only if a padding seed won (all real costs non-finite or huge)
            flagged = !(b2[p] - b1[p] > 2.f * E) || GI[p] >= n;
            const long long j = rowbase + k0;
            if (flagged) {
                const unsigned slot = atomicAdd(&s.sc->flag_count, 1u);
                s.flags[slot] = (uint32_t)j;
                if (s.flag_gi) s.flag_gi[slot] = GI[p] < n ? GI[p] : -1;
            }
            if (s.labels) s.labels[j] = GI[p];
        }
        const int L = (valid && !flagged) ? GI[p] : -1;
        if (L != cur) {
            if (cur >= 0) end_run(cur, cnt, s0, s00);
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
    if (cur >= 0) end_run(cur, cnt, s0, s00);
    // Warp-level aggregation (neighbouring rows mostly share their labels): in
    // round q every lane offers its q-th run; the lanes holding the label of
    // the lowest offering lane sum their moments and that lane adds the sums
    // to the table, so each label costs one set of shared atomics per warp and
    // round instead of one per row.
#pragma unroll
    for (int q = 0; q < kRuns; ++q) {
        const bool has = rlab[q] >= 0;
        unsigned todo = __ballot_sync(0xffffffffu, has);
        if (!todo) break;
        unsigned long long own[K];
        run_moments<D>(rcnt[q], rs0[q], rs00[q], u1, u2, own);
        while (todo) {
            const int leader = __ffs(todo) - 1;
            const int L0 = __shfl_sync(0xffffffffu, rlab[q], leader);
            const bool mine = has && rlab[q] == L0;
            const unsigned grp = __ballot_sync(0xffffffffu, mine);
            if (grp == (1u << leader)) {
                if (lane == leader) table_add<D>(sm, s.gmom, L0, own);
            } else {
                unsigned long long sum[K];
#pragma unroll
                for (int v = 0; v < K; ++v) sum[v] = warp_sum_u64(mine ? own[v] : 0ull);
                if (lane == leader) table_add<D>(sm, s.gmom, L0, sum);
            }
            todo &= ~grp;
        }
    }
    __syncthreads();
    if (tid == 0 && s.pairs_scored) {
        atomicAdd(s.pairs_scored, sm.scored);
        sm.scored = 0ull;
    }
    // flush the table to the global moments and leave it empty
    for (int t = tid; t < kTable; t += NT) {
        const int key = sm.tkey[t];
        if (key >= 0) {
#pragma unroll
            for (int v = 0; v < K; ++v) {
                const unsigned long long val = sm.tval[t][v];
                if (val) atomicAdd(&s.gmom[(size_t)key * K + v], val);
                sm.tval[t][v] = 0ull;
            }
            sm.tkey[t] = -1;
        }
    }
    __syncthreads();
    return ok;
}

// Empty table and initialised chunk barriers; call once per CTA.
template <int D>
__device__ __forceinline__ void init_shared(SharedLayout<D> &sm) {
    constexpr int K = moment_width(D);
    for (int t = threadIdx.x; t < kTable; t += blockDim.x) {
        sm.tkey[t] = -1;
#pragma unroll
        for (int v = 0; v < K; ++v) sm.tval[t][v] = 0ull;
    }
    if (threadIdx.x == 0) {
        mbar_init(&sm.bar[0], 1);
        mbar_init(&sm.bar[1], 1);
        fence_mbar_init();
        sm.scored = 0ull;
    }
    __syncthreads();
}

}  // namespace fp32
}  // namespace apd
