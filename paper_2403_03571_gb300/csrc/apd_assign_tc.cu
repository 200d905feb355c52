// Algorithm 1 on the 5th-generation tensor cores (tcgen05), fused with the
// per-cell integer moments.
//
// Expanded cost.  Around the centre c of a CTA's pixel tile, with y' = y - c
// and x' = x_i - c, the cost of eq. (2.1) is a dot product of pixel features
// and seed features:
//   C_ij + const = [y'_a y'_b (a <= b), y'_a, 1] . [A_ab (x2 off-diagonal), -2 (A x')_a, x'^T A x' - w'_i]
// (10 features in 3D, 6 in 2D, padded to the MMA's K).  The pixel features
// depend only on the pixel's place in its tile, so they are built once per CTA.
//
// Pipeline.  One persistent CTA per SM (16 warps) owns 512 pixels at a time
// (four M = 128 tiles, one tensor-memory lane per pixel) and walks the stream
// of (tile, seed chunk) steps, 64 seeds per chunk, with two accumulator stages
// in tensor memory (4 tiles x 2 stages x 64 columns = all 512 columns): while
// the epilogue of step q reads stage q & 1, the MMAs of step q + 1 fill the
// other stage.  Seed records arrive by 1-D bulk async copies into a 3-slot
// ring; four warps turn the records of step q + 2 into recentred seed features
// (TF32 or BF16) in the free B buffer; thread 0 issues the MMAs of step q + 2
// after the iteration's single CTA barrier.  Per-tile centres (FP64, split into
// FP32 high/low parts) and Morton start chunks come from a small pre-kernel.
//
// Epilogue.  Each thread owns one pixel and reads its 64 scores of the step
// with two tcgen05.ld.  Minima of 8-seed slices (3-input min) are compared with
// the pixel's fourth-best score; only slices that can enter the top-4 list are
// inserted.
//
// Exactness.  A score differs from the exact cost (up to the common shift)
// by at most err_unit * sum_k |f_k phi_k|, err_unit covering the rounding of both
// operands to TF32 (2^-11 each) or BF16 (2^-9 each) and the FP32 work.  The
// three best seeds of a pixel are rescored in FP32 direct form with per-seed
// bounds (the helper of the rescoring kernel).  Any other seed scored at least
// the fourth-best score s4, so its exact cost is at least s4 - psi, psi
// bounding the term magnitude of a seed of that cost from max ||A||_F,
// min lambda_min and the tile radius.  The label is decided when the best
// rescored upper bound lies below both s4 - psi and the other candidates' lower
// bounds; otherwise the pixel is queued for the full rescoring kernel, which
// ends in the FP64 reference arithmetic.
#include <cuda_bf16.h>
#include <float.h>

#include <algorithm>
#include <cmath>

#include "apd_cost.cuh"
#include "apd_internal.cuh"
#include "apd_tcgen05.cuh"

namespace apd {

namespace {

constexpr int kTcN = 64;        // seeds per MMA (N) and per pipeline step
constexpr int kTcM = 128;       // pixels per M tile
constexpr int kTcTiles = 4;     // M tiles per CTA tile
constexpr int kTcThreads = kTcTiles * kTcM;
constexpr int kTcStages = 2;    // accumulator stages in tensor memory
constexpr int kTcRaw = 3;       // bulk-copy ring slots
constexpr int kTcTable = 128;   // shared hash slots for the moments
constexpr uint32_t kTcCols = kTcTiles * kTcStages * kTcN;  // 512 tensor-memory columns
constexpr int kXformWarp0 = 12;  // warps 12..15 build the seed features (one warp per SM sub-partition)
constexpr int kNumXformWarps = 4;
constexpr int kProducerWarp = kTcThreads / 32;       // warp 16: bulk copies and MMAs
constexpr int kTcThreadsAll = kTcThreads + 32;

template <int D>
struct TcGeom;
template <>
struct TcGeom<3> {
    static constexpr int TX = 8, TY = 8, TZ = 8, F = 10;  // 64 rows of 8 pixels
};
template <>
struct TcGeom<2> {
    static constexpr int TX = 32, TY = 16, TZ = 1, F = 6;  // 16 rows of 32 pixels
};

template <int D, int KIND>
struct TcFmt {
    static constexpr int EB = KIND == tc::KIND_TF32 ? 4 : 2;              // bytes per element
    static constexpr int EPR = 16 / EB;                                   // elements per core-matrix row
    static constexpr int KSTEP = KIND == tc::KIND_TF32 ? 8 : 16;          // K of one MMA
    static constexpr int KT = (D == 2 && KIND == tc::KIND_TF32) ? 8 : 16;  // padded feature count
    static constexpr int STEPS = KT / KSTEP;
    static constexpr uint32_t LBO = 128;                                  // K-adjacent core matrices
    static constexpr uint32_t SBO = (KT / EPR) * 128;                     // next 8-row group
    static constexpr int A_BYTES = kTcM * KT * EB;
    static constexpr int B_BYTES = kTcN * KT * EB;
};

template <int D, int KIND>
struct TcShared {
    alignas(1024) uint8_t A[kTcTiles][TcFmt<D, KIND>::A_BYTES];
    alignas(1024) uint8_t B[kTcStages][TcFmt<D, KIND>::B_BYTES];
    alignas(16) SeedRec32 raw[kTcRaw][kTcN];
    uint64_t bar_raw[kTcRaw];
    uint64_t bar_acc[kTcStages];     // accumulator stage full (MMA commit)
    uint64_t bar_aempty[kTcStages];  // accumulator stage read by all 16 epilogue warps
    uint64_t bar_bfull[kTcStages];   // B operand built by the 4 transform warps
    uint32_t tslot;
    int abort;
};

__device__ __forceinline__ uint32_t cm_off(int row, int k, int eb, int epr, uint32_t lbo, uint32_t sbo) {
    return (uint32_t)(row >> 3) * sbo + (uint32_t)(k / epr) * lbo + (uint32_t)(row & 7) * 16u +
           (uint32_t)(k % epr) * (uint32_t)eb;
}

template <int KIND>
__device__ __forceinline__ void put_op(uint8_t *base, uint32_t off, float v) {
    if (KIND == tc::KIND_TF32)
        *reinterpret_cast<float *>(base + off) = tc::to_tf32(v);
    else
        *reinterpret_cast<__nv_bfloat16 *>(base + off) = __float2bfloat16_rn(v);
}

// One 16-byte core-matrix row: 4 TF32 or 8 BF16 operand values.
template <int KIND>
__device__ __forceinline__ void put_row(uint8_t *dst, const float (&e)[KIND == tc::KIND_TF32 ? 4 : 8]) {
    if (KIND == tc::KIND_TF32) {
        *reinterpret_cast<float4 *>(dst) = make_float4(tc::to_tf32(e[0]), tc::to_tf32(e[1]), tc::to_tf32(e[2]),
                                                       tc::to_tf32(e[3]));
    } else {
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(e[2 * i], e[2 * i + 1]);
            w[i] = *reinterpret_cast<const uint32_t *>(&h);
        }
        *reinterpret_cast<uint4 *>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ float fmin3_f(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

__device__ __forceinline__ void split2(double v, float &h, float &l) {
    h = (float)v;
    l = (float)(v - (double)h);
}

template <int D>
__device__ __forceinline__ void tc_table_add(int *tkey, unsigned long long (*tval)[moment_width(D)],
                                             unsigned long long *gmom, int label,
                                             const unsigned long long (&val)[moment_width(D)]) {
    constexpr int K = moment_width(D);
    int slot = label & (kTcTable - 1);
    for (int probe = 0; probe < kTcTable; ++probe) {
        const int k = atomicCAS(&tkey[slot], -1, label);
        if (k == -1 || k == label) {
#pragma unroll
            for (int v = 0; v < K; ++v)
                if (val[v]) atomicAdd(&tval[slot][v], val[v]);
            return;
        }
        slot = (slot + 1) & (kTcTable - 1);
    }
#pragma unroll
    for (int v = 0; v < K; ++v)
        if (val[v]) atomicAdd(&gmom[(size_t)label * K + v], val[v]);
}

// insert (v, id) into the ascending top-4 (s, ix); strict comparisons keep the
// earlier entry first among equal scores
__device__ __forceinline__ void top4_insert(float (&s)[4], int (&ix)[4], float v, int id) {
    if (!(v < s[3])) return;
    s[3] = v;
    ix[3] = id;
#pragma unroll
    for (int k = 3; k > 0; --k) {
        if (s[k] < s[k - 1]) {
            const float t = s[k];
            s[k] = s[k - 1];
            s[k - 1] = t;
            const int u = ix[k];
            ix[k] = ix[k - 1];
            ix[k - 1] = u;
        }
    }
}

// Per-tile data: FP32 high/low split of the tile centre lo + (kb + T/2) h, and
// the 64-seed chunk holding the tile centre's Morton position (0 without order).
template <int D>
__global__ void tc_tile_prep_kernel(const GridDev g, const int ntx, const int nty, const int ntiles, const int n,
                                    const int n_chunks, const uint32_t *__restrict__ scodes,
                                    float *__restrict__ centre, int *__restrict__ start) {
    using G = TcGeom<D>;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    const int kb[3] = {(t % ntx) * G::TX, ((t / ntx) % nty) * G::TY, (t / (ntx * nty)) * G::TZ};
    const int td[3] = {G::TX, G::TY, G::TZ};
    double frac[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float h = 0.f, l = 0.f;
        if (a < D) {
            const double cc = g.lo[a] + (double)(kb[a] + td[a] / 2) * g.h[a];
            split2(cc, h, l);
            frac[a] = ((double)(kb[a] + td[a] / 2) + 0.5) / (double)g.res[a];
        }
        centre[(size_t)t * 6 + a] = h;
        centre[(size_t)t * 6 + 3 + a] = l;
    }
    int st = 0;
    if (scodes) {
        const uint32_t code = morton_code(D, frac);
        int lo = 0, hi = n;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (scodes[mid] < code) lo = mid + 1;
            else hi = mid;
        }
        st = min(lo / kTcN, n_chunks - 1);
    }
    start[t] = st;
}

template <int D, int KIND>
__global__ void __launch_bounds__(kTcThreadsAll, 1)
    assign_tc_kernel(const GridDev g, const int n, const int n_chunks, const int ntx, const int nty,
                     const int ntiles, const SeedRec32 *__restrict__ rs, const float *__restrict__ tcentre,
                     const int *__restrict__ tstart, int4 *__restrict__ cand,
                     DevScalars *__restrict__ sc) {
    using G = TcGeom<D>;
    using Fm = TcFmt<D, KIND>;
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    TcShared<D, KIND> &sm = *reinterpret_cast<TcShared<D, KIND> *>(tc_smem_raw);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool producer = warp == kProducerWarp;
    const int mt = (tid >> 7) & (kTcTiles - 1);  // M tile of this (epilogue) thread
    const int row = tid & (kTcM - 1);             // tensor-memory lane = pixel of the M tile
    const int lt = mt * kTcM + row;               // pixel inside the CTA tile
    const int lx = lt % G::TX, ly = (lt / G::TX) % G::TY, lz = lt / (G::TX * G::TY);
    const int lk[3] = {lx, ly, lz};
    const int tdim[3] = {G::TX, G::TY, G::TZ};

    // this CTA's tiles: blockIdx.x, blockIdx.x + gridDim.x, ...
    const int my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int Q = my_tiles * n_chunks;  // pipeline steps (fits in 32 bits: tiles x chunks < 2^31)

    // pixel features (identical for every tile): A operand row `row` of M tile `mt`
    float yp[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int a = 0; a < D; ++a) yp[a] = ((float)(lk[a] - tdim[a] / 2) + 0.5f) * g.h32[a];
    if (!producer) {
        float f[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) f[k] = 0.f;
        if (D == 3) {
            f[0] = yp[0] * yp[0];
            f[1] = yp[0] * yp[1];
            f[2] = yp[0] * yp[2];
            f[3] = yp[1] * yp[1];
            f[4] = yp[1] * yp[2];
            f[5] = yp[2] * yp[2];
            f[6] = yp[0];
            f[7] = yp[1];
            f[8] = yp[2];
            f[9] = 1.f;
        } else {
            f[0] = yp[0] * yp[0];
            f[1] = yp[0] * yp[1];
            f[2] = yp[1] * yp[1];
            f[3] = yp[0];
            f[4] = yp[1];
            f[5] = 1.f;
        }
#pragma unroll
        for (int k = 0; k < Fm::KT; ++k)
            put_op<KIND>(sm.A[mt], cm_off(row, k, Fm::EB, Fm::EPR, Fm::LBO, Fm::SBO), f[k]);
    }
    if (warp == 0) {
        tc::tmem_alloc(&sm.tslot, kTcCols);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int i = 0; i < kTcRaw; ++i) mbar_init(&sm.bar_raw[i], 1);
        for (int i = 0; i < kTcStages; ++i) {
            mbar_init(&sm.bar_acc[i], 1);
            mbar_init(&sm.bar_aempty[i], kTcThreads / 32);
            mbar_init(&sm.bar_bfull[i], kNumXformWarps);
        }
        sm.abort = 0;
        fence_mbar_init();
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = sm.tslot;
    const uint32_t lane_base = ((uint32_t)((warp & 3) * 32)) << 16;

    const double wref = dkey_inv(sc->wref_key);
    float wrh, wrl;
    split2(wref, wrh, wrl);

    // Step q of this CTA is chunk position k = q mod n_chunks of tile i = q / n_chunks.
    // Each role keeps a cursor that advances one step at a time (no division in loops).
    struct Cursor {
        int tile, k, start;
    };
    auto cur_init = [&](int q) {
        Cursor c;
        const int i = q / n_chunks;
        c.k = q - i * n_chunks;
        c.tile = (int)blockIdx.x + i * (int)gridDim.x;
        c.start = c.tile < ntiles ? tstart[c.tile] : 0;
        return c;
    };
    auto cur_next = [&](Cursor &c) {
        if (++c.k == n_chunks) {
            c.k = 0;
            c.tile += (int)gridDim.x;
            c.start = c.tile < ntiles ? tstart[c.tile] : 0;
        }
    };
    // zig-zag outwards from the tile's Morton start chunk
    auto chunk_id = [&](const Cursor &c) {
        const int off = (c.k & 1) ? ((c.k + 1) >> 1) : -(c.k >> 1);
        int id = c.start + off;
        if (id >= n_chunks) id -= n_chunks;
        if (id < 0) id += n_chunks;
        return id;
    };
    // bounded wait that gives up at once after any timeout of the CTA
    auto wait = [&](uint64_t *bar, uint32_t parity) {
        if (*(volatile int *)&sm.abort) return false;
        if (mbar_wait_bounded(bar, parity, &sc->status)) return true;
        *(volatile int *)&sm.abort = 1;
        return false;
    };

    if (producer) {
        // ---------------- producer warp: bulk copies of seed records, MMAs ----------------
        if (lane == 0) {
            Cursor c_ld = cur_init(0);
            auto load_raw = [&](int q) {
                const int slot = q % kTcRaw;
                mbar_expect_tx(&sm.bar_raw[slot], kTcN * sizeof(SeedRec32));
                bulk_g2s(&sm.raw[slot][0], rs + (size_t)chunk_id(c_ld) * kTcN, kTcN * sizeof(SeedRec32),
                         &sm.bar_raw[slot]);
                cur_next(c_ld);
            };
            for (int q = 0; q < kTcRaw && q < Q; ++q) load_raw(q);
            const uint32_t idesc = tc::instr_desc(KIND, kTcM, kTcN);
            uint64_t adesc[kTcTiles][Fm::STEPS], bdesc[kTcStages][Fm::STEPS];
#pragma unroll
            for (int st = 0; st < Fm::STEPS; ++st) {
                const uint32_t off = (uint32_t)st * 2u * Fm::LBO;
#pragma unroll
                for (int m = 0; m < kTcTiles; ++m)
                    adesc[m][st] = tc::smem_desc((uint32_t)__cvta_generic_to_shared(sm.A[m]) + off, Fm::LBO, Fm::SBO);
#pragma unroll
                for (int bb = 0; bb < kTcStages; ++bb)
                    bdesc[bb][st] = tc::smem_desc((uint32_t)__cvta_generic_to_shared(sm.B[bb]) + off, Fm::LBO, Fm::SBO);
            }
            for (int q = 0; q < Q; ++q) {
                const int b = q & 1;
                if (!wait(&sm.bar_bfull[b], (uint32_t)((q >> 1) & 1))) break;
                if (q >= 2 && !wait(&sm.bar_aempty[b], (uint32_t)(((q >> 1) - 1) & 1))) break;
                tc::fence_after_sync();
#pragma unroll
                for (int m = 0; m < kTcTiles; ++m) {
                    const uint32_t d = taddr + (uint32_t)((b * kTcTiles + m) * kTcN);
#pragma unroll
                    for (int st = 0; st < Fm::STEPS; ++st) {
                        const uint64_t bd = b ? bdesc[1][st] : bdesc[0][st];
                        if (KIND == tc::KIND_TF32)
                            tc::mma_tf32(d, adesc[m][st], bd, idesc, st > 0 ? 1u : 0u);
                        else
                            tc::mma_bf16(d, adesc[m][st], bd, idesc, st > 0 ? 1u : 0u);
                    }
                }
                tc::mma_commit(&sm.bar_acc[b]);
                // the seed records of step q were consumed (B of step q is built): reuse the slot
                if (q + kTcRaw < Q) load_raw(q + kTcRaw);
            }
        }
    } else {
        // ---------------- 16 epilogue warps (warps 12..15 also build B) ----------------
        const bool xform = warp >= kXformWarp0;
        Cursor c_xf = cur_init(0);
        int xf_tile = -1;
        float xch[3] = {0.f, 0.f, 0.f}, xcl[3] = {0.f, 0.f, 0.f};
        auto transform = [&](int q) {  // xform warps: B operand of step q (two threads per seed)
            const int slot = q % kTcRaw;
            bool okw = wait(&sm.bar_raw[slot], (uint32_t)((q / kTcRaw) & 1));
            const int tt = tid - kXformWarp0 * 32;  // 0..127
            const int sl = tt >> 1, half = tt & 1;
            const int c = chunk_id(c_xf);
            const int s = c * kTcN + sl;
            if (c_xf.tile != xf_tile) {  // tile centre of the step, reloaded once per tile
                xf_tile = c_xf.tile;
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    xch[a] = tcentre[(size_t)xf_tile * 6 + a];
                    xcl[a] = tcentre[(size_t)xf_tile * 6 + 3 + a];
                }
            }
            float phv[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) phv[i] = 0.f;
            if (okw && s < n) {
                // the 64-byte record as four 16-byte loads (x hi, x lo, w hi/lo, A)
                const float4 *rv = reinterpret_cast<const float4 *>(&sm.raw[slot][sl]);
                const float4 q0 = rv[0], q1 = rv[1], q2 = rv[2], q3 = rv[3];
                const float rxh[3] = {q0.x, q0.y, q0.z}, rxl[3] = {q0.w, q1.x, q1.y};
                const float ra[6] = {q2.x, q2.y, q2.z, q2.w, q3.x, q3.y};
                float xp[3] = {0.f, 0.f, 0.f};
#pragma unroll
                for (int a = 0; a < D; ++a)
                    xp[a] = (rxh[a] - xch[a]) + (rxl[a] - xcl[a]);
                const float wp = (q1.z - wrh) + (q1.w - wrl);  // <= 0 up to rounding
                if (D == 3) {
                    const float A00 = ra[0], A01 = ra[1], A02 = ra[2], A11 = ra[3], A12 = ra[4], A22 = ra[5];
                    const float t0 = fmaf(A02, xp[2], fmaf(A01, xp[1], A00 * xp[0]));
                    const float t1 = fmaf(A12, xp[2], fmaf(A11, xp[1], A01 * xp[0]));
                    const float t2 = fmaf(A22, xp[2], fmaf(A12, xp[1], A02 * xp[0]));
                    phv[0] = A00;
                    phv[1] = 2.f * A01;
                    phv[2] = 2.f * A02;
                    phv[3] = A11;
                    phv[4] = 2.f * A12;
                    phv[5] = A22;
                    phv[6] = -2.f * t0;
                    phv[7] = -2.f * t1;
                    phv[8] = -2.f * t2;
                    phv[9] = fmaf(xp[2], t2, fmaf(xp[1], t1, xp[0] * t0)) - wp;
                } else {
                    const float A00 = ra[0], A01 = ra[1], A11 = ra[2];
                    const float t0 = fmaf(A01, xp[1], A00 * xp[0]);
                    const float t1 = fmaf(A11, xp[1], A01 * xp[0]);
                    phv[0] = A00;
                    phv[1] = 2.f * A01;
                    phv[2] = A11;
                    phv[3] = -2.f * t0;
                    phv[4] = -2.f * t1;
                    phv[5] = fmaf(xp[1], t1, xp[0] * t0) - wp;
                }
            } else {
                phv[G::F - 1] = 1e30f;  // padding seed: constant huge score
            }
            // this thread's half of the K features, one 16-byte core-matrix row per store
            constexpr int HALF = Fm::KT / 2;
            uint8_t *B = sm.B[q & 1];
#pragma unroll
            for (int ch = 0; ch < HALF / Fm::EPR; ++ch) {
                float e[Fm::EPR];
#pragma unroll
                for (int i = 0; i < Fm::EPR; ++i) e[i] = half ? phv[HALF + ch * Fm::EPR + i] : phv[ch * Fm::EPR + i];
                put_row<KIND>(B + cm_off(sl, half * HALF + ch * Fm::EPR, Fm::EB, Fm::EPR, Fm::LBO, Fm::SBO), e);
            }
            tc::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.bar_bfull[q & 1]);
            cur_next(c_xf);
        };
        if (xform)
            for (int q = 0; q < 2 && q < Q; ++q) transform(q);

        Cursor c_epi = cur_init(0);
        float s4[4] = {FLT_MAX, FLT_MAX, FLT_MAX, FLT_MAX};
        int i4[4] = {0, 0, 0, 0};
        for (int q = 0; q < Q; ++q) {
            const int b = q & 1;
            const int k = c_epi.k;
            // epilogue of step q
            const bool okw = wait(&sm.bar_acc[b], (uint32_t)((q >> 1) & 1));
            tc::fence_after_sync();
            if (okw) {
                const int base = chunk_id(c_epi) * kTcN;
#pragma unroll
                for (int h = 0; h < kTcN / 32; ++h) {
                    float v[32], gm;
                    // the reducing load returns the slice's smallest score with the scores
                    tc::tmem_ld32_min(taddr + lane_base + (uint32_t)((b * kTcTiles + mt) * kTcN + h * 32), v,
                                      gm);
                    tc::tmem_wait_ld();
                    if (h == kTcN / 32 - 1) {
                        // every score of the stage is in registers: the stage can be refilled
                        tc::fence_before_sync();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&sm.bar_aempty[b]);
                    }
                    if (__any_sync(0xffffffffu, gm < s4[3])) {
                        // minima of the 8-seed slices (3-input min), only when some pixel may improve
                        float m8[4];
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            m8[j] = fmin3_f(fmin3_f(v[8 * j], v[8 * j + 1], v[8 * j + 2]),
                                            fmin3_f(v[8 * j + 3], v[8 * j + 4], v[8 * j + 5]),
                                            fminf(v[8 * j + 6], v[8 * j + 7]));
                        // The slice minima are distinct scores, so the 4th smallest of {top-4} +
                        // {slice minima} bounds the new 4th-best from above: only values at or
                        // below it can enter (min/max network, branch free).
                        float t0 = s4[0], t1 = s4[1], t2 = s4[2], t3 = s4[3];
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            float x = m8[j], lo;
                            lo = fminf(t0, x); x = fmaxf(t0, x); t0 = lo;
                            lo = fminf(t1, x); x = fmaxf(t1, x); t1 = lo;
                            lo = fminf(t2, x); x = fmaxf(t2, x); t2 = lo;
                            t3 = fminf(t3, x);
                        }
                        const float thr = t3;
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            if (m8[j] <= thr) {
#pragma unroll
                                for (int i = 0; i < 8; ++i)
                                    if (v[8 * j + i] <= thr)
                                        top4_insert(s4, i4, v[8 * j + i], base + h * 32 + 8 * j + i);
                            }
                        }
                    }
                }
            } else {
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm.bar_aempty[b]);
            }
            if (k == n_chunks - 1) {
                // this thread's pixel of the tile is complete: hand its three best seeds
                // (scan positions) and fourth-best score to the resolve kernel
                const int tile = c_epi.tile;
                const int kb[3] = {(tile % ntx) * G::TX, ((tile / ntx) % nty) * G::TY,
                                   (tile / (ntx * nty)) * G::TZ};
                const int kk3[3] = {kb[0] + lx, kb[1] + ly, kb[2] + lz};
                if (kk3[0] < g.res[0] && kk3[1] < g.res[1] && (D == 2 || kk3[2] < g.res[2])) {
                    const long long j = (long long)kk3[0] +
                                        (long long)g.res[0] * ((long long)kk3[1] + (long long)g.res[1] * (long long)kk3[2]);
                    cand[j] = make_int4(i4[0], i4[1], i4[2], __float_as_int(s4[3]));
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    s4[i] = FLT_MAX;
                    i4[i] = 0;
                }
            }
            cur_next(c_epi);
            // B of step q + 2 (its buffer was read by the MMAs of step q, which completed)
            if (xform && q + 2 < Q) transform(q + 2);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(taddr, kTcCols);
}

// Resolve the tensor-core candidates: one thread per row of 16 pixels along the
// first axis.  For every pixel the three best seeds by tensor-core score are
// rescored in FP32 direct form with per-seed bounds (around the row's exact
// pixel-centre coordinates); the fourth-best score s4 certifies every other
// seed: its exact cost is at least s4 - psi, psi bounding the term magnitude of
// a seed of that cost from max ||A||_F, min lambda_min and the tensor-core tile
// radius.  Decided pixels get their label and enter the integer moments
// (run-length per row, shared hash table, one atomic per (cell, word));
// undecided pixels are queued for the full rescoring kernel.
constexpr int kResP = 16;
template <int D>
struct ResGeom;
template <>
struct ResGeom<3> {
    static constexpr int TY = 16, TZ = 16;
};
template <>
struct ResGeom<2> {
    static constexpr int TY = 256, TZ = 1;
};

template <int D>
__global__ void __launch_bounds__(256)
    tc_resolve_kernel(const GridDev g, const int n, const float R_tile, const float err_unit,
                      const int4 *__restrict__ cand, const int32_t *__restrict__ perm,
                      const SeedRec32 *__restrict__ r32, unsigned long long *__restrict__ gmom,
                      uint32_t *__restrict__ flags, int32_t *__restrict__ flag_gi, int32_t *__restrict__ labels,
                      DevScalars *__restrict__ sc) {
    using RG = ResGeom<D>;
    constexpr int KM = moment_width(D);
    __shared__ unsigned long long tval[kTcTable][KM];
    __shared__ int tkey[kTcTable];
    const int tid = threadIdx.x;
    for (int t = tid; t < kTcTable; t += blockDim.x) {
        tkey[t] = -1;
#pragma unroll
        for (int v = 0; v < KM; ++v) tval[t][v] = 0ull;
    }
    __syncthreads();
    const int k0b = blockIdx.x * kResP;
    const int k1 = blockIdx.y * RG::TY + tid % RG::TY;
    const int k2 = D == 3 ? blockIdx.z * RG::TZ + tid / RG::TY : 0;
    const bool row_valid = k1 < g.res[1] && (D == 2 || k2 < g.res[2]);
    const double wref = dkey_inv(sc->wref_key);
    float wrh, wrl;
    split2(wref, wrh, wrl);
    const float lam_abs = (float)__longlong_as_double((long long)sc->lam_abs_bits);
    const float inv_lam = 1.f / fmaxf((float)__longlong_as_double((long long)sc->lam_min_bits), 1e-30f);
    float ch[3] = {0.f, 0.f, 0.f}, cl[3] = {0.f, 0.f, 0.f};
    if (row_valid) {
        const int kc[3] = {k0b + kResP / 2, k1, k2};
        const double half[3] = {0.0, 0.5, 0.5};
#pragma unroll
        for (int a = 0; a < D; ++a) split2(g.lo[a] + ((double)kc[a] + half[a]) * g.h[a], ch[a], cl[a]);
    }
    const long long rowbase = (long long)g.res[0] * ((long long)k1 + (long long)g.res[1] * (long long)k2);
    const unsigned long long u1 = 2ull * (unsigned long long)k1 + 1ull;
    const unsigned long long u2 = 2ull * (unsigned long long)k2 + 1ull;
    int cur = -1;
    unsigned long long cnt = 0, s0 = 0, s00 = 0;
    auto moments_of = [&](unsigned long long c_, unsigned long long a_, unsigned long long b_,
                          unsigned long long (&val)[KM]) {
        if (D == 3) {
            val[0] = c_; val[1] = a_; val[2] = c_ * u1; val[3] = c_ * u2; val[4] = b_;
            val[5] = a_ * u1; val[6] = a_ * u2; val[7] = c_ * u1 * u1; val[8] = c_ * u1 * u2; val[9] = c_ * u2 * u2;
        } else {
            val[0] = c_; val[1] = a_; val[2] = c_ * u1; val[3] = b_; val[4] = a_ * u1; val[5] = c_ * u1 * u1;
        }
    };
    // runs of equal labels along the row: the first kRuns are summed across the
    // warp per label below (one set of shared atomics per label and warp), any
    // further ones go to the table at once
    constexpr int kRuns = 4;
    int rlab[kRuns];
    unsigned long long rcnt[kRuns], rs0[kRuns], rs00[kRuns];
#pragma unroll
    for (int q = 0; q < kRuns; ++q) {
        rlab[q] = -1;
        rcnt[q] = rs0[q] = rs00[q] = 0ull;
    }
    int nr = 0;
    auto flush = [&](int L) {
        if (nr < kRuns) {
#pragma unroll
            for (int q = 0; q < kRuns; ++q)
                if (q == nr) {
                    rlab[q] = L;
                    rcnt[q] = cnt;
                    rs0[q] = s0;
                    rs00[q] = s00;
                }
            ++nr;
        } else {
            unsigned long long val[KM];
            moments_of(cnt, s0, s00, val);
            tc_table_add<D>(tkey, tval, gmom, L, val);
        }
    };
    for (int p = 0; p < kResP; ++p) {
        const int k0 = k0b + p;
        int label = -1;
        if (row_valid && k0 < g.res[0]) {
            const long long j = rowbase + k0;
            const int4 cd = cand[j];
            const float yp[3] = {((float)(p - kResP / 2) + 0.5f) * g.h32[0], 0.f, 0.f};
            const int ids[3] = {cd.x, cd.y, cd.z};
            int orig[3];
            float cv[3], ev[3];
            int best = -1;
            bool queue = false;
#pragma unroll
            for (int qq = 0; qq < 3; ++qq) {
                int id = ids[qq];
                if (id >= 0 && id < n && perm) id = perm[id];
                orig[qq] = (id >= 0 && id < n) ? id : n;
                if (orig[qq] < n) {
                    cost32_bound_rel<D>(r32[orig[qq]], ch, cl, yp, wrh, wrl, cv[qq], ev[qq]);
                    if (best < 0 || cv[qq] < (best == 0 ? cv[0] : (best == 1 ? cv[1] : cv[2]))) best = qq;
                } else {
                    cv[qq] = FLT_MAX;
                    ev[qq] = 0.f;
                }
            }
            if (best < 0) {
                queue = true;
            } else {
                // the best candidate's values, selected without indexing by a run-time value
                const float cb = best == 0 ? cv[0] : (best == 1 ? cv[1] : cv[2]);
                const float eb = best == 0 ? ev[0] : (best == 1 ? ev[1] : ev[2]);
                const int ob = best == 0 ? orig[0] : (best == 1 ? orig[1] : orig[2]);
                const float U = cb + eb;
                const float s3 = __int_as_float(cd.w);
                float c_out = fabsf(s3);
                float r1 = 2.f * R_tile + sqrtf(c_out * inv_lam);
                float psi = err_unit * (lam_abs * r1 * r1 + c_out);
                c_out = fabsf(s3) + psi;
                r1 = 2.f * R_tile + sqrtf(c_out * inv_lam);
                psi = 1.1f * err_unit * (lam_abs * r1 * r1 + c_out);
                if (!(s3 - psi > U)) queue = true;
#pragma unroll
                for (int qq = 0; qq < 3; ++qq)
                    if (qq != best && orig[qq] < n && !(cv[qq] - ev[qq] > U)) queue = true;
                if (!queue) label = ob;
            }
            if (queue) {
                const unsigned slot = atomicAdd(&sc->flag_count, 1u);
                flags[slot] = (uint32_t)j;
                if (flag_gi) flag_gi[slot] = best == 0 ? orig[0] : (best == 1 ? orig[1] : (best == 2 ? orig[2] : -1));
            } else if (labels) {
                labels[j] = label;
            }
        }
        if (label != cur) {
            if (cur >= 0) flush(cur);
            cur = label;
            cnt = s0 = s00 = 0;
        }
        if (label >= 0) {
            const unsigned long long u0 = 2ull * (unsigned long long)k0 + 1ull;
            cnt += 1;
            s0 += u0;
            s00 += u0 * u0;
        }
    }
    if (cur >= 0) flush(cur);
    const int lane = tid & 31;
#pragma unroll
    for (int q = 0; q < kRuns; ++q) {
        const bool has = rlab[q] >= 0;
        unsigned todo = __ballot_sync(0xffffffffu, has);
        if (!todo) break;
        unsigned long long own[KM];
        moments_of(rcnt[q], rs0[q], rs00[q], own);
        while (todo) {
            const int leader = __ffs(todo) - 1;
            const int L0 = __shfl_sync(0xffffffffu, rlab[q], leader);
            const bool mine = has && rlab[q] == L0;
            const unsigned grp = __ballot_sync(0xffffffffu, mine);
            if (grp == (1u << leader)) {
                if (lane == leader) tc_table_add<D>(tkey, tval, gmom, L0, own);
            } else {
                unsigned long long sum[KM];
#pragma unroll
                for (int v = 0; v < KM; ++v) {
                    unsigned long long t = mine ? own[v] : 0ull;
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
                    sum[v] = t;
                }
                if (lane == leader) tc_table_add<D>(tkey, tval, gmom, L0, sum);
            }
            todo &= ~grp;
        }
    }
    __syncthreads();
    for (int t = tid; t < kTcTable; t += blockDim.x) {
        const int key = tkey[t];
        if (key >= 0) {
#pragma unroll
            for (int v = 0; v < KM; ++v) {
                const unsigned long long val = tval[t][v];
                if (val) atomicAdd(&gmom[(size_t)key * KM + v], val);
            }
        }
    }
}

template <int D, int KIND>
cudaError_t launch_tc_t(const GridDev &g, int n, Workspace &ws, int32_t *labels, unsigned long long *gmom,
                        cudaStream_t st) {
    using G = TcGeom<D>;
    const int ntx = (g.res[0] + G::TX - 1) / G::TX;
    const int nty = (g.res[1] + G::TY - 1) / G::TY;
    const int ntz = D == 3 ? (g.res[2] + G::TZ - 1) / G::TZ : 1;
    const long long ntl = (long long)ntx * nty * ntz;
    if (ntl > ws.tc_tile_cap) return cudaErrorInvalidValue;  // caller falls back (see launch_assign_tc)
    const int ntiles = (int)ntl;
    const int n_chunks = (n + kTcN - 1) / kTcN;
    // more than 114 KB of shared memory keeps one CTA (512 tensor-memory columns) per SM
    const size_t smem = sizeof(TcShared<D, KIND>) < 120 * 1024 ? 120 * 1024 : sizeof(TcShared<D, KIND>);
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(assign_tc_kernel<D, KIND>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const uint32_t *scodes = ws.sorted ? ws.scodes : nullptr;
    tc_tile_prep_kernel<D><<<(ntiles + 255) / 256, 256, 0, st>>>(g, ntx, nty, ntiles, n, n_chunks, scodes,
                                                                 ws.tc_centre, ws.tc_start);
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ws.device);
    const int grid = std::min(ntiles, sms);
    const double hx = 0.5 * G::TX * g.h[0], hy = 0.5 * G::TY * g.h[1], hz = D == 3 ? 0.5 * G::TZ * g.h[2] : 0.0;
    const float R = (float)(sqrt(hx * hx + hy * hy + hz * hz) * (1.0 + 1e-6));
    // per-score rounding: both operands (2 x 2^-11 TF32, 2 x 2^-9 BF16) plus ~100 FP32
    // roundings of the features and the accumulation, with a 1.5x margin
    const double u = 5.9604644775390625e-8;
    const double ein = KIND == tc::KIND_TF32 ? std::ldexp(1.0, -11) : std::ldexp(1.0, -9);
    const float err_unit = (float)(1.5 * (2.0 * ein + ein * ein + 100.0 * u));
    const SeedRec32 *rs = ws.sorted ? ws.recs32s : ws.recs32;
    assign_tc_kernel<D, KIND><<<grid, kTcThreadsAll, smem, st>>>(g, n, n_chunks, ntx, nty, ntiles, rs, ws.tc_centre,
                                                                 ws.tc_start, ws.tc_cand, ws.sc);
    const dim3 rgrid((g.res[0] + kResP - 1) / kResP, (g.res[1] + ResGeom<D>::TY - 1) / ResGeom<D>::TY,
                     D == 3 ? (g.res[2] + ResGeom<D>::TZ - 1) / ResGeom<D>::TZ : 1);
    tc_resolve_kernel<D><<<rgrid, ResGeom<D>::TY * ResGeom<D>::TZ, 0, st>>>(
        g, n, R, err_unit, ws.tc_cand, ws.sorted ? ws.perm : nullptr, ws.recs32, gmom, ws.flags, ws.flag_gi, labels,
        ws.sc);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_assign_tc(const GridDev &g, int n, Workspace &ws, int32_t *labels, unsigned long long *moments,
                             int kind, cudaStream_t st) {
    if (g.dim == 3)
        return kind == tc::KIND_TF32 ? launch_tc_t<3, tc::KIND_TF32>(g, n, ws, labels, moments, st)
                                     : launch_tc_t<3, tc::KIND_BF16>(g, n, ws, labels, moments, st);
    return kind == tc::KIND_TF32 ? launch_tc_t<2, tc::KIND_TF32>(g, n, ws, labels, moments, st)
                                 : launch_tc_t<2, tc::KIND_BF16>(g, n, ws, labels, moments, st);
}

long long tc_tile_count(const GridDev &g) {
    if (g.dim == 3)
        return (long long)((g.res[0] + TcGeom<3>::TX - 1) / TcGeom<3>::TX) * ((g.res[1] + TcGeom<3>::TY - 1) / TcGeom<3>::TY) *
               ((g.res[2] + TcGeom<3>::TZ - 1) / TcGeom<3>::TZ);
    return (long long)((g.res[0] + TcGeom<2>::TX - 1) / TcGeom<2>::TX) * ((g.res[1] + TcGeom<2>::TY - 1) / TcGeom<2>::TY);
}

}  // namespace apd
