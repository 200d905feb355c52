// Algorithm 1 on the 5th-generation tensor cores (tcgen05), fused with the
// per-cell integer moments.
//
// Expanded cost.  Around the centre c of a CTA tile, with y' = y - c and
// x' = x_i - c, the cost of eq. (2.1) relative to the largest weight w_ref is
//     C'_ij = f(y') . phi_i,   f = [y'_a y'_b (a <= b), y'_a, 1],
//     phi_i = [A_ab (x2 off the diagonal), -2 (A x')_a, x'^T A x' + (w_ref - w_i)]
// (10 features in 3D, 6 in 2D).  Both vectors are formed in FP32 and each is
// split into two operands of the tensor format, f = fh + fl (fl = the rounded
// remainder), and one contraction of K = 32 computes fh.phih + fl.phih +
// fh.phil with FP32 accumulation.  The dropped fl.phil and the remainders'
// roundings leave about 3 e^2 |f_k phi_k| per feature (e = 2^-11 for TF32,
// 2^-8 for BF16), so a score is within err_unit * sum_k |f_k phi_k| of the
// exact cost, err_unit ~ 1e-4 (BF16) / 3e-5 (TF32) with the FP32 work, the
// accumulation and the packed index below included.
//
// Candidate lists (pruned form).  A pre-pass gives every 512-pixel CTA tile
// the seeds that can matter there: with rigorous FP32 bounds over the box of
// the tile's pixel centres, LB_i <= C'_i <= UB_i (the better of an eigenvalue
// form, lambda_min,i dist(x_i, box)^2 and lambda_max,i maxdist(x_i, box)^2,
// and a centre form around the box centre; plus w_ref - w_i), and T the
// fourth smallest UB_i, the list holds the seeds with LB_i <= T.  One kernel
// does it per super-tile of 2 x 2 (x 2) tiles: eight warps visit the 32-seed
// Morton groups in increasing order of their group bound for the super-tile's
// box, then each warp narrows the super-tile's list for one tile and stores
// the tile's list and split seed operands.  T_excl = the smallest LB of every
// seed left out is a lower bound of every excluded seed's cost at every pixel
// of the tile.  The dense form takes all seeds, in 32-seed chunks zig-zagging
// out from the tile's Morton position.
//
// Pipeline (one persistent CTA per SM, warp-specialised).  A CTA tile is four
// M = 128 tiles (one tensor-memory lane per pixel); a step scores 32 seeds of
// the tile's list: the seed operand B (32 x 32, recentred and split) is the
// stored one of the pruned form, brought in by a 1-D bulk copy, or built from
// the FP32 seed records by two transform warps (dense form); one thread issues the MMAs
// (4 M tiles x K = 32) into one of four accumulator stages (4 x 4 x 32 = 512
// tensor-memory columns), and sixteen epilogue warps (thread = pixel) read the
// stage with the min-reducing tensor-memory load, release it, and fold the 32
// scores into the pixel's two smallest (packed: the step-local index in the
// five low mantissa bits) unless the slice minimum cannot enter them.
//
// Certificate.  At the end of a tile, with s1 <= s2 the two smallest scores
// and psi(s) = the bound above for a seed scoring s (the term sum bounded by
// max ||A||_F (2R + sqrt(C/lambda_min))^2 + C, R the tile half-diagonal),
// the label is the best seed when U = s1 + psi(s1) < s2 - psi(s2) and
// U < T_excl: every other candidate and every excluded seed then costs more
// than the best one.  Other pixels go to the FP64 rescoring queue (with the
// best seed as the threshold hint), which settles them with the reference
// arithmetic (pixels the scores leave undecided are first settled in FP32
// direct form by the warp over the tile's candidate list).  Certified pixels
// enter the integer moments in the epilogue: the lanes of a warp holding the
// same label sum their moments (32-bit warp reductions; the last axis's
// coordinate is uniform over a warp), and lanes 0 .. K-1 add the K words to
// the global int64 moments.
#include <cuda_bf16.h>
#include <float.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "apd_cost.cuh"
#include "apd_internal.cuh"
#include "apd_tcgen05.cuh"

namespace apd {

namespace {

constexpr int kN = 32;                       // seeds per step (MMA N)
constexpr int kM = 128;                      // pixels per M tile
constexpr int kMT = 4;                       // M tiles per CTA tile
constexpr int kPix = kMT * kM;               // 512 pixels per CTA tile
constexpr int kStages = 4;                   // accumulator stages
constexpr uint32_t kCols = kStages * kMT * kN;  // 512 tensor-memory columns
constexpr int kK = 32;                       // split operand width: [fh | fl | fh] . [ph | ph | pl]
constexpr int kEpiWarps = kPix / 32;         // 16
constexpr int kProdWarp = kEpiWarps;         // warp 16: MMA issue
constexpr int kXfWarp0 = kEpiWarps + 1;      // warps 17, 18: seed operands
constexpr int kXfWarps = 2;
constexpr int kThreads = (kEpiWarps + 1 + kXfWarps) * 32;  // 608
constexpr int kListCap = 128;                // candidate seeds stored per tile
constexpr int kMaxSteps = kListCap / kN;     // steps of a pruned tile (B operands stored per tile)
constexpr int kBandChunk = 2048;             // pixels per block step of the re-decision kernel
constexpr int kAhead = 2;                    // pruned form: bulk copies issued ahead of the MMAs
constexpr int kBMax = kN * kK * 4;           // bytes of one stored B operand (TF32; BF16 uses half)

template <int D>
struct TcGeom;
template <>
struct TcGeom<3> {
    static constexpr int TX = 8, TY = 8, TZ = 8, F = 10;
};
template <>
struct TcGeom<2> {
    static constexpr int TX = 32, TY = 16, TZ = 1, F = 6;
};

template <int KIND>
struct TcFmt {
    static constexpr int EB = KIND == tc::KIND_TF32 ? 4 : 2;      // bytes per element
    static constexpr int EPR = 16 / EB;                           // elements per core-matrix row
    static constexpr int KSTEP = KIND == tc::KIND_TF32 ? 8 : 16;  // K of one MMA
    static constexpr int STEPS = kK / KSTEP;
    static constexpr uint32_t LBO = 128;                          // K-adjacent core matrices
    static constexpr uint32_t SBO = (kK / EPR) * 128;             // next 8-row group
    static constexpr int A_BYTES = kM * kK * EB;
    static constexpr int B_BYTES = kN * kK * EB;
};

template <int D, int KIND>
struct TcShared {
    alignas(1024) uint8_t A[kMT][TcFmt<KIND>::A_BYTES];
    alignas(1024) uint8_t B[kStages][TcFmt<KIND>::B_BYTES];
    uint64_t bar_bfull[kStages];   // B operand built (the transform warps)
    uint64_t bar_acc[kStages];     // accumulator stage written (MMA commit)
    uint64_t bar_aempty[kStages];  // accumulator stage read (the epilogue warps)
    uint32_t tslot;
    int abort;
};

// one 16-byte core-matrix row of operand values, rounded to the operand format
template <int KIND>
__device__ __forceinline__ void put_row(uint8_t *dst, const float *e) {
    if (KIND == tc::KIND_TF32) {
        *reinterpret_cast<float4 *>(dst) = make_float4(e[0], e[1], e[2], e[3]);
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

// the operand-format value nearest to v (exactly representable afterwards)
template <int KIND>
__device__ __forceinline__ float rnd_op(float v) {
    if (KIND == tc::KIND_TF32) return tc::to_tf32(v);
    return __bfloat162float(__float2bfloat16_rn(v));
}

// split row: [vh | vl | vh] (A side, pixels) or [vh | vh | vl] (B side, seeds), zero padded
template <int F, int KIND, bool kSeed>
__device__ __forceinline__ void split_row(const float (&v)[F], float (&row)[kK]) {
#pragma unroll
    for (int k = 0; k < kK; ++k) row[k] = 0.f;
#pragma unroll
    for (int k = 0; k < F; ++k) {
        const float h = rnd_op<KIND>(v[k]);
        const float l = rnd_op<KIND>(v[k] - h);  // the remainder v - h is exact in FP32
        row[k] = h;
        row[F + k] = kSeed ? h : l;
        row[2 * F + k] = kSeed ? l : h;
    }
}

// Seed features of record r relative to the tile centre ch + cl (FP32 split):
// [A_ab (x2 off the diagonal), -2 (A x')_a, x'^T A x' - (w - w_ref)].
template <int D>
__device__ __forceinline__ void seed_features(const float4 q0, const float4 q1, const float4 q2, const float4 q3,
                                              const float (&ch)[3], const float (&cl)[3], float wrh, float wrl,
                                              float (&ph)[TcGeom<D>::F]) {
    const float rxh[3] = {q0.x, q0.y, q0.z}, rxl[3] = {q0.w, q1.x, q1.y};
    const float ra[6] = {q2.x, q2.y, q2.z, q2.w, q3.x, q3.y};
    float xp[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int d = 0; d < D; ++d) xp[d] = (rxh[d] - ch[d]) + (rxl[d] - cl[d]);
    const float wp = (q1.z - wrh) + (q1.w - wrl);  // w_i - w_ref <= 0 up to rounding
    if (D == 3) {
        const float A00 = ra[0], A01 = ra[1], A02 = ra[2], A11 = ra[3], A12 = ra[4], A22 = ra[5];
        const float t0 = fmaf(A02, xp[2], fmaf(A01, xp[1], A00 * xp[0]));
        const float t1 = fmaf(A12, xp[2], fmaf(A11, xp[1], A01 * xp[0]));
        const float t2 = fmaf(A22, xp[2], fmaf(A12, xp[1], A02 * xp[0]));
        ph[0] = A00;
        ph[1] = 2.f * A01;
        ph[2] = 2.f * A02;
        ph[3] = A11;
        ph[4] = 2.f * A12;
        ph[5] = A22;
        ph[6] = -2.f * t0;
        ph[7] = -2.f * t1;
        ph[8] = -2.f * t2;
        ph[9] = fmaf(xp[2], t2, fmaf(xp[1], t1, xp[0] * t0)) - wp;
    } else {
        const float A00 = ra[0], A01 = ra[1], A11 = ra[2];
        const float t0 = fmaf(A01, xp[1], A00 * xp[0]);
        const float t1 = fmaf(A11, xp[1], A01 * xp[0]);
        ph[0] = A00;
        ph[1] = 2.f * A01;
        ph[2] = A11;
        ph[3] = -2.f * t0;
        ph[4] = -2.f * t1;
        ph[5] = fmaf(xp[1], t1, xp[0] * t0) - wp;
    }
}

// The split operand row of one seed slot (padding: a huge constant score).
template <int D, int KIND>
__device__ __forceinline__ void seed_row(const SeedRec32 *__restrict__ recs, const int pos, const float (&ch)[3],
                                         const float (&cl)[3], float wrh, float wrl, float (&row)[kK]) {
    constexpr int F = TcGeom<D>::F;
    float ph[F];
#pragma unroll
    for (int e = 0; e < F; ++e) ph[e] = 0.f;
    if (pos >= 0) {
        const float4 *rv = reinterpret_cast<const float4 *>(recs + pos);
        seed_features<D>(__ldg(rv), __ldg(rv + 1), __ldg(rv + 2), __ldg(rv + 3), ch, cl, wrh, wrl, ph);
    } else {
        ph[F - 1] = 1e30f;
    }
    split_row<F, KIND, true>(ph, row);
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
// The reference weight's FP32 split, formed once per block (FP64 instructions
// issue slowly; a per-warp conversion showed in the pre-pass kernels' time).
// Every thread of the block calls it, before any early exit.
__device__ __forceinline__ void block_wref(const DevScalars *__restrict__ sc, float &wrh, float &wrl) {
    __shared__ float sw[2];
    if (threadIdx.x == 0) split2(dkey_inv(sc->wref_key), sw[0], sw[1]);
    __syncthreads();
    wrh = sw[0];
    wrl = sw[1];
}

__device__ __forceinline__ unsigned okey(float v) {  // order-preserving float -> unsigned
    const unsigned u = __float_as_uint(v);
    return u ^ ((u >> 31) ? 0xffffffffu : 0x80000000u);
}
__device__ __forceinline__ float okey_inv(unsigned k) {
    return __uint_as_float(k ^ ((k >> 31) ? 0x80000000u : 0xffffffffu));
}


// Tile t of the scoring window -> its first pixel per axis.
template <int D>
__device__ __forceinline__ void tile_origin(int t, int ntx, int nty, int tlo, int (&kb)[3]) {
    using G = TcGeom<D>;
    const int tx = t % ntx, r = t / ntx;
    if (D == 3) {
        kb[0] = tx * G::TX;
        kb[1] = (r % nty) * G::TY;
        kb[2] = (r / nty + tlo) * G::TZ;
    } else {
        kb[0] = tx * G::TX;
        kb[1] = (r + tlo) * G::TY;
        kb[2] = 0;
    }
}

// Per-axis tile data, FP64 once per tile coordinate: for coordinate c along
// axis a (table entry off_a + c, off = 0, ntx, ntx + nty), the FP32 split of
// the tile centre lo + (kb + T/2) h and the absolute box of the tile's valid
// pixel centres rounded outwards.
template <int D>
__global__ void __launch_bounds__(256)
    tc_axis_kernel(const GridDev g, const int ntx, const int nty, const int ntz, const int tlo,
                   float4 *__restrict__ tab) {
    using G = TcGeom<D>;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    int a, c;
    if (i < ntx) {
        a = 0;
        c = i;
    } else if (i < ntx + nty) {
        a = 1;
        c = i - ntx;
    } else if (D == 3 && i < ntx + nty + ntz) {
        a = 2;
        c = i - ntx - nty;
    } else {
        return;
    }
    const int td = a == 0 ? G::TX : (a == 1 ? G::TY : G::TZ);
    const bool last = a == D - 1;
    const int kb = (c + (last ? tlo : 0)) * td;
    const int resa = a == 0 ? g.res[0] : (a == 1 ? g.res[1] : g.res[2]);
    const int hi = last ? win_hi(g) : resa;
    const int khi = min(kb + td, hi) - 1;
    const double lo = a == 0 ? g.lo[0] : (a == 1 ? g.lo[1] : g.lo[2]);
    const double h = a == 0 ? g.h[0] : (a == 1 ? g.h[1] : g.h[2]);
    float ch, cl;
    split2(lo + (double)(kb + td / 2) * h, ch, cl);
    tab[i] = make_float4(ch, cl, __double2float_rd(lo + ((double)kb + 0.5) * h),
                         __double2float_ru(lo + ((double)khi + 0.5) * h));
}

// ---------------------------------------------------------------------------
// Dense-form pre-pass: one warp per tile writes the tile centre (FP32 high/low
// split) and the Morton start chunk of the tile's zig-zag seed scan.
// ---------------------------------------------------------------------------
template <int D, int KIND>
__global__ void __launch_bounds__(256)
    tc_tile_kernel(const GridDev g, const int ntx, const int nty, const int tlo, const int ntiles, const int n,
                   const SeedRec32 *__restrict__ r32, const GroupBound *__restrict__ groups,
                   const uint32_t *__restrict__ scodes, const int32_t *__restrict__ perm, const int n_chunks,
                   float *__restrict__ centre, int *__restrict__ start, int4 *__restrict__ meta,
                   float *__restrict__ texcl, int *__restrict__ list, uint8_t *__restrict__ bops,
                   const float4 *__restrict__ axis_tab, const DevScalars *__restrict__ sc) {
    using Fm = TcFmt<KIND>;
    using G = TcGeom<D>;
    const int lane = threadIdx.x & 31;
    const int t = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    float wrh, wrl;
    block_wref(sc, wrh, wrl);
    if (t >= ntiles) return;
    int kb[3];
    tile_origin<D>(t, ntx, nty, tlo, kb);
    const int td[3] = {G::TX, G::TY, G::TZ};
    float ch[3] = {0.f, 0.f, 0.f}, cl[3] = {0.f, 0.f, 0.f};
    double frac[3] = {0.0, 0.0, 0.0};
    // valid pixels of the tile: inside the grid and (last axis) the window
    int khi[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (a < D) {
            const int hi = a == D - 1 ? win_hi(g) : g.res[a];
            khi[a] = min(kb[a] + td[a], hi) - 1;
            // the Morton position only orders the scan: FP32 is enough
            frac[a] = (double)(((float)(kb[a] + td[a] / 2) + 0.5f) / (float)g.res[a]);
        }
    }
    // the tile centre and the absolute pixel box, per axis from the table
    float alo[3] = {0.f, 0.f, 0.f}, ahi[3] = {0.f, 0.f, 0.f};
    {
        const int tx = t % ntx, r = t / ntx;
        const int idx[3] = {tx, ntx + (D == 3 ? r % nty : r), ntx + nty + (D == 3 ? r / nty : 0)};
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const float4 e = axis_tab[idx[a]];
            ch[a] = e.x;
            cl[a] = e.y;
            alo[a] = e.z;
            ahi[a] = e.w;
        }
    }
    if (lane < 6) centre[(size_t)t * 6 + lane] = lane < 3 ? ch[lane] : cl[lane - 3];
    uint32_t code = 0u;
    int spos = 0;  // scan position of the tile centre's Morton code (needed with several blocks of groups)
    if (scodes && (list == nullptr || n > 1024)) {
        code = morton_code(D, frac);
        int lo = 0, hi = n;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (scodes[mid] < code) lo = mid + 1;
            else hi = mid;
        }
        spos = min(lo, n - 1);
    }
    if (lane == 0) {
        start[t] = spos / kN;
        meta[t] = make_int4(kb[0], kb[1], kb[2], 0);
    }
}

// Lower bound of the costs of the seeds of group gb over an absolute box of
// pixel centres [alo, ahi] (FP32 rounded outwards).
template <int D>
__device__ __forceinline__ float group_lower(const GroupBound &gb, const float (&alo)[3], const float (&ahi)[3]) {
    float d2 = 0.f;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const float slack = 1e-6f * (fabsf(alo[a]) + fabsf(ahi[a]) + fabsf(gb.lo[a]) + fabsf(gb.hi[a]));
        const float q = fmaxf(fmaxf(gb.lo[a] - ahi[a], alo[a] - gb.hi[a]) - slack, 0.f);
        d2 = __fmaf_rd(q, q, d2);
    }
    return __fadd_rd(__fmul_rd(__fmul_rd(gb.lam, d2), 1.f - 1e-5f), gb.wgap);
}

// Lower and upper bounds of seed r's costs (relative to w_ref) over the box
// [rlo, rhi] of pixel centres given relative to the centre ch + cl, the better
// of two forms for each:
//  - eigenvalue form: lambda_min dist(x, box)^2 and lambda_max maxdist(x, box)^2;
//  - centre form: with d = c - x (c the box centre) and e = y - c, |e_a| <= r_a,
//    (y - x)^T A (y - x) = d^T A d + 2 (A d).e + e^T A e lies within
//    q -/+ 2 sum_a |(A d)_a| r_a (+ sum_ab |A_ab| r_a r_b above), q = d^T A d;
//    tight for anisotropic A, where the eigenvalue form is off by up to the
//    condition number.
// The position slack widens r (it covers the FP32 offsets as in the eigenvalue
// form); E = 1e-5 S, S = sum_ab |A_ab| (|d_a| + r_a)(|d_b| + r_b), covers the
// FP32 rounding of q and of the linear term and the FP32 storage of A (about
// 20 roundings of at most 2^-24 S each).  Only the lower bound decides
// correctness (a seed left out costs at least its lower bound); the upper
// bound only sets how short the lists are.
template <int D>
__device__ __forceinline__ void seed_bounds(const SeedRec32 &r, const float (&ch)[3], const float (&cl)[3],
                                            const float (&rlo)[3], const float (&rhi)[3], float wrh, float wrl,
                                            float &lb, float &ub) {
    float d2lo = 0.f, d2hi = 0.f;
    float dv[3] = {0.f, 0.f, 0.f}, rr[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const float xs = (r.xh[a] - ch[a]) + (r.xl[a] - cl[a]);
        const float slack = 1e-6f * (fabsf(rlo[a]) + fabsf(rhi[a]) + 2.f * fabsf(xs)) + 1e-30f;
        const float dl = fmaxf(fmaxf(xs - rhi[a], rlo[a] - xs) - slack, 0.f);
        const float dh = fmaxf(fabsf(xs - rlo[a]), fabsf(xs - rhi[a])) + slack;
        d2lo = __fmaf_rd(dl, dl, d2lo);
        d2hi = __fmaf_ru(dh, dh, d2hi);
        dv[a] = 0.5f * (rlo[a] + rhi[a]) - xs;
        rr[a] = 0.5f * (rhi[a] - rlo[a]) + slack;
    }
    const float wn = -((r.wh - wrh) + (r.wl - wrl));  // w_ref - w_i, up to rounding
    const float wslack = 1e-6f * fabsf(wn) + 1e-30f;
    const float lb1 = __fadd_rd(__fmul_rd(__fmul_rd(r.pad[0], d2lo), 1.f - 1e-5f), __fsub_rd(wn, wslack));
    const float ub1 = __fadd_ru(__fmul_ru(__fmul_ru(r.pad[1], d2hi), 1.f + 1e-5f), __fadd_ru(wn, wslack));
    // the symmetric matrix from the record (upper triangle, row order)
    float M[3][3];
    if (D == 3) {
        M[0][0] = r.a[0];
        M[0][1] = M[1][0] = r.a[1];
        M[0][2] = M[2][0] = r.a[2];
        M[1][1] = r.a[3];
        M[1][2] = M[2][1] = r.a[4];
        M[2][2] = r.a[5];
    } else {
        M[0][0] = r.a[0];
        M[0][1] = M[1][0] = r.a[1];
        M[1][1] = r.a[2];
        M[0][2] = M[2][0] = M[1][2] = M[2][1] = M[2][2] = 0.f;
    }
    float q = 0.f, lin = 0.f, quad = 0.f, S = 0.f;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        float ga = 0.f, qa = 0.f, sa = 0.f;
#pragma unroll
        for (int b = 0; b < D; ++b) {
            ga = fmaf(M[a][b], dv[b], ga);
            qa = fmaf(fabsf(M[a][b]), rr[b], qa);
            sa = fmaf(fabsf(M[a][b]), fabsf(dv[b]) + rr[b], sa);
        }
        q = fmaf(dv[a], ga, q);
        lin = fmaf(fabsf(ga), rr[a], lin);
        quad = fmaf(qa, rr[a], quad);
        S = fmaf(sa, fabsf(dv[a]) + rr[a], S);
    }
    lin = 2.f * lin;
    const float E = 1e-5f * S + 1e-30f;
    const float lb2 = __fadd_rd(__fsub_rd(__fsub_rd(q, lin), E), __fsub_rd(wn, wslack));
    const float ub2 = __fadd_ru(__fadd_ru(__fadd_ru(q, lin), __fadd_ru(quad, E)), __fadd_ru(wn, wslack));
    lb = fmaxf(lb1, lb2);
    ub = fminf(ub1, ub2);
}

// Merge the smallest four of the warp's 32 keys (one per lane) into the
// warp-uniform ascending four smallest values u0 <= u1 <= u2 <= u3.
__device__ __forceinline__ void merge_smallest4(unsigned ku, float &u0, float &u1, float &u2, float &u3) {
    const int lane = threadIdx.x & 31;
    if (!(__reduce_min_sync(0xffffffffu, ku) < okey(u3))) return;
    float b[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const unsigned m = __reduce_min_sync(0xffffffffu, ku);
        b[e] = m == 0xffffffffu ? __int_as_float(0x7f800000) : okey_inv(m);
        const int l = __ffs(__ballot_sync(0xffffffffu, ku == m)) - 1;
        if (lane == l) ku = 0xffffffffu;
    }
    // the four smallest of two ascending lists of four: the elementwise minima of
    // one list against the other reversed, then sorted
    float c0 = fminf(u0, b[3]), c1 = fminf(u1, b[2]), c2 = fminf(u2, b[1]), c3 = fminf(u3, b[0]);
    auto cswap = [](float &x, float &y) {
        const float lo = fminf(x, y), hi = fmaxf(x, y);
        x = lo;
        y = hi;
    };
    cswap(c0, c2);
    cswap(c1, c3);
    cswap(c0, c1);
    cswap(c2, c3);
    cswap(c1, c2);
    u0 = c0;
    u1 = c1;
    u2 = c2;
    u3 = c3;
}

// Pruned form, step 1: one block of eight warps per super-tile of 2 x 2 (x 2)
// tiles finds the candidates of the super-tile's box (groups visited by
// increasing bound, shared out among the warps; the threshold is the fourth
// smallest upper bound, then the seeds with a lower bound below it) and T_excl.  A seed left out there is left out of each tile
// too: its bound over a sub-box is at least its bound over the box.
constexpr int kSuperCap = 256;

// Tile-coordinate range of a super-tile, and the box of a tile range [ca, cb]:
// centre of tile ca (FP32 split), pixel box relative to it and absolute.
struct SuperGeom {
    int ntx, nty, ntz, tlo;
};
template <int D>
__device__ __forceinline__ void super_range(const SuperGeom &sg, int sup, int (&c0)[3], int (&c1)[3]) {
    const int nsx = (sg.ntx + 1) / 2, nsy = (sg.nty + 1) / 2;
    const int sx = sup % nsx, rr = sup / nsx;
    const int sy = rr % nsy, sz = D == 3 ? rr / nsy : 0;
    c0[0] = 2 * sx;
    c0[1] = 2 * sy;
    c0[2] = 2 * sz;
    c1[0] = min(2 * sx + 1, sg.ntx - 1);
    c1[1] = min(2 * sy + 1, sg.nty - 1);
    c1[2] = D == 3 ? min(2 * sz + 1, sg.ntz - 1) : 0;
}
template <int D>
__device__ __forceinline__ void range_box(const GridDev &g, const SuperGeom &sg, const float4 *__restrict__ axis_tab,
                                          const int (&ca)[3], const int (&cb)[3], float (&ch)[3], float (&cl)[3],
                                          float (&rlo)[3], float (&rhi)[3], float (&alo)[3], float (&ahi)[3]) {
    using G = TcGeom<D>;
    const int td[3] = {G::TX, G::TY, G::TZ};
    const int toff[3] = {0, sg.ntx, sg.ntx + sg.nty};
    const int tl[3] = {0, D == 2 ? sg.tlo : 0, D == 3 ? sg.tlo : 0};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        ch[a] = cl[a] = rlo[a] = rhi[a] = alo[a] = ahi[a] = 0.f;
        if (a < D) {
            const float4 ea = axis_tab[toff[a] + ca[a]], eb = axis_tab[toff[a] + cb[a]];
            ch[a] = ea.x;
            cl[a] = ea.y;
            alo[a] = ea.z;
            ahi[a] = eb.w;
            const int kb = (ca[a] + tl[a]) * td[a];
            const int hi = a == D - 1 ? win_hi(g) : g.res[a];
            const int khi = min((cb[a] + tl[a]) * td[a] + td[a], hi) - 1;
            const int cc = kb + td[a] / 2;
            rlo[a] = ((float)(kb - cc) + 0.5f) * g.h32[a];
            rhi[a] = ((float)(khi - cc) + 0.5f) * g.h32[a];
        }
    }
}

// Pruned form, step 2 (in the same kernel, one warp per tile of the
// super-tile): the warp narrows the super-tile's list with the tile's own
// bounds (the fourth smallest upper bound over the tile), sets T_excl = min(the
// super-tile's, the bounds of the seeds it drops), and stores its list (seed
// indices) and split seed operands.  sl: the super-tile's list (shared memory).
template <int D, int KIND>
__device__ __forceinline__ void tile_list(const GridDev &g, const SuperGeom &sg, const int t, const int (&tc3)[3],
                                          const SeedRec32 *__restrict__ r32, const int32_t *__restrict__ perm,
                                          const float4 *__restrict__ axis_tab, const int *sl, const int cntS,
                                          const float tex_sup, float *__restrict__ centre, int4 *__restrict__ meta,
                                          float *__restrict__ texcl, int *__restrict__ list, uint8_t *__restrict__ bops,
                                          const float wrh, const float wrl) {
    using G = TcGeom<D>;
    using Fm = TcFmt<KIND>;
    const int lane = threadIdx.x & 31;
    const float finf = __int_as_float(0x7f800000);
    float ch[3], cl[3], rlo[3], rhi[3], alo[3], ahi[3];
    range_box<D>(g, sg, axis_tab, tc3, tc3, ch, cl, rlo, rhi, alo, ahi);
    if (lane < 6) centre[(size_t)t * 6 + lane] = lane < 3 ? ch[lane] : cl[lane - 3];
    // the tile's bounds of the super-tile's candidates: at most 8 rounds of 32,
    // taken two at a time (indices, then records, loaded together)
    float lbv[kSuperCap / 32];
    float u0 = finf, u1 = finf, u2 = finf, u3 = finf;
    const SeedRec32 zrec{};
#pragma unroll
    for (int r = 0; r < kSuperCap / 32; r += 2) {
        lbv[r] = lbv[r + 1] = finf;
        if (r * 32 < cntS) {
            const int e0 = r * 32 + lane, e1 = e0 + 32;
            const int i0 = e0 < cntS ? sl[e0] : -1, i1 = e1 < cntS ? sl[e1] : -1;
            const SeedRec32 q0 = i0 >= 0 ? r32[i0] : zrec;
            const SeedRec32 q1 = i1 >= 0 ? r32[i1] : zrec;
            float ub0 = finf, ub1 = finf;
            if (i0 >= 0) seed_bounds<D>(q0, ch, cl, rlo, rhi, wrh, wrl, lbv[r], ub0);
            if (i1 >= 0) seed_bounds<D>(q1, ch, cl, rlo, rhi, wrh, wrl, lbv[r + 1], ub1);
            merge_smallest4(i0 >= 0 ? okey(ub0) : 0xffffffffu, u0, u1, u2, u3);
            if ((r + 1) * 32 < cntS) merge_smallest4(i1 >= 0 ? okey(ub1) : 0xffffffffu, u0, u1, u2, u3);
        }
    }
    const float T = u3;
    float tex = tex_sup;
    int cnt = 0;
#pragma unroll
    for (int r = 0; r < kSuperCap / 32; ++r) {
        if (r * 32 < cntS) {
            const int e = r * 32 + lane;
            const bool cand = e < cntS && lbv[r] <= T;
            const unsigned cm = __ballot_sync(0xffffffffu, cand);
            const int rank = __popc(cm & ((1u << lane) - 1u));
            if (cand) {
                if (cnt + rank < kListCap) list[(size_t)t * kListCap + cnt + rank] = sl[e];
                else tex = fminf(tex, lbv[r]);
            } else if (e < cntS) {
                tex = fminf(tex, lbv[r]);
            }
            cnt += __popc(cm);
        }
    }
    tex = okey_inv(__reduce_min_sync(0xffffffffu, okey(tex)));
    const int cnt_c = min(cnt, kListCap);
    if (lane == 0) {
        const int td[3] = {G::TX, G::TY, G::TZ};
        const int tl[3] = {0, D == 2 ? sg.tlo : 0, D == 3 ? sg.tlo : 0};
        int kb[3] = {0, 0, 0};
#pragma unroll
        for (int a = 0; a < D; ++a) kb[a] = (tc3[a] + tl[a]) * td[a];
        meta[t] = make_int4(kb[0], kb[1], kb[2], cnt_c);
        texcl[t] = tex;
    }
    __syncwarp();  // the list entries written by the other lanes
    const int ns = max(1, (cnt_c + kN - 1) / kN);
    for (int k = 0; k < ns; ++k) {
        const int slot = k * kN + lane;
        const int pos = slot < cnt_c ? list[(size_t)t * kListCap + slot] : -1;
        float row[kK];
        seed_row<D, KIND>(r32, pos, ch, cl, wrh, wrl, row);
        uint8_t *dst = bops + ((size_t)t * kMaxSteps + k) * Fm::B_BYTES;
#pragma unroll
        for (int c = 0; c < kK / Fm::EPR; ++c)
            put_row<KIND>(dst + tc::core_offset(lane, c * Fm::EPR, Fm::EB, Fm::LBO, Fm::SBO), row + c * Fm::EPR);
        if (pos >= 0) list[(size_t)t * kListCap + slot] = perm ? perm[pos] : pos;  // seed index for the labels
    }
}

constexpr int kSupWarps = 8;  // warps sharing one super-tile's scan

template <int D, int KIND>
__global__ void __launch_bounds__(kSupWarps * 32)
    tc_lists_kernel(const GridDev g, const SuperGeom sg, const int nsup, const int n,
                    const SeedRec32 *__restrict__ r32, const int32_t *__restrict__ perm,
                    const GroupBound *__restrict__ groups, const uint32_t *__restrict__ scodes,
                    const float4 *__restrict__ axis_tab, float *__restrict__ centre, int4 *__restrict__ meta,
                    float *__restrict__ texcl, int *__restrict__ list, uint8_t *__restrict__ bops,
                    const DevScalars *__restrict__ sc, const int *__restrict__ skip) {
    using G = TcGeom<D>;
    constexpr int W = kSupWarps;
    if (skip && *(volatile const int *)skip) return;  // an incremental re-decision keeps the lists
    __shared__ unsigned s_T;                 // okey of the smallest threshold found so far
    __shared__ float s_u[W][4];              // each warp's four smallest upper bounds
    __shared__ int s_pos[W][kSuperCap];      // each warp's candidates (scan positions) ...
    __shared__ float s_lb[W][kSuperCap];     // ... and their lower bounds
    __shared__ int s_cnt[W];
    __shared__ float s_tex[W], s_tex2[W];
    __shared__ int s_list[kSuperCap];        // the super-tile's list, warp order
    __shared__ int s_total;
    __shared__ float s_texs;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int sup = (int)blockIdx.x;
    float wrh, wrl;
    block_wref(sc, wrh, wrl);
    if (sup >= nsup) return;  // uniform over the block
    const float finf = __int_as_float(0x7f800000);
    if (threadIdx.x == 0) s_T = okey(finf);
    int c0[3], c1[3];
    super_range<D>(sg, sup, c0, c1);
    float ch[3], cl[3], rlo[3], rhi[3], alo[3], ahi[3];
    range_box<D>(g, sg, axis_tab, c0, c1, ch, cl, rlo, rhi, alo, ahi);
    const int n_groups = (n + 31) / 32;
    const int n_blocks = (n_groups + 31) / 32;
    int bstart = 0;
    if (scodes && n_blocks > 1) {
        const int td[3] = {G::TX, G::TY, G::TZ};
        const int tl[3] = {0, D == 2 ? sg.tlo : 0, D == 3 ? sg.tlo : 0};
        double frac[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int a = 0; a < D; ++a)
            frac[a] = (double)(((float)((c0[a] + tl[a]) * td[a] + td[a]) + 0.5f) / (float)g.res[a]);
        const uint32_t code = morton_code(D, frac);
        int lo = 0, hi = n;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (scodes[mid] < code) lo = mid + 1;
            else hi = mid;
        }
        bstart = min(min(lo, n - 1) / 1024, n_blocks - 1);
    }
    auto block_of = [&](int bi) {
        const int off = (bi & 1) ? ((bi + 1) >> 1) : -(bi >> 1);
        int blk = bstart + off;
        if (blk >= n_blocks) blk -= n_blocks;
        if (blk < 0) blk += n_blocks;
        return blk;
    };
    const SeedRec32 zrec{};
    __syncthreads();  // s_T set
    // Pass 1: T = the fourth smallest upper bound of all seeds.  Per block of 32
    // groups, warp w visits the groups of bound rank w, w + 8, ... (increasing
    // bounds) and stops at the first whose bound exceeds its own fourth smallest
    // upper bound or the block-wide smallest one (s_T): neither is below the
    // final T, so every group left out has all its upper bounds above T.
    float u0 = finf, u1 = finf, u2 = finf, u3 = finf;
    for (int bi = 0; bi < n_blocks; ++bi) {
        const int blk = block_of(bi);
        const int grp = blk * 32 + lane;
        const bool valid = grp < n_groups;
        const float lbg = valid ? group_lower<D>(groups[grp], alo, ahi) : finf;
        const unsigned key = valid ? okey(lbg) : 0xffffffffu;
        int rank = 0;  // position of this lane's group in increasing bound order (ties by lane)
#pragma unroll 8
        for (int j = 0; j < 32; ++j) {
            const unsigned kj = __shfl_sync(0xffffffffu, key, j);
            rank += (kj < key || (kj == key && j < lane)) ? 1 : 0;
        }
        const int nvalid = __popc(__ballot_sync(0xffffffffu, valid));
        for (int r = wid; r < nvalid; r += W) {
            const int gl = __ffs(__ballot_sync(0xffffffffu, valid && rank == r)) - 1;
            const float bnd = __shfl_sync(0xffffffffu, lbg, gl);
            if (bnd > fminf(u3, okey_inv(*(volatile unsigned *)&s_T))) break;
            const int p = (blk * 32 + gl) * 32 + lane;
            const SeedRec32 q = p < n ? r32[p] : zrec;
            float lb, ub = finf;
            if (p < n) seed_bounds<D>(q, ch, cl, rlo, rhi, wrh, wrl, lb, ub);
            merge_smallest4(p < n ? okey(ub) : 0xffffffffu, u0, u1, u2, u3);
            if (lane == 0) atomicMin(&s_T, okey(u3));
        }
    }
    if (lane == 0) {
        s_u[wid][0] = u0;
        s_u[wid][1] = u1;
        s_u[wid][2] = u2;
        s_u[wid][3] = u3;
    }
    __syncthreads();
    float T;
    {  // the fourth smallest of the warps' four smallest (the same in every warp)
        unsigned k = okey((&s_u[0][0])[lane]);
        unsigned m = 0xffffffffu;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            m = __reduce_min_sync(0xffffffffu, k);
            const int l = __ffs(__ballot_sync(0xffffffffu, k == m)) - 1;
            if (lane == l) k = 0xffffffffu;
        }
        T = okey_inv(m);
    }
    // Pass 2: the candidates (lower bound <= T), the groups with a bound <= T
    // shared out by rank as above, each warp's list kept in shared memory; then
    // the lists are stored in warp order, and T_excl = the smallest bound of all
    // that is left out (skipped groups by their bound, seeds by theirs).
    float tex = finf;
    int cnt = 0;
    for (int bi = 0; bi < n_blocks; ++bi) {
        const int blk = block_of(bi);
        const int grp = blk * 32 + lane;
        const bool valid = grp < n_groups;
        const float lbg = valid ? group_lower<D>(groups[grp], alo, ahi) : finf;
        const bool in = valid && lbg <= T;
        tex = fminf(tex, (valid && !in) ? lbg : finf);
        const unsigned inm = __ballot_sync(0xffffffffu, in);
        const int rin = __popc(inm & ((1u << lane) - 1u));
        for (int r = wid; r < __popc(inm); r += W) {
            const int gl = __ffs(__ballot_sync(0xffffffffu, in && rin == r)) - 1;
            const int p = (blk * 32 + gl) * 32 + lane;
            const SeedRec32 q = p < n ? r32[p] : zrec;
            float lb = finf, ub = finf;
            if (p < n) seed_bounds<D>(q, ch, cl, rlo, rhi, wrh, wrl, lb, ub);
            const bool cand = p < n && lb <= T;
            const unsigned cm = __ballot_sync(0xffffffffu, cand);
            const int e = cnt + __popc(cm & ((1u << lane) - 1u));
            if (cand) {
                if (e < kSuperCap) {
                    s_pos[wid][e] = p;
                    s_lb[wid][e] = lb;
                } else {
                    tex = fminf(tex, lb);  // beyond the capacity: excluded
                }
            } else if (p < n) {
                tex = fminf(tex, lb);
            }
            cnt += __popc(cm);
        }
    }
    const int cnt_c = min(cnt, kSuperCap);
    tex = okey_inv(__reduce_min_sync(0xffffffffu, okey(tex)));
    if (lane == 0) {
        s_cnt[wid] = cnt_c;
        s_tex[wid] = tex;
    }
    __syncthreads();
    int off = 0;
    for (int w = 0; w < wid; ++w) off += s_cnt[w];
    float tex2 = finf;
    for (int e = lane; e < cnt_c; e += 32) {
        if (off + e < kSuperCap) s_list[off + e] = s_pos[wid][e];
        else tex2 = fminf(tex2, s_lb[wid][e]);  // beyond the capacity: excluded
    }
    tex2 = okey_inv(__reduce_min_sync(0xffffffffu, okey(tex2)));
    if (lane == 0) s_tex2[wid] = tex2;
    __syncthreads();
    if (threadIdx.x == 0) {
        int total = 0;
        float tx = finf;
        for (int w = 0; w < W; ++w) {
            total += s_cnt[w];
            tx = fminf(tx, fminf(s_tex[w], s_tex2[w]));
        }
        s_total = min(total, kSuperCap);
        s_texs = tx;
    }
    __syncthreads();
    // step 2: warp w takes tile c0 + (w & 1, (w >> 1) & 1, w >> 2) of the super-tile
    const int tc3[3] = {c0[0] + (wid & 1), c0[1] + ((wid >> 1) & 1), D == 3 ? c0[2] + (wid >> 2) : 0};
    if ((D == 2 && wid >= 4) || tc3[0] > c1[0] || tc3[1] > c1[1] || (D == 3 && tc3[2] > c1[2])) return;
    const int t = tc3[0] + sg.ntx * (tc3[1] + (D == 3 ? sg.nty * tc3[2] : 0));
    tile_list<D, KIND>(g, sg, t, tc3, r32, perm, axis_tab, s_list, s_total, s_texs, centre, meta, texcl, list, bops,
                       wrh, wrl);
}


// ---------------------------------------------------------------------------
// Main kernel
// ---------------------------------------------------------------------------
struct TcArgs {
    GridDev g;
    int n, ntx, nty, tlo, ntiles, n_chunks;
    const SeedRec32 *recs;   // scan order
    const SeedRec32 *recs_nat;  // natural order (the FP32 resolution of undecided pixels)
    const int32_t *perm;     // scan position -> seed index (null: identity)
    const float *centre;     // [ntiles][6]
    int pruned;              // per-tile candidate lists (else all seeds)
    const int *start;        // dense form: Morton start chunk per tile
    const int4 *meta;        // per tile: first pixel per axis, candidate count (pruned form)
    const float *texcl;      // pruned form: bound of the excluded seeds per tile
    const int *list;         // pruned form: [ntiles][kListCap] seed indices
    const uint8_t *bops;     // pruned form: [ntiles][kMaxSteps] stored seed operands
    float err_unit, R_tile;
    unsigned long long *gmom;
    uint32_t *flags;
    int32_t *flag_gi;
    int32_t *labels;
    // recording pass (REC) only, per pixel: gap0 = a certified lower bound of every
    // other seed's cost minus the label's (0: none); rec = {gl, gu, g3, b}: the
    // runner-up seed b (-1: none), certified bounds gl <= C_b - C_a <= gu and
    // g3 <= C_k - C_a for every other seed k (all 0: none)
    float *gap0;
    float4 *rec;
    DevScalars *sc;
    unsigned long long *pairs_scored;
    int wide;  // some axis has more than 4096 pixels: 64-bit moment sums across the warp
    const int *skip;  // incremental pass: nothing to do when *skip (a re-decision)
    unsigned *hist;   // REC: recorded pixels by the float exponent of their g3 margin
};

template <int D, int KIND, bool REC>
__global__ void __launch_bounds__(kThreads, 1) assign_tc_kernel(const __grid_constant__ TcArgs a) {
    using G = TcGeom<D>;
    using Fm = TcFmt<KIND>;
    constexpr int F = G::F;
    constexpr int KM = moment_width(D);
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    TcShared<D, KIND> &sm = *reinterpret_cast<TcShared<D, KIND> *>(tc_smem_raw);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const GridDev &g = a.g;
    if (a.skip && *(volatile const int *)a.skip) return;  // the whole block, before any setup
    __shared__ unsigned s_hist[REC ? kIncBins : 1];
    if constexpr (REC)
        for (int i = tid; i < kIncBins; i += blockDim.x) s_hist[i] = 0u;
    const bool pruned = a.pruned != 0;
    const int my_tiles = (int)blockIdx.x < a.ntiles ? (a.ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    auto tile_of = [&](int i) { return (int)blockIdx.x + i * (int)gridDim.x; };
    auto nsteps = [&](int t) { return pruned ? max(1, (a.meta[t].w + kN - 1) / kN) : a.n_chunks; };

    // epilogue threads: M tile and row (tensor-memory lane) of their pixel
    const int mt = warp >> 2;
    const int row = ((warp & 3) << 5) + lane;
    const int lt = mt * kM + row;
    const int lk[3] = {lt % G::TX, (lt / G::TX) % G::TY, lt / (G::TX * G::TY)};
    const int tdim[3] = {G::TX, G::TY, G::TZ};

    if (warp < kEpiWarps) {
        // A operand: the split pixel features of row `row` of M tile `mt` (the same for every tile)
        float yp[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int d = 0; d < D; ++d) yp[d] = ((float)(lk[d] - tdim[d] / 2) + 0.5f) * g.h32[d];
        float f[F];
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
        float rowv[kK];
        split_row<F, KIND, false>(f, rowv);
#pragma unroll
        for (int c = 0; c < kK / Fm::EPR; ++c)
            put_row<KIND>(sm.A[mt] + tc::core_offset(row, c * Fm::EPR, Fm::EB, Fm::LBO, Fm::SBO),
                          rowv + c * Fm::EPR);
    }
    if (warp == 0) {
        tc::tmem_alloc(&sm.tslot, kCols);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int i = 0; i < kStages; ++i) {
            mbar_init(&sm.bar_bfull[i], pruned ? 1 : kXfWarps);  // bulk copy (pruned) or the transform warps
            mbar_init(&sm.bar_acc[i], 1);
            mbar_init(&sm.bar_aempty[i], kEpiWarps);
        }
        sm.abort = 0;
        fence_mbar_init();
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = sm.tslot;

    // bounded wait that gives up at once after any timeout of the CTA
    auto wait = [&](uint64_t *bar, uint32_t parity) {
        if (*(volatile int *)&sm.abort) return false;
        if (mbar_wait_bounded(bar, parity, &a.sc->status)) return true;
        *(volatile int *)&sm.abort = 1;
        return false;
    };
    auto chunk_id = [&](int start, int k) {  // dense form: zig-zag from the tile's chunk
        const int off = (k & 1) ? ((k + 1) >> 1) : -(k >> 1);
        int c = start + off;
        if (c >= a.n_chunks) c -= a.n_chunks;
        if (c < 0) c += a.n_chunks;
        return c;
    };

    if (warp == kProdWarp) {
        // ---------------- MMA issue ----------------
        if (lane == 0) {
            const uint32_t idesc = tc::instr_desc(KIND, kM, kN);
            int q = 0;
            bool ok = true;
            // pruned form: a second cursor issues the bulk copy of step tq's operand
            // into B[tq % 4] up to kAhead steps before its MMAs
            int tq = 0, ti = 0, tk = 0, tns = my_tiles > 0 ? nsteps(tile_of(0)) : 0;
            auto issue_copy = [&]() {
                const int s = tq & (kStages - 1);
                // the MMAs of step tq - 4 (the last readers of B[s]) are complete
                if (tq >= kStages && !wait(&sm.bar_acc[s], (uint32_t)(((tq >> 2) - 1) & 1))) return false;
                mbar_expect_tx(&sm.bar_bfull[s], (uint32_t)Fm::B_BYTES);
                bulk_g2s(sm.B[s], a.bops + ((size_t)tile_of(ti) * kMaxSteps + tk) * Fm::B_BYTES, (uint32_t)Fm::B_BYTES,
                         &sm.bar_bfull[s]);
                ++tq;
                if (++tk == tns) {
                    tk = 0;
                    if (++ti < my_tiles) tns = nsteps(tile_of(ti));
                }
                return true;
            };
            for (int i = 0; i < my_tiles && ok; ++i) {
                const int ns = nsteps(tile_of(i));
                for (int k = 0; k < ns && ok; ++k, ++q) {
                    const int s = q & (kStages - 1);
                    if (pruned) {
                        while (ok && ti < my_tiles && tq <= q + kAhead) ok = issue_copy();
                        if (!ok) break;
                    }
                    if (!wait(&sm.bar_bfull[s], (uint32_t)((q >> 2) & 1))) { ok = false; break; }
                    if (q >= kStages && !wait(&sm.bar_aempty[s], (uint32_t)(((q >> 2) - 1) & 1))) { ok = false; break; }
                    tc::fence_after_sync();
                    const uint32_t b0 = (uint32_t)__cvta_generic_to_shared(sm.B[s]);
#pragma unroll
                    for (int m = 0; m < kMT; ++m) {
                        const uint32_t a0 = (uint32_t)__cvta_generic_to_shared(sm.A[m]);
                        const uint32_t d = taddr + (uint32_t)(s * kMT * kN + m * kN);
#pragma unroll
                        for (int st = 0; st < Fm::STEPS; ++st) {
                            const uint32_t off = (uint32_t)st * (uint32_t)(Fm::KSTEP / Fm::EPR) * Fm::LBO;
                            const uint64_t ad = tc::smem_desc(a0 + off, Fm::LBO, Fm::SBO);
                            const uint64_t bd = tc::smem_desc(b0 + off, Fm::LBO, Fm::SBO);
                            if (KIND == tc::KIND_TF32)
                                tc::mma_tf32(d, ad, bd, idesc, st > 0 ? 1u : 0u);
                            else
                                tc::mma_bf16(d, ad, bd, idesc, st > 0 ? 1u : 0u);
                        }
                    }
                    tc::mma_commit(&sm.bar_acc[s]);
                }
            }
            // no MMA may still run when the tensor memory is released, and no copy may
            // still land in shared memory when the CTA exits: wait for both
            if (q > 0) {
                const int s = (q - 1) & (kStages - 1);
                mbar_wait_bounded(&sm.bar_acc[s], (uint32_t)(((q - 1) >> 2) & 1), &a.sc->status);
            }
            for (int r = q; r < tq; ++r)
                mbar_wait_bounded(&sm.bar_bfull[r & (kStages - 1)], (uint32_t)((r >> 2) & 1), &a.sc->status);
        }
    } else if (warp >= kXfWarp0) {
        // ---------------- dense form: seed operands (two threads per seed, each half of K) ----------------
        const int tt = tid - kXfWarp0 * 32;
        const int sl = tt >> 1, half = tt & 1;
        const double wref = dkey_inv(a.sc->wref_key);
        float wrh, wrl;
        split2(wref, wrh, wrl);
        int q = 0;
        bool ok = !pruned;
        for (int i = 0; i < my_tiles && ok; ++i) {
            const int t = tile_of(i);
            const int ns = nsteps(t);
            float ch[3] = {0.f, 0.f, 0.f}, cl[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int d = 0; d < D; ++d) {
                ch[d] = a.centre[(size_t)t * 6 + d];
                cl[d] = a.centre[(size_t)t * 6 + 3 + d];
            }
            const int st0 = a.start[t];
            for (int k = 0; k < ns; ++k, ++q) {
                const int s = q & (kStages - 1);
                // the MMAs of step q - 4 have read B[s]
                if (q >= kStages && !wait(&sm.bar_acc[s], (uint32_t)(((q >> 2) - 1) & 1))) { ok = false; break; }
                const int p = chunk_id(st0, k) * kN + sl;
                float rowv[kK];
                seed_row<D, KIND>(a.recs, p < a.n ? p : -1, ch, cl, wrh, wrl, rowv);
                uint8_t *B = sm.B[s];
                if (half == 0) {
#pragma unroll
                    for (int c = 0; c < kK / 2 / Fm::EPR; ++c)
                        put_row<KIND>(B + tc::core_offset(sl, c * Fm::EPR, Fm::EB, Fm::LBO, Fm::SBO), rowv + c * Fm::EPR);
                } else {
#pragma unroll
                    for (int c = 0; c < kK / 2 / Fm::EPR; ++c) {
                        constexpr int H = kK / 2;
                        put_row<KIND>(B + tc::core_offset(sl, H + c * Fm::EPR, Fm::EB, Fm::LBO, Fm::SBO),
                                      rowv + H + c * Fm::EPR);
                    }
                }
                tc::fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm.bar_bfull[s]);
            }
        }
    } else {
        // ---------------- epilogue: one pixel per thread ----------------
        const uint32_t lane_base = ((uint32_t)((warp & 3) * 32)) << 16;
        const float lam_abs = (float)__longlong_as_double((long long)a.sc->lam_abs_bits);
        const float inv_lam = 1.f / fmaxf((float)__longlong_as_double((long long)a.sc->lam_min_bits), 1e-30f);
        // Bound of |score - cost| for a seed scoring s, linear in |s|: the term sum
        // Lambda (2R + sqrt(C / lambda))^2 + C is at most 8 Lambda R^2 + (2 Lambda /
        // lambda + 1) C (from (a + b)^2 <= 2 a^2 + 2 b^2), evaluated at an upper bound
        // of the exact cost C <= |s| + err_unit (that sum at |s|).
        const float ps0 = 8.f * lam_abs * a.R_tile * a.R_tile;
        const float ps1 = 2.f * lam_abs * inv_lam + 1.f;
        auto psi = [&](float s) {
            const float c = fabsf(s) + a.err_unit * fmaf(ps1, fabsf(s), ps0);
            return 1.1f * a.err_unit * fmaf(ps1, c, ps0);
        };
        int q = 0;
        float wrh = 0.f, wrl = 0.f;
        split2(dkey_inv(a.sc->wref_key), wrh, wrl);
        float ypx[3] = {0.f, 0.f, 0.f};  // this thread's pixel relative to the tile centre
#pragma unroll
        for (int d = 0; d < D; ++d) ypx[d] = ((float)(lk[d] - tdim[d] / 2) + 0.5f) * g.h32[d];
        // per-tile values, loaded one tile ahead
        const float finf = __int_as_float(0x7f800000);
        int4 nx_meta = my_tiles > 0 ? a.meta[tile_of(0)] : make_int4(0, 0, 0, 0);
        float nx_tex = pruned && my_tiles > 0 ? a.texcl[tile_of(0)] : finf;
        int nx_st0 = !pruned && my_tiles > 0 ? a.start[tile_of(0)] : 0;
        for (int i = 0; i < my_tiles; ++i) {
            const int t = tile_of(i);
            const int4 mt4 = nx_meta;
            const int cnt = mt4.w;
            const float tex = nx_tex;
            const int st0 = nx_st0;
            const int ns = pruned ? max(1, (cnt + kN - 1) / kN) : a.n_chunks;
            if (i + 1 < my_tiles) {
                const int tn = tile_of(i + 1);
                nx_meta = a.meta[tn];
                if (pruned) nx_tex = a.texcl[tn];
                else nx_st0 = a.start[tn];
            }
            int lv[kMaxSteps];  // pruned form: the seed of list slot k * 32 + lane
#pragma unroll
            for (int k = 0; k < kMaxSteps; ++k)
                lv[k] = (pruned && k * kN + lane < cnt) ? a.list[(size_t)t * kListCap + k * kN + lane] : -1;
            float k1 = FLT_MAX, k2 = FLT_MAX;  // two smallest packed scores
            float k3 = FLT_MAX;                // REC: the third smallest
            int bstep = 0, bstep2 = 0;         // steps of k1 and (REC) k2
            bool ok = true;
            for (int k = 0; k < ns; ++k, ++q) {
                const int s = q & (kStages - 1);
                // warp-uniform: the tensor-memory load below is a whole-warp instruction
                const bool got = __all_sync(0xffffffffu, wait(&sm.bar_acc[s], (uint32_t)((q >> 2) & 1)));
                ok = ok && got;
                tc::fence_after_sync();
                float v[32], mn = FLT_MAX;
                if (got) {
                    tc::tmem_ld32_min(taddr + lane_base + (uint32_t)(s * kMT * kN + mt * kN), v, mn);
                    tc::tmem_wait_ld();
                }
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm.bar_aempty[s]);
                // a slice whose smallest score lies above the second-best (REC: third)
                // by more than the packing (< 32 ulp) cannot change the kept keys
                const float kq = REC ? k3 : k2;
                if (got && !(mn > fmaf(fabsf(kq), 0x1p-16f, kq))) {
#pragma unroll
                    for (int e = 0; e < 32; ++e) v[e] = __uint_as_float((__float_as_uint(v[e]) & ~31u) | (unsigned)e);
                  if constexpr (REC) {
                    // the three smallest: sorted pairs, then sorted triples merged (the
                    // m-th smallest of two sorted lists A, B is min over i + j = m of
                    // max(A_i, B_j), A_0 = B_0 = -inf)
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const float lo = fminf(v[2 * e], v[2 * e + 1]), hi = fmaxf(v[2 * e], v[2 * e + 1]);
                        v[2 * e] = lo;
                        v[2 * e + 1] = hi;
                    }
#pragma unroll
                    for (int e = 0; e < 32; e += 4) {
                        const float a1 = v[e], a2 = v[e + 1], b1 = v[e + 2], b2 = v[e + 3];
                        v[e] = fminf(a1, b1);
                        v[e + 1] = fminf(fmaxf(a1, b1), fminf(a2, b2));
                        v[e + 2] = fminf(fmaxf(a1, b2), fmaxf(a2, b1));
                    }
#pragma unroll
                    for (int w = 8; w <= 32; w <<= 1) {
#pragma unroll
                        for (int e = 0; e < 32; e += w) {
                            const float a1 = v[e], a2 = v[e + 1], a3 = v[e + 2];
                            const float b1 = v[e + w / 2], b2 = v[e + w / 2 + 1], b3 = v[e + w / 2 + 2];
                            v[e] = fminf(a1, b1);
                            v[e + 1] = fmin3_f(a2, b2, fmaxf(a1, b1));
                            v[e + 2] = fminf(fmin3_f(a3, b3, fmaxf(a2, b1)), fmaxf(a1, b2));
                        }
                    }
                    const float o1 = k1, o2 = k2;
                    const bool better = v[0] < o1;
                    k1 = fminf(o1, v[0]);
                    k2 = fmin3_f(o2, v[1], fmaxf(o1, v[0]));
                    k3 = fminf(fmin3_f(k3, v[2], fmaxf(o2, v[0])), fmaxf(o1, v[1]));
                    // k2 is the old best, the old second or one of this step's scores
                    bstep2 = k2 == o1 ? bstep : (k2 == o2 ? bstep2 : k);
                    bstep = better ? k : bstep;
                  } else {
                    // tournament: pairs (lo, hi), then merge pairs of pairs
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const float lo = fminf(v[2 * e], v[2 * e + 1]), hi = fmaxf(v[2 * e], v[2 * e + 1]);
                        v[2 * e] = lo;
                        v[2 * e + 1] = hi;
                    }
#pragma unroll
                    for (int w = 4; w <= 32; w <<= 1) {
#pragma unroll
                        for (int e = 0; e < 32; e += w) {
                            const float a1 = v[e], a2 = v[e + 1], b1 = v[e + w / 2], b2 = v[e + w / 2 + 1];
                            v[e] = fminf(a1, b1);
                            v[e + 1] = fmin3_f(fmaxf(a1, b1), a2, b2);
                        }
                    }
                    const bool better = v[0] < k1;
                    k2 = fmin3_f(fmaxf(k1, v[0]), k2, v[1]);
                    k1 = fminf(k1, v[0]);
                    bstep = better ? k : bstep;
                  }
                }
            }
            // ---- end of tile: certificate, label, FP64 queue, moments ----
            const int kk[3] = {mt4.x + lk[0], mt4.y + lk[1], mt4.z + lk[2]};
            const int klast = D == 3 ? kk[2] : kk[1];
            const bool valid = ok && kk[0] < g.res[0] && kk[1] < g.res[1] && (D == 2 || kk[2] < g.res[2]) &&
                               klast >= win_lo(g) && klast < win_hi(g);
            int label = -1;
            bool queue = false;
            int hint = -1;
            long long j = 0;
            // the best seed: list slot bstep * 32 + idx (pruned) or scan position (dense)
            const int idx = (int)(__float_as_uint(k1) & 31u);
            int seed = -1;
            int seed_b = -1;  // REC: the seed of k2
            if (pruned) {
                const int idx2 = (int)(__float_as_uint(k2) & 31u);
#pragma unroll
                for (int kk = 0; kk < kMaxSteps; ++kk) {
                    const int v = __shfl_sync(0xffffffffu, lv[kk], idx);
                    if (kk == bstep) seed = v;
                    if constexpr (REC) {
                        const int v2 = __shfl_sync(0xffffffffu, lv[kk], idx2);
                        if (kk == bstep2) seed_b = v2;
                    }
                }
            }
            // REC: this pixel's record (all 0: re-decided in full by a later pass)
            float r_gl = 0.f, r_gu = 0.f, r_g3 = 0.f;
            int r_b = -1;
            if (valid) {
                j = (long long)kk[0] + (long long)g.res[0] * ((long long)kk[1] + (long long)g.res[1] * (long long)kk[2]);
                if (!pruned) {
                    const int p = chunk_id(st0, bstep) * kN + idx;
                    seed = p < a.n ? (a.perm ? a.perm[p] : p) : -1;
                }
                hint = seed;
                const float U = k1 + psi(k1);
                const bool cert = seed >= 0 && k1 < 1e29f && U < k2 - psi(k2) && U < tex;
                if (cert) label = seed;
                else queue = true;
                if constexpr (REC) {
                    // margins of the certificate: C_b - C_a lies within [s2 - psi(s2) - U,
                    // s2 + psi(s2) - (s1 - psi(s1))]; every seed but a and b costs at least
                    // min(s3 - psi(s3), T_excl) (s - psi(s) grows with s), every listed
                    // seed at least its score less psi
                    if (cert) {
                        const float Uu = __fadd_ru(k1, psi(k1)), Ld = __fsub_rd(k1, psi(k1));
                        const float l2 = k2 < 1e29f ? __fsub_rd(k2, psi(k2)) : finf;
                        const float l3 = k3 < 1e29f ? __fsub_rd(k3, psi(k3)) : finf;
                        if (k2 < 1e29f && seed_b >= 0 && seed_b != seed) {
                            r_b = seed_b;
                            r_gl = __fsub_rd(l2, Uu);
                            r_gu = __fsub_ru(__fadd_ru(k2, psi(k2)), Ld);
                            r_g3 = __fsub_rd(fminf(l3, tex), Uu);
                        } else {  // no runner-up identified: one bound for every other seed
                            r_gl = r_gu = finf;
                            r_g3 = __fsub_rd(fminf(l2, tex), Uu);
                        }
                    }
                }
            }
            // Pruned form: the pixels the scores leave undecided are settled in FP32
            // direct form by the warp (lane l takes list slots l, l + 32, ..): the label
            // is certified when the best upper bound c + E lies below every other
            // candidate's lower bound c - E and below the excluded seeds' bound.
            if (pruned) {
                unsigned unc = __ballot_sync(0xffffffffu, queue);
                if (unc) {
                    float ch[3] = {0.f, 0.f, 0.f}, cl[3] = {0.f, 0.f, 0.f};
#pragma unroll
                    for (int d = 0; d < D; ++d) {
                        ch[d] = a.centre[(size_t)t * 6 + d];
                        cl[d] = a.centre[(size_t)t * 6 + 3 + d];
                    }
                    while (unc) {
                        const int p = __ffs(unc) - 1;
                        unc &= unc - 1u;
                        float yp[3] = {0.f, 0.f, 0.f};
#pragma unroll
                        for (int d = 0; d < D; ++d) yp[d] = __shfl_sync(0xffffffffu, ypx[d], p);
                        float cv[kMaxSteps], ev[kMaxSteps];
                        float ub = finf;
                        int us = 0x7fffffff;
#pragma unroll
                        for (int kk2 = 0; kk2 < kMaxSteps; ++kk2) {
                            cv[kk2] = finf;
                            ev[kk2] = 0.f;
                            if (kk2 < ns && lv[kk2] >= 0) {
                                cost32_bound_rel<D>(a.recs_nat[lv[kk2]], ch, cl, yp, wrh, wrl, cv[kk2], ev[kk2]);
                                const float u1 = cv[kk2] + ev[kk2];
                                if (u1 < ub || (u1 == ub && lv[kk2] < us)) {
                                    ub = u1;
                                    us = lv[kk2];
                                }
                            }
                        }
                        // the smallest upper bound of the warp and its seed
                        const unsigned kub = okey(ub);
                        const unsigned kmin = __reduce_min_sync(0xffffffffu, kub);
                        const int smin = __reduce_min_sync(0xffffffffu, kub == kmin ? (unsigned)us : 0x7fffffffu);
                        const float Ub = okey_inv(kmin);
                        bool other = false;  // another candidate may cost as little
#pragma unroll
                        for (int kk2 = 0; kk2 < kMaxSteps; ++kk2)
                            if (kk2 < ns && lv[kk2] >= 0 && lv[kk2] != smin && !(cv[kk2] - ev[kk2] > Ub)) other = true;
                        const bool ok2 = !__any_sync(0xffffffffu, other) && Ub < tex && smin < a.n;
                        if constexpr (REC) {
                            if (ok2) {
                                // the runner-up: smallest lower bound among the other candidates;
                                // then its upper bound, the label's lower bound and the rest's
                                float lb2 = finf;
                                int sb2 = 0x7fffffff;
#pragma unroll
                                for (int kk2 = 0; kk2 < kMaxSteps; ++kk2)
                                    if (kk2 < ns && lv[kk2] >= 0 && lv[kk2] != smin) {
                                        const float l = __fsub_rd(cv[kk2], ev[kk2]);
                                        if (l < lb2 || (l == lb2 && lv[kk2] < sb2)) {
                                            lb2 = l;
                                            sb2 = lv[kk2];
                                        }
                                    }
                                const unsigned kl2 = __reduce_min_sync(0xffffffffu, okey(lb2));
                                const int sb = (int)__reduce_min_sync(0xffffffffu, okey(lb2) == kl2 ? (unsigned)sb2 : 0x7fffffffu);
                                float hb = finf, la = finf, l3 = finf;
#pragma unroll
                                for (int kk2 = 0; kk2 < kMaxSteps; ++kk2)
                                    if (kk2 < ns && lv[kk2] >= 0) {
                                        if (lv[kk2] == sb) hb = __fadd_ru(cv[kk2], ev[kk2]);
                                        else if (lv[kk2] == smin) la = __fsub_rd(cv[kk2], ev[kk2]);
                                        else l3 = fminf(l3, __fsub_rd(cv[kk2], ev[kk2]));
                                    }
                                const float HB = okey_inv(__reduce_min_sync(0xffffffffu, okey(hb)));
                                const float LA = okey_inv(__reduce_min_sync(0xffffffffu, okey(la)));
                                const float L3 = okey_inv(__reduce_min_sync(0xffffffffu, okey(l3)));
                                const float LB2 = okey_inv(kl2);
                                if (lane == p) {
                                    if (sb < a.n && LB2 < finf) {
                                        r_b = sb;
                                        r_gl = __fsub_rd(LB2, Ub);
                                        r_gu = __fsub_ru(HB, LA);
                                        r_g3 = __fsub_rd(fminf(L3, tex), Ub);
                                    } else {
                                        r_b = -1;
                                        r_gl = r_gu = finf;
                                        r_g3 = __fsub_rd(fminf(LB2, tex), Ub);
                                    }
                                }
                            }
                        }
                        if (lane == p) {
                            if (ok2) {
                                label = smin;
                                queue = false;
                            } else if (smin < a.n) {
                                hint = smin;
                            }
                        }
                    }
                }
            }
            // queued pixels: one atomic per warp
            const unsigned qm = __ballot_sync(0xffffffffu, queue);
            if (qm) {
                unsigned base = 0u;
                if (lane == __ffs(qm) - 1) base = atomicAdd(&a.sc->flag_count, (unsigned)__popc(qm));
                base = __shfl_sync(0xffffffffu, base, __ffs(qm) - 1);
                if (queue) {
                    const unsigned slot = base + (unsigned)__popc(qm & ((1u << lane) - 1u));
                    a.flags[slot] = (uint32_t)j;
                    if (a.flag_gi) a.flag_gi[slot] = hint;
                }
            }
            if (label >= 0 && a.labels) a.labels[j] = label;
            if constexpr (REC) {
                if (valid) {
                    a.rec[j] = make_float4(r_gl, r_gu, r_g3, __int_as_float(r_b));
                    a.gap0[j] = label >= 0 ? fmaxf(fminf(r_gl, r_g3), 0.f) : 0.f;
                    atomicAdd(&s_hist[r_g3 > 0.f ? min(__float_as_uint(r_g3) >> 21, (unsigned)kIncBins - 1u) : 0u], 1u);
                }
            }
            // Moments of the certified pixels.  The lanes holding the same label sum
            // their words across the warp; the last axis's coordinate is the same for
            // the whole warp (3D: one z of an 8 x 4 block, 2D: one row), so the words
            // with it follow from the count and the other sums.  Lanes 0 .. K-1 then
            // add one word each to the global int64 moments.
            unsigned todo = __ballot_sync(0xffffffffu, label >= 0);
            const unsigned long long uz = 2ull * (unsigned long long)(D == 3 ? kk[2] : kk[1]) + 1ull;
            while (todo) {
                const int leader = __ffs(todo) - 1;
                const int L0 = __shfl_sync(0xffffffffu, label, leader);
                const bool mine = label == L0;
                const unsigned grp = __ballot_sync(0xffffffffu, mine);
                const unsigned long long m = (unsigned long long)__popc(grp);
                unsigned long long sum[KM];
                if (!a.wide) {
                    // u < 2^13: every product is below 2^26 and 32 of them below 2^31
                    const unsigned u0 = mine ? 2u * (unsigned)kk[0] + 1u : 0u;
                    const unsigned u1 = (mine && D == 3) ? 2u * (unsigned)kk[1] + 1u : 0u;
                    const unsigned long long s0 = __reduce_add_sync(0xffffffffu, u0);
                    const unsigned long long s00 = __reduce_add_sync(0xffffffffu, u0 * u0);
                    if (D == 3) {
                        const unsigned long long s1 = __reduce_add_sync(0xffffffffu, u1);
                        const unsigned long long s01 = __reduce_add_sync(0xffffffffu, u0 * u1);
                        const unsigned long long s11 = __reduce_add_sync(0xffffffffu, u1 * u1);
                        sum[0] = m; sum[1] = s0; sum[2] = s1; sum[3] = m * uz;
                        sum[4] = s00; sum[5] = s01; sum[6] = s0 * uz; sum[7] = s11; sum[8] = s1 * uz;
                        sum[9] = m * uz * uz;
                    } else {
                        sum[0] = m; sum[1] = s0; sum[2] = m * uz; sum[3] = s00; sum[4] = s0 * uz;
                        sum[5] = m * uz * uz;
                    }
                } else {
                    unsigned long long u[3] = {0ull, 0ull, 0ull};
#pragma unroll
                    for (int d = 0; d < D; ++d) u[d] = mine ? 2ull * (unsigned long long)kk[d] + 1ull : 0ull;
                    unsigned long long own[KM];
                    own[0] = mine ? 1ull : 0ull;
#pragma unroll
                    for (int d = 0; d < D; ++d) own[1 + d] = u[d];
                    int e = 1 + D;
#pragma unroll
                    for (int d = 0; d < D; ++d)
#pragma unroll
                        for (int d2 = d; d2 < D; ++d2) own[e++] = u[d] * u[d2];
#pragma unroll
                    for (int v = 0; v < KM; ++v) {
                        unsigned long long x = own[v];
#pragma unroll
                        for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
                        sum[v] = x;
                    }
                }
                unsigned long long word = 0ull;
#pragma unroll
                for (int v = 0; v < KM; ++v)
                    if (lane == v) word = sum[v];
                if (lane < KM && word) atomicAdd(&a.gmom[(size_t)L0 * KM + lane], word);
                todo &= ~grp;
            }
            if (warp == 0 && lane == 0 && a.pairs_scored)
                atomicAdd(a.pairs_scored, (unsigned long long)ns * kN * kPix);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(taddr, kCols);
    if constexpr (REC)
        for (int i = tid; i < kIncBins; i += blockDim.x)
            if (s_hist[i]) atomicAdd(&a.hist[i], s_hist[i]);
}

template <int D>
void tile_grid(const GridDev &g, int &ntx, int &nty, int &tlo, long long &ntiles) {
    using G = TcGeom<D>;
    ntx = (g.res[0] + G::TX - 1) / G::TX;
    if (D == 3) {
        nty = (g.res[1] + G::TY - 1) / G::TY;
        tlo = win_lo(g) / G::TZ;
        const int thi = (win_hi(g) - 1) / G::TZ;
        ntiles = (long long)ntx * nty * (thi - tlo + 1);
    } else {
        tlo = win_lo(g) / G::TY;
        const int thi = (win_hi(g) - 1) / G::TY;
        nty = thi - tlo + 1;
        ntiles = (long long)ntx * nty;
    }
}

template <int D>
cudaError_t ensure_axis(const GridDev &g, int ntx, int nty, int ntz, int tlo, Workspace &ws, cudaStream_t st) {
    const double key[12] = {(double)D,          (double)g.res[0], (double)g.res[1], (double)g.res[2],
                            g.lo[0],            g.lo[1],          g.lo[2],          g.h[0],
                            g.h[1],             g.h[2],           (double)tlo,      (double)win_hi(g)};
    if (std::memcmp(key, ws.tc_axis_key, sizeof key) == 0) return cudaSuccess;
    const int naxis = ntx + nty + ntz;
    tc_axis_kernel<D><<<(naxis + 255) / 256, 256, 0, st>>>(g, ntx, nty, ntz, tlo, ws.tc_axis);
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        std::memcpy(ws.tc_axis_key, key, sizeof key);
        ++ws.kernel_launches;
    }
    return e;
}

template <int D, int KIND>
cudaError_t launch_tc_t(const GridDev &g, int n, Workspace &ws, int32_t *labels, unsigned long long *gmom,
                        cudaStream_t st) {
    using G = TcGeom<D>;
    int ntx = 0, nty = 0, tlo = 0;
    long long ntl = 0;
    tile_grid<D>(g, ntx, nty, tlo, ntl);
    if (ntl > ws.tc_tile_cap) return cudaErrorInvalidValue;  // the caller checks tc_tile_count first
    const int ntiles = (int)ntl;
    const int n_chunks = (n + kN - 1) / kN;
    const bool pruned = ws.prune;
    const SeedRec32 *rs = ws.sorted ? ws.recs32s : ws.recs32;
    const int ntz = D == 3 ? (int)(ntl / ((long long)ntx * nty)) : 0;
    // the per-axis table depends on the grid and the tiling only: recomputed when
    // they change (a graph capture leaves it to the caller, before every replay)
    if (!ws.capturing) {
        const cudaError_t e = ensure_axis<D>(g, ntx, nty, ntz, tlo, ws, st);
        if (e != cudaSuccess) return e;
    }
    if (pruned) {
        const SuperGeom sg{ntx, nty, ntz, tlo};
        const int nsup = ((ntx + 1) / 2) * ((nty + 1) / 2) * (D == 3 ? (ntz + 1) / 2 : 1);
        ws.kernel_launches += 1;
        tc_lists_kernel<D, KIND><<<nsup, kSupWarps * 32, 0, st>>>(
            g, sg, nsup, n, rs, ws.sorted ? ws.perm : nullptr, ws.groups, ws.sorted ? ws.scodes : nullptr, ws.tc_axis,
            ws.tc_centre, ws.tc_meta, ws.tc_texcl, ws.tc_list, ws.tc_bops, ws.sc,
            ws.inc_auto ? &ws.sc->inc_go : nullptr);
    } else {
        const int pblocks = (int)((ntl * 32 + 255) / 256);
        ws.kernel_launches += 1;
        tc_tile_kernel<D, KIND><<<pblocks, 256, 0, st>>>(
            g, ntx, nty, tlo, ntiles, n, rs, ws.groups, ws.sorted ? ws.scodes : nullptr,
            ws.sorted ? ws.perm : nullptr, n_chunks, ws.tc_centre, ws.tc_start, ws.tc_meta, ws.tc_texcl, nullptr,
            ws.tc_bops, ws.tc_axis, ws.sc);
    }
    // more than 114 KB of shared memory keeps one CTA (512 tensor-memory columns) per SM
    const size_t smem = std::max<size_t>(sizeof(TcShared<D, KIND>), 120 * 1024);
    // the recording variant (incremental passes) also keeps each pixel's runner-up and margins
    const bool rec = ws.rec_gap != nullptr;
    if (rec && (!pruned || !ws.inc_rec || !ws.inc_hist)) return cudaErrorInvalidValue;
    const unsigned bit = (rec ? kAttrTcScoreRec : kAttrTcScore) << ((D == 3 ? 2 : 0) + (KIND == tc::KIND_BF16 ? 1 : 0));
    if (!(ws.attr_done & bit)) {
        const cudaError_t e = cudaFuncSetAttribute(rec ? assign_tc_kernel<D, KIND, true> : assign_tc_kernel<D, KIND, false>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        ws.attr_done |= bit;
    }
    const int sms = ws.sms;
    const double hx = 0.5 * G::TX * g.h[0], hy = 0.5 * G::TY * g.h[1], hz = D == 3 ? 0.5 * G::TZ * g.h[2] : 0.0;
    TcArgs args;
    args.g = g;
    args.n = n;
    args.ntx = ntx;
    args.nty = nty;
    args.tlo = tlo;
    args.ntiles = ntiles;
    args.n_chunks = n_chunks;
    args.recs = rs;
    args.recs_nat = ws.recs32;
    args.perm = ws.sorted ? ws.perm : nullptr;
    args.centre = ws.tc_centre;
    args.pruned = pruned ? 1 : 0;
    args.start = ws.tc_start;
    args.meta = ws.tc_meta;
    args.texcl = ws.tc_texcl;
    args.list = ws.tc_list;
    args.bops = ws.tc_bops;
    // per score: the split operands' 3 e^2 (e = 2^-11 TF32, 2^-8 BF16), 32 accumulations at
    // 2^-22, ~100 FP32 roundings of the features and the packed index (2^-18), with a 1.5x margin
    const double e_op = KIND == tc::KIND_TF32 ? std::ldexp(1.0, -11) : std::ldexp(1.0, -8);
    args.err_unit = (float)(1.5 * (3.1 * e_op * e_op + 32.0 * std::ldexp(1.0, -22) + 100.0 * std::ldexp(1.0, -24) +
                                   std::ldexp(1.0, -18)));
    args.R_tile = (float)(std::sqrt(hx * hx + hy * hy + hz * hz) * (1.0 + 1e-6));
    args.gmom = gmom;
    args.flags = ws.flags;
    args.flag_gi = ws.flag_gi;
    args.labels = labels;
    args.gap0 = ws.rec_gap;
    args.rec = rec ? ws.inc_rec : nullptr;
    args.hist = rec ? ws.inc_hist : nullptr;
    args.skip = ws.inc_auto ? &ws.sc->inc_go : nullptr;
    args.sc = ws.sc;
    args.pairs_scored = ws.pairs_scored;
    args.wide = (g.res[0] > 4096 || g.res[1] > 4096 || (D == 3 && g.res[2] > 4096)) ? 1 : 0;
    const int grid = (int)std::min<long long>(ntl, sms);
    const cudaError_t ep = record_scoring_start(ws, st);
    if (ep != cudaSuccess) return ep;
    if (rec) assign_tc_kernel<D, KIND, true><<<grid, kThreads, smem, st>>>(args);
    else assign_tc_kernel<D, KIND, false><<<grid, kThreads, smem, st>>>(args);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Incremental pass.  The weights enter every cost linearly: at weights w the
// cost of seed k differs from the recorded pass's (weights w0) by -(w_k - w0_k),
// so C_k - C_a moves by -(Delta_k - Delta_a), Delta = w - w0.  Per pixel, with
// a its recorded label:
//  * gap0 > D = max Delta - min Delta: a stays (no other seed gained enough);
//  * else, from the record {gl, gu, g3, b}: when g3 > max Delta - Delta_a no
//    seed but a and b can be the argmin, and the sign of C_b - C_a, within
//    [gl, gu] - (Delta_b - Delta_a), decides between them; an interval that
//    holds 0 is settled by both costs in FP32 direct form (cost32_bound_rel's
//    rigorous bound), or else by the FP64 rescoring;
//  * else the pixel is re-decided in full: the warp scores the tile's recorded
//    candidate list in FP32 direct form against the recorded bound of the
//    excluded seeds, moved by the largest weight rise and re-expressed
//    relative to the current w_ref; what that cannot settle goes to the FP64
//    rescoring queue.
// A pixel whose label changed moves its moment words from a's cell to the new
// one (lanes with the same pair of cells summed first); the pass starts from
// the recorded moments.  One warp per 32 pixels of a tile.  D, max Delta and
// Delta per seed (float intervals, rounded outwards) and the shift of the
// excluded bound (rounded down) come from the trial-weights kernel.
// ---------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(256)
    tc_band_kernel(const GridDev g, const int ntx, const int nty, const int tlo, const int n,
                   const SeedRec32 *__restrict__ recs_nat, const float *__restrict__ centre,
                   const int4 *__restrict__ meta, const float *__restrict__ texcl, const int *__restrict__ list,
                   const int32_t *__restrict__ lab0, const float *__restrict__ gap0,
                   const float4 *__restrict__ rec0, const float2 *__restrict__ drift,
                   unsigned long long *__restrict__ gmom, uint32_t *__restrict__ flags,
                   int32_t *__restrict__ flag_gi, DevScalars *__restrict__ sc, const int wide) {
    using G = TcGeom<D>;
    constexpr int KM = moment_width(D);
    constexpr int kPer = kBandChunk / 256;  // margins per thread and chunk
    const unsigned full_mask = 0xffffffffu;
    if (!*(volatile const int *)&sc->inc_go) return;  // a recording pass: the scorer did it all
    __shared__ uint32_t s_q[kBandChunk];  // the chunk's candidate pixels ...
    __shared__ uint32_t s_f[kBandChunk];  // ... and those left for a full re-decision
    __shared__ unsigned s_nq, s_nf, s_full;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) s_full = 0u;
    float wrh, wrl;
    block_wref(sc, wrh, wrl);  // (its barrier also orders the counter's clearing)
    const float finf = __int_as_float(0x7f800000);
    const float bandD = sc->band_D, drift_hi = sc->drift_hi;
    const long long plane = (long long)g.res[0] * (D == 3 ? g.res[1] : 1);
    const long long jlo = (long long)win_lo(g) * plane, jhi = (long long)win_hi(g) * plane;
    const int tdim[3] = {G::TX, G::TY, G::TZ};
    // pixel j -> grid coordinates, its tile and its position relative to the tile centre
    auto place = [&](long long j, int (&kk)[3], int &t, float (&yp)[3]) {
        kk[0] = (int)(j % g.res[0]);
        const long long r = j / g.res[0];
        kk[1] = D == 3 ? (int)(r % g.res[1]) : (int)r;
        kk[2] = D == 3 ? (int)(r / g.res[1]) : 0;
        const int tx = kk[0] / G::TX, ty = kk[1] / G::TY, tz = D == 3 ? kk[2] / G::TZ : 0;
        t = D == 3 ? tx + ntx * (ty + nty * (tz - tlo)) : tx + ntx * (ty - tlo);
        const int tc[3] = {tx, ty, tz};
#pragma unroll
        for (int d = 0; d < 3; ++d)
            yp[d] = d < D ? ((float)(kk[d] - tc[d] * tdim[d] - tdim[d] / 2) + 0.5f) * g.h32[d] : 0.f;
    };
    for (long long base = jlo + (long long)blockIdx.x * kBandChunk; base < jhi;
         base += (long long)gridDim.x * kBandChunk) {
        if (tid == 0) {
            s_nq = 0u;
            s_nf = 0u;
        }
        __syncthreads();
        // 1. the chunk's margins (coalesced, kPer loads in flight per thread) -> candidates
        float gv[kPer];
#pragma unroll
        for (int e = 0; e < kPer; ++e) {
            const long long j = base + e * 256 + tid;
            gv[e] = j < jhi ? gap0[j] : finf;
        }
#pragma unroll
        for (int e = 0; e < kPer; ++e)
            if (!(gv[e] > bandD)) s_q[atomicAdd(&s_nq, 1u)] = (uint32_t)(base + e * 256 + tid);
        __syncthreads();
        const unsigned nq = s_nq;
        // 2. one thread per candidate: keep a, or decide between a and b
        for (unsigned i0 = 0; i0 < nq; i0 += 256) {
            const unsigned i = i0 + (unsigned)tid;
            const bool act = i < nq;
            long long j = 0;
            int kk[3] = {0, 0, 0}, t = 0;
            float yp[3] = {0.f, 0.f, 0.f};
            int a0 = -1, nl = -1, b = -1, hint = -1;
            bool flag = false;
            if (act) {
                j = s_q[i];
                a0 = lab0[j];
                if (a0 < 0 || a0 >= n) {  // no valid record (its pass failed): leave the pixel alone
                    atomicOr(&sc->status, ST_BAD_LABEL);
                    a0 = -1;
                }
            }
            if (a0 >= 0) {
                const float4 rc = rec0[j];
                b = __float_as_int(rc.w);
                const float2 da = drift[a0];
                // every seed but a and b: C_k - C_a >= g3 - (Delta_k - Delta_a) >= g3 - (max Delta - Delta_a)
                const float thr = __fsub_ru(drift_hi, da.x);
                if (!(rc.z > thr)) {
                    s_f[atomicAdd(&s_nf, 1u)] = (uint32_t)j;  // a full re-decision
                } else if (b < 0 || b >= n) {
                    nl = a0;
                } else {
                    const float2 db = drift[b];
                    const float lo = __fsub_rd(rc.x, __fsub_ru(db.y, da.x));  // C_b - C_a, rounded outwards
                    const float hi = __fsub_ru(rc.y, __fsub_rd(db.x, da.y));
                    if (lo > 0.f) {
                        nl = a0;
                    } else if (hi < 0.f) {
                        nl = b;
                    } else {  // a against b in FP32 direct form
                        place(j, kk, t, yp);
                        float ch[3] = {0.f, 0.f, 0.f}, cl[3] = {0.f, 0.f, 0.f};
#pragma unroll
                        for (int d = 0; d < D; ++d) {
                            ch[d] = centre[(size_t)t * 6 + d];
                            cl[d] = centre[(size_t)t * 6 + 3 + d];
                        }
                        float ca, ea, cb, eb;
                        cost32_bound_rel<D>(recs_nat[a0], ch, cl, yp, wrh, wrl, ca, ea);
                        cost32_bound_rel<D>(recs_nat[b], ch, cl, yp, wrh, wrl, cb, eb);
                        if (__fadd_ru(ca, ea) < __fsub_rd(cb, eb)) nl = a0;
                        else if (__fadd_ru(cb, eb) < __fsub_rd(ca, ea)) nl = b;
                        else {
                            flag = true;
                            hint = a0;
                        }
                    }
                }
            }
            // near ties to the FP64 rescoring (which moves their words from a's cell)
            const unsigned qm = __ballot_sync(full_mask, flag);
            if (qm) {
                unsigned qb = 0u;
                if (lane == __ffs(qm) - 1) qb = atomicAdd(&sc->flag_count, (unsigned)__popc(qm));
                qb = __shfl_sync(full_mask, qb, __ffs(qm) - 1);
                if (flag) {
                    const unsigned slot = qb + (unsigned)__popc(qm & ((1u << lane) - 1u));
                    flags[slot] = (uint32_t)j;
                    if (flag_gi) flag_gi[slot] = hint;
                }
            }
            // moved pixels: their words leave a's cell for the new one, summed per
            // pair of cells across the warp (neighbouring candidates share pairs)
            const bool moved = nl >= 0 && nl != a0;
            if (moved) place(j, kk, t, yp);
            unsigned todo = __ballot_sync(full_mask, moved);
            while (todo) {
                const int leader = __ffs(todo) - 1;
                const int A0 = __shfl_sync(full_mask, a0, leader), NL = __shfl_sync(full_mask, nl, leader);
                const bool mine = moved && a0 == A0 && nl == NL;
                const unsigned grp = __ballot_sync(full_mask, mine);
                unsigned long long u[3] = {0ull, 0ull, 0ull};
#pragma unroll
                for (int d = 0; d < D; ++d) u[d] = mine ? 2ull * (unsigned long long)kk[d] + 1ull : 0ull;
                unsigned long long word = 0ull;
                int e = 0;
                auto fold = [&](unsigned long long x) {
                    if (!wide) {
                        // u < 2^13: every product is below 2^26 and 32 of them below 2^31
                        x = __reduce_add_sync(full_mask, (unsigned)x);
                    } else {
#pragma unroll
                        for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(full_mask, x, off);
                    }
                    if (lane == e) word = x;
                    ++e;
                };
                fold(mine ? 1ull : 0ull);
#pragma unroll
                for (int d = 0; d < D; ++d) fold(u[d]);
#pragma unroll
                for (int d = 0; d < D; ++d)
#pragma unroll
                    for (int d2 = d; d2 < D; ++d2) fold(u[d] * u[d2]);
                if (lane < KM && word) {
                    atomicAdd(&gmom[(size_t)NL * KM + lane], word);
                    atomicAdd(&gmom[(size_t)A0 * KM + lane], 0ull - word);
                }
                todo &= ~grp;
            }
        }
        __syncthreads();
        // 3. full re-decisions, one warp per pixel: lanes over its tile's recorded
        // candidate list, against the excluded seeds' bound moved by the drift
        const unsigned nf = s_nf;
        if (tid == 0) s_full += nf;
        for (unsigned f = (unsigned)wid; f < nf; f += 8u) {
            const long long j = s_f[f];
            int kk[3], t;
            float yp[3];
            place(j, kk, t, yp);
            const int a0 = lab0[j];
            const int cnt = meta[t].w;
            const int ns = (cnt + kN - 1) / kN;
            float ch[3] = {0.f, 0.f, 0.f}, cl[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int d = 0; d < D; ++d) {
                ch[d] = centre[(size_t)t * 6 + d];
                cl[d] = centre[(size_t)t * 6 + 3 + d];
            }
            const float t0 = texcl[t];
            const float tex = t0 < finf ? __fadd_rd(t0, sc->band_shift) : finf;
            float cv[kMaxSteps], ev[kMaxSteps];
            int lv[kMaxSteps];
            float ub = finf;
            int us = 0x7fffffff;
#pragma unroll
            for (int k = 0; k < kMaxSteps; ++k) {
                lv[k] = k * kN + lane < cnt ? list[(size_t)t * kListCap + k * kN + lane] : -1;
                cv[k] = finf;
                ev[k] = 0.f;
                if (k < ns && lv[k] >= 0) {
                    cost32_bound_rel<D>(recs_nat[lv[k]], ch, cl, yp, wrh, wrl, cv[k], ev[k]);
                    const float u1 = __fadd_ru(cv[k], ev[k]);
                    if (u1 < ub || (u1 == ub && lv[k] < us)) {
                        ub = u1;
                        us = lv[k];
                    }
                }
            }
            const unsigned kub = okey(ub);
            const unsigned kmin = __reduce_min_sync(full_mask, kub);
            const int smin = (int)__reduce_min_sync(full_mask, kub == kmin ? (unsigned)us : 0x7fffffffu);
            const float Ub = okey_inv(kmin);
            bool other = false;
#pragma unroll
            for (int k = 0; k < kMaxSteps; ++k)
                if (k < ns && lv[k] >= 0 && lv[k] != smin && !(__fsub_rd(cv[k], ev[k]) > Ub)) other = true;
            const bool ok2 = !__any_sync(full_mask, other) && Ub < tex && smin < n;
            if (!ok2) {
                if (lane == 0) {
                    const unsigned slot = atomicAdd(&sc->flag_count, 1u);
                    flags[slot] = (uint32_t)j;
                    if (flag_gi) flag_gi[slot] = smin < n ? smin : -1;
                }
            } else if (smin != a0 && lane < KM) {
                // this pixel's words from a's cell to smin's
                unsigned long long u[3] = {0ull, 0ull, 0ull};
#pragma unroll
                for (int d = 0; d < D; ++d) u[d] = 2ull * (unsigned long long)kk[d] + 1ull;
                unsigned long long word = 0ull;
                int e = 0;
                auto put = [&](unsigned long long x) {
                    if (lane == e) word = x;
                    ++e;
                };
                put(1ull);
#pragma unroll
                for (int d = 0; d < D; ++d) put(u[d]);
#pragma unroll
                for (int d = 0; d < D; ++d)
#pragma unroll
                    for (int d2 = d; d2 < D; ++d2) put(u[d] * u[d2]);
                atomicAdd(&gmom[(size_t)smin * KM + lane], word);
                atomicAdd(&gmom[(size_t)a0 * KM + lane], 0ull - word);
            }
        }
        __syncthreads();  // the queues are refilled by the next chunk
    }
    if (tid == 0 && s_full) atomicAdd(&sc->band_count, s_full);
}

template <int D>
cudaError_t launch_band_t(const GridDev &g, int n, Workspace &ws, cudaStream_t st) {
    int ntx = 0, nty = 0, tlo = 0;
    long long ntl = 0;
    tile_grid<D>(g, ntx, nty, tlo, ntl);
    if (ntl > ws.tc_tile_cap || !ws.inc_labels || !ws.inc_gap || !ws.inc_rec || !ws.inc_drift)
        return cudaErrorInvalidValue;
    // chunks of kBandChunk pixels, grid-strided over as many blocks as stay resident
    // together (a recording pass launches it for nothing)
    int &bps = ws.band_bps[D == 3 ? 1 : 0];
    if (!bps) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, tc_band_kernel<D>, 256, 0) != cudaSuccess || bps < 1)
            bps = 2;
        cudaGetLastError();
    }
    const long long plane = (long long)g.res[0] * (D == 3 ? g.res[1] : 1);
    const long long pix = (long long)(win_hi(g) - win_lo(g)) * plane;
    const long long blocks =
        std::max<long long>(1, std::min<long long>((pix + kBandChunk - 1) / kBandChunk, (long long)ws.sms * bps));
    const int wide = (g.res[0] > 4096 || g.res[1] > 4096 || (D == 3 && g.res[2] > 4096)) ? 1 : 0;
    tc_band_kernel<D><<<(unsigned)blocks, 256, 0, st>>>(
        g, ntx, nty, tlo, n, ws.recs32, ws.tc_centre, ws.tc_meta, ws.tc_texcl, ws.tc_list, ws.inc_labels, ws.inc_gap,
        ws.inc_rec, ws.inc_drift, ws.moments, ws.flags, ws.flag_gi, ws.sc, wide);
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

cudaError_t launch_tc_axis(const GridDev &g, Workspace &ws, cudaStream_t st) {
    int ntx = 0, nty = 0, tlo = 0;
    long long ntl = 0;
    if (g.dim == 3) {
        tile_grid<3>(g, ntx, nty, tlo, ntl);
        if (ntl > ws.tc_tile_cap) return cudaSuccess;  // scored by the FP32 kernel
        return ensure_axis<3>(g, ntx, nty, (int)(ntl / ((long long)ntx * nty)), tlo, ws, st);
    }
    tile_grid<2>(g, ntx, nty, tlo, ntl);
    if (ntl > ws.tc_tile_cap) return cudaSuccess;
    return ensure_axis<2>(g, ntx, nty, 0, tlo, ws, st);
}

cudaError_t launch_tc_band(const GridDev &g, int n, Workspace &ws, cudaStream_t st) {
    return g.dim == 3 ? launch_band_t<3>(g, n, ws, st) : launch_band_t<2>(g, n, ws, st);
}

long long tc_tile_count(const GridDev &g) {
    int ntx = 0, nty = 0, tlo = 0;
    long long ntl = 0;
    if (g.dim == 3) tile_grid<3>(g, ntx, nty, tlo, ntl);
    else tile_grid<2>(g, ntx, nty, tlo, ntl);
    return ntl;
}

int tc_list_cap() { return kListCap; }
size_t tc_bops_bytes_per_tile() { return (size_t)kMaxSteps * kBMax; }

}  // namespace apd
