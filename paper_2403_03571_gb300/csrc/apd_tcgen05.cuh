// Thin inline-PTX wrappers for the 5th-generation tensor cores (tcgen05) of
// sm_100/sm_103: tensor-memory allocation, the MMA with operands in shared
// memory and the FP32 accumulator in tensor memory, commit to an mbarrier,
// and the tensor-memory -> register loads of the epilogue.
#pragma once

#include <stdint.h>

namespace apd {
namespace tc {

// ---- tensor memory allocation (one warp executes these) ----------------------
__device__ __forceinline__ void tmem_alloc(uint32_t *smem_slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(smem_slot)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// ---- ordering between thread synchronisation and tcgen05 operations ----------
__device__ __forceinline__ void fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// generic-proxy shared-memory writes -> visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---- descriptors ---------------------------------------------------------------
// Byte offset of element (row, k) of a K-major operand without swizzling: the
// operand is tiled in "core matrices" of 8 rows x 16 bytes (128 contiguous
// bytes, row r of a core matrix at 16 r); `lbo` is the byte distance between
// core matrices adjacent along K, `sbo` between core matrices adjacent along
// M (or N); eb = bytes per element.
__host__ __device__ __forceinline__ uint32_t core_offset(int row, int k, int eb, uint32_t lbo, uint32_t sbo) {
    const int epr = 16 / eb;  // elements per 16-byte core-matrix row
    return (uint32_t)(row >> 3) * sbo + (uint32_t)(k / epr) * lbo + (uint32_t)(row & 7) * 16u +
           (uint32_t)(k % epr) * (uint32_t)eb;
}

// Shared-memory matrix descriptor of such an operand starting at shared
// address saddr (16-byte aligned).
__host__ __device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3ffffu) >> 4);          // bits 0-13: start address / 16
    d |= (uint64_t)((lbo >> 4) & 0x3fffu) << 16;        // bits 16-29: leading byte offset / 16
    d |= (uint64_t)((sbo >> 4) & 0x3fffu) << 32;        // bits 32-45: stride byte offset / 16
    d |= (uint64_t)1 << 46;                             // bits 46-48: fixed 0b001
    // base offset 0, relative LBO mode, swizzle none (bits 61-63 = 0)
    return d;
}

enum Kind { KIND_TF32 = 0, KIND_BF16 = 1 };

// Instruction descriptor: FP32 accumulator, A and B K-major, M x N tile.
__host__ __device__ constexpr uint32_t instr_desc(int kind, int M, int N) {
    return (1u << 4)                                   // D format: F32
           | ((kind == KIND_TF32 ? 2u : 1u) << 7)      // A format: TF32 (tf32 kind) / BF16 (f16 kind)
           | ((kind == KIND_TF32 ? 2u : 1u) << 10)     // B format
           | ((uint32_t)(N >> 3) << 17)                // N / 8
           | ((uint32_t)(M >> 4) << 24);               // M / 16
}

// D[tmem] (+)= A[smem] * B[smem]^T, issued by one thread.
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// arrive on an mbarrier when all previously issued MMAs of this thread complete
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(bar))
                 : "memory");
}

// ---- tensor memory -> registers: 32 lanes x 32 consecutive 32-bit columns ------
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// The same load with a min-reduction (sm_103): mn receives the smallest of the
// thread's 32 loaded values.
__device__ __forceinline__ void tmem_ld32_min(uint32_t taddr, float (&v)[32], float &mn) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.red.sync.aligned.32x32b.x32.min.f32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, %32, [%33];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=f"(mn)
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 8 consecutive columns with their minimum.
__device__ __forceinline__ void tmem_ld8_min(uint32_t taddr, float (&v)[8], float &mn) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.red.sync.aligned.32x32b.x8.min.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, %8, [%9];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=f"(mn)
                 : "r"(taddr)
                 : "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// ---- rounding to the operand formats ------------------------------------------
__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

}  // namespace tc
}  // namespace apd
