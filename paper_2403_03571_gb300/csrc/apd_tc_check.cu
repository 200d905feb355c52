// Self-check of the tensor-core plumbing used by the tcgen05 scoring path: one
// 128 x 128 x 16 MMA (TF32: two K = 8 steps; BF16: one K = 16 step) from
// shared memory into tensor memory, read back with tcgen05.ld and compared,
// element by element, with the same dot products on CUDA cores.  The operands
// are small integers, exact in TF32 and BF16, so every product and sum is
// exact and any difference is a layout or descriptor error.
#include "apd_internal.cuh"
#include "apd_tcgen05.cuh"

#include <cuda_bf16.h>

namespace apd {
namespace {

constexpr int kM = 128, kN = 128, kK = 16;

__device__ __forceinline__ float check_a(int r, int k) { return (float)(((r * 5 + k * 3) % 9) - 4); }
__device__ __forceinline__ float check_b(int n, int k) { return (float)(((n * 7 + k) % 7) - 3); }

template <int KIND>
__global__ void __launch_bounds__(128) tc_check_kernel(int variant, int *mismatches, unsigned *max_err_bits,
                                                       int *status) {
    constexpr int eb = KIND == tc::KIND_TF32 ? 4 : 2;
    constexpr int epr = 16 / eb;
    constexpr uint32_t LBO = 128;                       // K-adjacent core matrices contiguous
    constexpr uint32_t SBO = (kK / epr) * 128;          // next 8-row group after all K
    __shared__ __align__(1024) uint8_t smA[kM * kK * 4];
    __shared__ __align__(1024) uint8_t smB[kN * kK * 4];
    __shared__ uint64_t bar;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    for (int e = tid; e < kM * kK; e += blockDim.x) {
        const int r = e / kK, k = e % kK;
        const uint32_t oa = tc::core_offset(r, k, eb, LBO, SBO);
        if (KIND == tc::KIND_TF32) {
            *reinterpret_cast<float *>(smA + oa) = check_a(r, k);
            *reinterpret_cast<float *>(smB + oa) = check_b(r, k);
        } else {
            *reinterpret_cast<__nv_bfloat16 *>(smA + oa) = __float2bfloat16(check_a(r, k));
            *reinterpret_cast<__nv_bfloat16 *>(smB + oa) = __float2bfloat16(check_b(r, k));
        }
    }
    if (warp == 0) {
        tc::tmem_alloc(&tslot, 128);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = tslot;
    if (tid == 0) {
        const uint32_t idesc = tc::instr_desc(KIND, kM, kN);
        const uint32_t a0 = (uint32_t)__cvta_generic_to_shared(smA);
        const uint32_t b0 = (uint32_t)__cvta_generic_to_shared(smB);
        constexpr int ksteps = KIND == tc::KIND_TF32 ? 2 : 1;  // K = 8 (TF32) or 16 (BF16) per MMA
        for (int ks = 0; ks < ksteps; ++ks) {
            const uint32_t off = (uint32_t)ks * 2u * LBO;       // two core matrices along K per step
            const uint64_t ad = tc::smem_desc(a0 + off, LBO, SBO);
            const uint64_t bd = tc::smem_desc(b0 + off, LBO, SBO);
            if (KIND == tc::KIND_TF32)
                tc::mma_tf32(taddr, ad, bd, idesc, ks > 0 ? 1u : 0u);
            else
                tc::mma_bf16(taddr, ad, bd, idesc, ks > 0 ? 1u : 0u);
        }
        tc::mma_commit(&bar);
    }
    const bool ok = mbar_wait_bounded(&bar, 0, status);
    tc::fence_after_sync();
    int bad = 0;
    float worst = 0.f;
    if (ok) {
        const int r = warp * 32 + lane;
        for (int c0 = 0; c0 < kN; c0 += 32) {
            float v[32], mn = 0.f;
            if (variant == 2)
                tc::tmem_ld32_min(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v, mn);
            else
                tc::tmem_ld32(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            tc::tmem_wait_ld();
            float ref_min = 3.0e38f;
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                float ref = 0.f;
                for (int k = 0; k < kK; ++k) ref += check_a(r, k) * check_b(c0 + i, k);
                ref_min = fminf(ref_min, ref);
                const float e = fabsf(v[i] - ref);
                if (!(e == 0.f)) ++bad;
                worst = fmaxf(worst, e == e ? e : 3.0e38f);
            }
            // the reduced load's minimum must equal the minimum of the 32 references
            if (variant == 2 && !(mn == ref_min)) ++bad;
        }
    }
    atomicAdd(mismatches, bad);
    atomicMax(max_err_bits, __float_as_uint(worst));
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(taddr, 128);
}

}  // namespace
}  // namespace apd

extern "C" int apd_tensor_core_check(int32_t kind, int32_t variant, int32_t *mismatches, float *max_err) {
    if ((kind != 0 && kind != 1) || (variant != 0 && variant != 2) || !mismatches || !max_err) return APD_ERR_ARG;
    int *d = nullptr;
    if (cudaMalloc((void **)&d, 3 * sizeof(int)) != cudaSuccess) return APD_ERR_CUDA;
    cudaMemset(d, 0, 3 * sizeof(int));
    if (kind == 0)
        apd::tc_check_kernel<apd::tc::KIND_TF32><<<1, 128>>>(variant, d, (unsigned *)(d + 1), d + 2);
    else
        apd::tc_check_kernel<apd::tc::KIND_BF16><<<1, 128>>>(variant, d, (unsigned *)(d + 1), d + 2);
    int h[3] = {0, 0, 0};
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof h, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return APD_ERR_CUDA;
    *mismatches = h[0];
    float w;
    memcpy(&w, &h[1], sizeof w);
    *max_err = w;
    return h[2] ? APD_ERR_TIMEOUT : APD_OK;
}
