// Shared-memory mbarriers and bulk copies (cp.async.bulk, completed through an
// mbarrier's transaction count), used by the tensor-core kernels and the
// staged transfer passes.  Every wait is bounded by kSpinLimit polls; the
// caller turns a timeout into an error flag.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

namespace h2 {

constexpr uint32_t kSpinLimit = 1u << 25;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Non-blocking test of a phase (acquire semantics when it reports completion):
// a caller issues it ahead of the work it overlaps and reads the result later.
__device__ __forceinline__ bool mbar_test(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity) {
    for (uint32_t i = 0; i < kSpinLimit; ++i)
        if (mbar_try(b, parity)) return true;
    return false;
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
// dst, src 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// L2 policies for bulk copies: data streamed once (evict first) and data read again
// by later copies (evict last).
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
// bulk_g2s with an L2 cache policy
__device__ __forceinline__ void bulk_g2s_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                              uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

// Byte offset of element (row r, column c) of a core-matrix tile whose rows hold
// kp values of es bytes (kp·es a multiple of 16): 8-row groups outermost, then
// 16-byte column chunks, then the 8 rows of 16 bytes of one core matrix.
__host__ __device__ __forceinline__ int64_t cm_off(int r, int c, int kp, int es) {
    const int per = 16 / es;
    return ((int64_t)(r >> 3) * (kp / per) + (c / per)) * 128 + (r & 7) * 16 + (c % per) * es;
}

// Rows 2i (high part) and 2i + 1 (low part) at contraction indices κ0 .. κ0+3
// (κ0 % 4 == 0) of a split activation tile with kp columns: es = 4 (TF32):
// v and v - tf32(v), the MMA reading the top 19 bits of the first; es = 2
// (BF16): bf16(v) and bf16(v - bf16(v)).  One 16- or 8-byte store per row.
__device__ __forceinline__ void put_act4(uint8_t* tile, int kp, int es, int i, int kappa0, const float (&v)[4]) {
    if (es == 4) {
        float4 hi, lo;
        hi.x = v[0]; hi.y = v[1]; hi.z = v[2]; hi.w = v[3];
        lo.x = v[0] - __uint_as_float(__float_as_uint(v[0]) & 0xFFFFE000u);
        lo.y = v[1] - __uint_as_float(__float_as_uint(v[1]) & 0xFFFFE000u);
        lo.z = v[2] - __uint_as_float(__float_as_uint(v[2]) & 0xFFFFE000u);
        lo.w = v[3] - __uint_as_float(__float_as_uint(v[3]) & 0xFFFFE000u);
        *(float4*)(tile + cm_off(2 * i, kappa0, kp, 4)) = hi;
        *(float4*)(tile + cm_off(2 * i + 1, kappa0, kp, 4)) = lo;
    } else {
        uint32_t h[2] = {0u, 0u}, l[2] = {0u, 0u};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const __nv_bfloat16 bh = __float2bfloat16_rn(v[u]);
            const __nv_bfloat16 bl = __float2bfloat16_rn(v[u] - __bfloat162float(bh));
            h[u >> 1] |= (uint32_t)__bfloat16_as_ushort(bh) << (16 * (u & 1));
            l[u >> 1] |= (uint32_t)__bfloat16_as_ushort(bl) << (16 * (u & 1));
        }
        *(uint2*)(tile + cm_off(2 * i, kappa0, kp, 2)) = make_uint2(h[0], h[1]);
        *(uint2*)(tile + cm_off(2 * i + 1, kappa0, kp, 2)) = make_uint2(l[0], l[1]);
    }
}

}  // namespace h2
