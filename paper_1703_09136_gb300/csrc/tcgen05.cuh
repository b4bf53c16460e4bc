// tcgen05 / TMA / mbarrier helpers shared by the tensor-core kernels
// (sm_103a inline PTX).  Every mbarrier wait is bounded by TC_SPIN polls and
// reports a timeout instead of hanging.
#pragma once

#include <cstdint>

#include <cuda_fp16.h>

namespace tc {

// Bounded mbarrier waits: each poll suspends the thread until the phase
// completes or TC_SUSPEND_NS pass (a woken thread returns at once), so
// waiting warps leave the issue slots to the copy and MMA threads; TC_SPIN
// polls (the default; plans may set their own) bound a wait at about 2 s,
// after which the caller reports a timeout.
constexpr long TC_SPIN = 2000000;
#define TC_SUSPEND_NS "1000"

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t sbo = 512) {
    // no-swizzle K-major canonical layout: core matrices of 8 rows x 16 B;
    // K-direction core stride (LBO) 128 B, M/N-direction core stride (SBO)
    // 512 B for K chunks of 64 B per row (4 cores), 256 B for 32 B (2 cores)
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)(128 >> 4) << 16;
    d |= (uint64_t)(sbo >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long spin = TC_SPIN) {
    const uint32_t a = su32(bar);
    for (long it = 0; it < spin; ++it) {
        uint32_t ok;
        asm volatile("{\n\t.reg .pred P;\n\tmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2, " TC_SUSPEND_NS ";\n\t"
                     "selp.u32 %0, 1, 0, P;\n\t}\n" : "=r"(ok) : "r"(a), "r"(parity) : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(su32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(su32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(su32(dst)), "l"(src), "r"(bytes), "r"(su32(bar)) : "memory");
}

// 8-byte asynchronous global -> shared copy (completed by cp_async_wait_all).
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" :: "r"(su32(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// Bring [src, src + bytes) into L2 ahead of a later bulk copy (16-byte aligned, multiple of 16).
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" :: "l"(src), "r"(bytes) : "memory");
}

// D (FP32, TMEM) (+)= A B^T with f16 A and B (both f16: kind::f16 takes one
// operand type), K = 16 per instruction.
__device__ __forceinline__ void mma_f16(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
                 :: "r"(dtmem), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}

// Instruction descriptor of kind::f16 with f16 A and B (K-major), FP32 D, M = 128.
__host__ __device__ constexpr uint32_t idesc_f16(int n) {
    return (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(n >> 3) << 17) | ((128u >> 4) << 24);
}

// Power-of-two exponent e that puts m * 2^e in [2^14, 2^15) (0 for m == 0),
// from the float's exponent field; clamped to [-120, 120].
__device__ __forceinline__ int f16_exp(float m) {
    if (!(m > 0.0f)) return 0;
    const int bx = (__float_as_int(m) >> 23) & 0xff;
    const int e = bx == 0 ? 120 : 141 - bx;
    return e < -120 ? -120 : (e > 120 ? 120 : e);
}

// 2^e for e in [-126, 127].
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

// x = hi + lo to 22 bits in two f16 (x already scaled below 2^15); raw bits.
__device__ __forceinline__ void split_f16(float x, uint16_t& h, uint16_t& l) {
    const __half hh = __float2half_rn(x);
    h = __half_as_ushort(hh);
    l = __half_as_ushort(__float2half_rn(x - __half2float(hh)));
}

__device__ __forceinline__ uint4 pack8(const uint16_t (&v)[8]) {
    return make_uint4((uint32_t)v[0] | ((uint32_t)v[1] << 16), (uint32_t)v[2] | ((uint32_t)v[3] << 16),
                      (uint32_t)v[4] | ((uint32_t)v[5] << 16), (uint32_t)v[6] | ((uint32_t)v[7] << 16));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(su32(bar)) : "memory");
}

}  // namespace tc
