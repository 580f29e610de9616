// spd_device.cuh -- device helpers shared by the detect kernels: packed
// (SNR, code) floats, packed f32x2 arithmetic, 1-D bulk (TMA) copies with a
// time-bounded mbarrier wait, vector loads of stored samples and
// double-float sums.
#pragma once
#include "spd_internal.cuh"

#include <math.h>

namespace spd {

namespace {

constexpr int kWaitLimit = 1 << 22;          // polls, a backstop to the time bound
constexpr uint32_t kSuspendNs = 20000;       // suspend hint of one poll

__device__ __forceinline__ float packw(float s, uint32_t code) {
    return __uint_as_float((__float_as_uint(s) & 0xFFFFFFC0u) | code);
}
__device__ __forceinline__ float trunc17(float s) {
    return __uint_as_float(__float_as_uint(s) & 0xFFFFFFC0u);
}

__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

__device__ __forceinline__ float fmin3(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// ------------------------------------------------------------- bulk copies

__device__ __forceinline__ uint32_t saddr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(bar)) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// One arrival that also expects `bytes` of bulk-copy completion.
__device__ __forceinline__ void mbar_expect(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes,
                                          uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(saddr(dst)), "l"(src), "r"(bytes), "r"(saddr(bar))
        : "memory");
}
// One poll; the thread may be suspended (up to kSuspendNs) until the phase
// completes instead of spinning on issue slots.
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(saddr(bar)), "r"(phase), "r"(kSuspendNs)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait for a phase of `bar`: false if it did not complete within
// limit_ns of wall time (or kWaitLimit polls).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t phase, uint64_t limit_ns) {
    if (mbar_test(bar, phase)) return true;
    const uint64_t t0 = global_ns();
    for (int it = 0; it < kWaitLimit; ++it) {
        if (mbar_test(bar, phase)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
    return false;
}

template <int DT>
__device__ __forceinline__ void load4v(const typename Elem<DT>::T *p, float &a, float &b,
                                       float &c, float &d);
template <>
__device__ __forceinline__ void load4v<SPD_F32>(const float *p, float &a, float &b, float &c,
                                                float &d) {
    const float4 v = *reinterpret_cast<const float4 *>(p);
    a = v.x; b = v.y; c = v.z; d = v.w;
}
template <>
__device__ __forceinline__ void load4v<SPD_F16>(const __half *p, float &a, float &b, float &c,
                                                float &d) {
    const uint2 v = *reinterpret_cast<const uint2 *>(p);
    const float2 lo = __half22float2(*reinterpret_cast<const __half2 *>(&v.x));
    const float2 hi = __half22float2(*reinterpret_cast<const __half2 *>(&v.y));
    a = lo.x; b = lo.y; c = hi.x; d = hi.y;
}
template <>
__device__ __forceinline__ void load4v<SPD_BF16>(const __nv_bfloat16 *p, float &a, float &b,
                                                 float &c, float &d) {
    const uint2 v = *reinterpret_cast<const uint2 *>(p);
    const float2 lo = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&v.x));
    const float2 hi = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&v.y));
    a = lo.x; b = lo.y; c = hi.x; d = hi.y;
}

// ------------------------------------------------------- double-float sums

__device__ __forceinline__ float2 two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return make_float2(s, e);
}
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
    float2 s = two_sum(a.x, b.x);
    const float lo = __fadd_rn(s.y, __fadd_rn(a.y, b.y));
    return two_sum(s.x, lo);
}

}  // namespace

}  // namespace spd
