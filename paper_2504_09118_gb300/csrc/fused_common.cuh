// Device helpers shared by the fused step kernels (one and two leapfrog steps per HBM pass).
#pragma once

#include "fdtd_internal.cuh"

namespace fdtd {
namespace fused {

#ifndef FDTD_SCALAR_MATH
#define FDTD_SCALAR_MATH 1   // 1: per-element fmaf (measured faster); 0: packed FP32x2 instructions (same rounding)
#endif

// a * b + c on the two cells of a lane (one rounding per element).
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
#if FDTD_SCALAR_MATH
    return make_float2(__fmaf_rn(a.x, b.x, c.x), __fmaf_rn(a.y, b.y, c.y));
#else
    return __ffma2_rn(a, b, c);
#endif
}

// a - b on the two cells of a lane: fma(b, -1, a) rounds exactly like a - b.
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
#if FDTD_SCALAR_MATH
    return make_float2(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y));
#else
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
#endif
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

#ifndef FDTD_CHECK
#define FDTD_CHECK 0   // 1: every global store and TMA x origin of the fused kernels is checked first
#endif

// Checked builds (FDTD_CHECK=1, the library variant built beside the normal one): an access that would
// leave its buffer, or a TMA x origin off the 16-byte granule, is skipped and STATUS_BADINDEX latched
// (reported by the next synchronising call).  In normal builds both checks are constant `true`.
__device__ __forceinline__ bool store_ok(int *status, long long g, long long n, long long elems) {
#if FDTD_CHECK
    if (g < 0 || g + n > elems) {
        atomicOr(status, STATUS_BADINDEX);
        return false;
    }
#endif
    return true;
}
__device__ __forceinline__ bool tma_x_ok(int *status, int x, int esize) {
#if FDTD_CHECK
    if (((long long)x * esize) % 16 != 0) {
        atomicOr(status, STATUS_BADINDEX);
        return false;
    }
#endif
    return true;
}

// Named barrier over `nthreads` threads that also ORs a predicate across them.
__device__ __forceinline__ bool bar_sync_or(int id, int nthreads, bool pred) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "barrier.cta.red.or.pred p, %2, %3, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(id), "r"(nthreads)
        : "memory");
    return r != 0;
}

// Two adjacent storage elements <-> two floats.  16-bit storage holds E scaled by s_E and
// H scaled by s_H; the kernel computes in those scaled units (the ratio s_E/s_H is folded
// into the coefficients of its tile records), so loads and stores are plain conversions.
// st_cs stores with the streaming (evict-first) cache hint: a launch never re-reads what it
// writes, so its outputs should not push the neighbouring tiles' halo rows out of L2.
template <typename T> struct Pair;
template <> struct Pair<float> {
    __device__ __forceinline__ static float2 ld(const float *p) { return *reinterpret_cast<const float2 *>(p); }
    __device__ __forceinline__ static float ld1(const float *p) { return *p; }
    __device__ __forceinline__ static void st(float *p, float a, float b) {
        *reinterpret_cast<float2 *>(p) = make_float2(a, b);
    }
    __device__ __forceinline__ static void st_cs(float *p, float a, float b) {
        __stcs(reinterpret_cast<float2 *>(p), make_float2(a, b));
    }
};
template <> struct Pair<__half> {
    __device__ __forceinline__ static float2 ld(const __half *p) {
        return __half22float2(*reinterpret_cast<const __half2 *>(p));
    }
    __device__ __forceinline__ static float ld1(const __half *p) { return __half2float(*p); }
    __device__ __forceinline__ static void st(__half *p, float a, float b) {
        *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(a, b);
    }
    __device__ __forceinline__ static void st_cs(__half *p, float a, float b) {
        __stcs(reinterpret_cast<__half2 *>(p), __floats2half2_rn(a, b));
    }
};
template <> struct Pair<__nv_bfloat16> {
    __device__ __forceinline__ static float2 ld(const __nv_bfloat16 *p) {
        return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(p));
    }
    __device__ __forceinline__ static float ld1(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
    __device__ __forceinline__ static void st(__nv_bfloat16 *p, float a, float b) {
        *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(a, b);
    }
    __device__ __forceinline__ static void st_cs(__nv_bfloat16 *p, float a, float b) {
        __stcs(reinterpret_cast<__nv_bfloat162 *>(p), __floats2bfloat162_rn(a, b));
    }
};


}  // namespace fused
}  // namespace fdtd
