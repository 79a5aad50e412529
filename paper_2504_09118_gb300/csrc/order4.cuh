// The staggered fourth-order difference of the (2,4) Yee scheme, shared by every kernel that
// computes with it (unfused step, fused step, reductions) so that all of them round alike.
//
// Sec. 6 of the paper names higher-order schemes as the way to raise FDTD's arithmetic intensity
// on accelerators; the scheme here replaces each difference of Eq. 2 by
//     D f(p) = c1 [f(p + 1/2) - f(p - 1/2)] + c2 [f(p + 3/2) - f(p - 3/2)],  c1 = 9/8, c2 = -1/24,
// and closes the PEC walls by image theory: about a wall the tangential E is odd and the
// tangential H even.  A tap past a wall therefore mirrors onto an inner tap of the same
// difference, and the image folds into that tap's weight:
//   * D of E at H index m (inner taps m, m + 1): the tap m - 1 = -1 mirrors onto m + 1 with sign
//     -1, so for m = 0 the weight of tap m + 1 becomes c1 + c2; for m = n - 1 the tap n + 1 mirrors
//     onto n - 1 (= m) and that weight becomes c1 + c2 (E at index n is zero, tangential);
//   * D of H at E index i (inner taps i - 1, i): for i = 1 the tap -1 mirrors onto 0 (= i - 1);
//     for i = n - 1 the tap n mirrors onto n - 1 (= i).
// The same weights serve the divergences (normal E even, normal H odd about a wall).  A tap past
// a wall is then read as 0, so the difference is
//     wb * b - wa * a + c2 * (b2 - a2),   evaluated as fma(c2, b2 - a2, fma(-wa, a, wb * b)).
#pragma once

#include <cuda_runtime.h>

namespace fdtd {
namespace o4 {

constexpr float kC1 = 1.125f;                  // 9/8 (exact)
constexpr float kC2 = (float)(-1.0 / 24.0);    // -1/24, rounded to FP32
constexpr float kC12 = (float)(13.0 / 12.0);   // c1 + c2: an inner tap that absorbs its image

// a2, a: outer and inner taps below the point; b, b2: inner and outer taps above it.
__device__ __forceinline__ float d4(float a2, float a, float b, float b2, float wa, float wb) {
    return __fmaf_rn(kC2, __fsub_rn(b2, a2), __fmaf_rn(-wa, a, __fmul_rn(wb, b)));
}

#ifndef FDTD_O4_PACKED
#define FDTD_O4_PACKED 1   // 1: the two cells of a lane in packed FP32x2 instructions (same rounding; measured
                           // 2-3 % faster than per-element instructions in the fused fourth-order kernel)
#endif

// a * b + c and a - b on the two cells of a lane (one rounding per element either way).
__device__ __forceinline__ float2 fma2o(float2 a, float2 b, float2 c) {
#if FDTD_O4_PACKED
    return __ffma2_rn(a, b, c);
#else
    return make_float2(__fmaf_rn(a.x, b.x, c.x), __fmaf_rn(a.y, b.y, c.y));
#endif
}
__device__ __forceinline__ float2 sub2o(float2 a, float2 b) {
#if FDTD_O4_PACKED
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);   // rounds exactly like a - b
#else
    return make_float2(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y));
#endif
}

__device__ __forceinline__ float2 d4(float2 a2, float2 a, float2 b, float2 b2, float2 wa, float2 wb) {
#if FDTD_O4_PACKED
    const float2 t = __ffma2_rn(make_float2(-wa.x, -wa.y), a, __fmul2_rn(wb, b));
    return __ffma2_rn(make_float2(kC2, kC2), sub2o(b2, a2), t);
#else
    return make_float2(d4(a2.x, a.x, b.x, b2.x, wa.x, wb.x), d4(a2.y, a.y, b.y, b2.y, wa.y, wb.y));
#endif
}

// Inner-tap weights of a difference of E at H index m of n cells along its axis.
__device__ __forceinline__ float wa_h(int m, int n) { return m == n - 1 ? kC12 : kC1; }
__device__ __forceinline__ float wb_h(int m, int n) { return m == 0 ? kC12 : kC1; }
// Inner-tap weights of a difference of H at E index i of n cells along its axis.
__device__ __forceinline__ float wa_e(int i, int n) { return i == 1 ? kC12 : kC1; }
__device__ __forceinline__ float wb_e(int i, int n) { return i == n - 1 ? kC12 : kC1; }

}  // namespace o4
}  // namespace fdtd
