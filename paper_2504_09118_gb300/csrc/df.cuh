// Compensated FP32 arithmetic for the energy and divergence reductions.
//
// GB300 executes FP64 at a small fraction of its FP32 rate, so the reductions form every term from
// FP32 error-free transformations instead of FP64 operations:
//   * two_sum (Knuth, TAOCP vol. 2, 4.2.2): s = fl(a + b) and the exact error e = (a + b) - s;
//   * two_prod with a fused multiply-add: p = fl(a b) and the exact error e = a b - p;
//   * the compensated dot product Dot2 of Ogita, Rump and Oishi ("Accurate sum and dot product",
//     SIAM J. Sci. Comput. 26(6), 2005): partial sums carried as an unevaluated pair, so that the result
//     is as accurate as a product sum computed with twice the FP32 precision (about 2^-48) and then
//     rounded.
// A lane accumulates one row's terms in such a pair and adds it to an FP64 sum once per row; every
// intrinsic below rounds to nearest and is not contracted by the compiler.
#pragma once

#include <cuda_runtime.h>

namespace fdtd {
namespace df {

// a + b = s + e exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    const float t = __fadd_rn(a, b);
    const float bb = __fsub_rn(t, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(t, bb)), __fsub_rn(b, bb));
    s = t;
}

// a b = p + e exactly.
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
    const float t = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -t);
    p = t;
}

// A value held as the unevaluated sum hi + lo.
struct F2 {
    float hi, lo;
};

// 1/c as a pair: hi is the correctly rounded reciprocal, lo corrects it from the exact residual
// 1 - c hi (one fused multiply-add), so hi + lo = 1/c to about 2^-48 relative.
__device__ __forceinline__ F2 recip(float c) {
    F2 r;
    r.hi = __frcp_rn(c);
    r.lo = __fmul_rn(__fmaf_rn(-c, r.hi, 1.0f), r.hi);
    return r;
}

// (a - b) - (c - d) as a pair, to about 2^-48 of |a - b| + |c - d|.
__device__ __forceinline__ F2 diff2(float a, float b, float c, float d) {
    float x, ex, y, ey, s, es;
    two_sum(a, -b, x, ex);
    two_sum(c, -d, y, ey);
    two_sum(x, -y, s, es);
    return F2{s, __fadd_rn(es, __fsub_rn(ex, ey))};
}

// x (y.hi + y.lo) as a pair: x y.hi exactly as two floats, then x y.lo into the low part.
__device__ __forceinline__ F2 mul(float x, F2 y) {
    float h, e;
    two_prod(x, y.hi, h, e);
    return F2{h, __fmaf_rn(x, y.lo, e)};
}

// Dot2 accumulator: sum of products and pairs.
struct Acc {
    float p = 0.f, s = 0.f;
    // += x y
    __device__ __forceinline__ void prod(float x, float y) {
        float h, r, q;
        two_prod(x, y, h, r);
        two_sum(p, h, p, q);
        s = __fadd_rn(s, __fadd_rn(q, r));
    }
    // += x (a term whose own rounding error is negligible: corrections 2^-24 below the main terms)
    __device__ __forceinline__ void small(float x) { s = __fadd_rn(s, x); }
    // += x (y.hi + y.lo)
    __device__ __forceinline__ void prod(float x, F2 y) {
        prod(x, y.hi);
        small(__fmul_rn(x, y.lo));
    }
    // += x^2 c with c a pair: x^2 = p2 + e2 exactly, then p2 c.hi compensated, p2 c.lo + e2 c.hi small
    __device__ __forceinline__ void sq_times(float x, F2 c) {
        float p2, e2;
        two_prod(x, x, p2, e2);
        prod(p2, c.hi);
        small(__fmaf_rn(p2, c.lo, __fmul_rn(e2, c.hi)));
    }
    // the accumulated value as a pair with |lo| <= ulp(hi) / 2
    __device__ __forceinline__ F2 pair() const {
        F2 r;
        two_sum(p, s, r.hi, r.lo);
        return r;
    }
    // += (v.hi + v.lo)^2 (the lo^2 term is 2^-48 below and dropped)
    __device__ __forceinline__ void square(F2 v) {
        prod(v.hi, v.hi);
        small(__fmul_rn(__fmul_rn(2.0f, v.hi), v.lo));
    }
    // the accumulated value in FP64, and a fresh start
    __device__ __forceinline__ double take() {
        const double r = (double)p + (double)s;
        p = s = 0.f;
        return r;
    }
};

}  // namespace df
}  // namespace fdtd
