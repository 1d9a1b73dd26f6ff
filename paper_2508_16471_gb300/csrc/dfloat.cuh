// Double-float ("float-float") arithmetic for the FP64-accuracy operator.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits (relative rounding ~2^-47).  The operations are
// built from two error-free transformations on FP32 numbers:
//   TwoSum (Knuth, TAOCP vol. 2, 4.2.2): s = fl(a + b) and the exact error
//     e with s + e = a + b, in six additions, for any a, b;
//   TwoProduct via fused multiply-add: p = fl(a b), e = fma(a, b, -p) with
//     p + e = a b exactly (no Dekker splitting needed where FMA exists).
// The sum of two double-floats adds the high parts with TwoSum, folds the
// error and both low parts into one float, and renormalises (the "sloppy"
// sum, whose absolute error is O(2^-47 (|x| + |y|)); the discrete Fourier
// transforms it serves are analysed normwise, so no relative bound under
// cancellation is needed).  The product keeps the exact high product and
// the two cross terms; a complex product forms each part as one two-term dot
// product in the same style.  On the device the complex sums and differences
// run their real and imaginary parts side by side in packed FP32x2
// instructions.
//
// GB300 runs FP32 at about 64 times its FP64 rate, so an FFT in double-float
// arithmetic (roughly 10 FP32 operations per FP64 operation) outruns the
// same transform in FP64 while matching its accuracy within a few units of
// 2^-47.  Nothing here may be reassociated: the library is built without
// fast-math, and the device products that feed additions are formed with the
// round-to-nearest intrinsics, which are never contracted into an FMA.
#pragma once

#include <cmath>

#include "common.cuh"

namespace vie {

struct __align__(8) dfl {
    float hi, lo;
    dfl() = default;
    __host__ __device__ constexpr dfl(float h, float l) : hi(h), lo(l) {}
    // nearest double-float of a double: hi = fl32(d), lo = fl32(d - hi)
    __host__ __device__ dfl(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ dfl(int v) : dfl((double)v) {}
};

__host__ __device__ __forceinline__ double to_double(dfl a) { return (double)a.hi + (double)a.lo; }

// s + e = a + b exactly
__host__ __device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
// s + e = a + b exactly, provided |a| >= |b| (or a == 0)
__host__ __device__ __forceinline__ void quick_two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    e = b - (s - a);
}

__host__ __device__ __forceinline__ dfl operator+(dfl x, dfl y) {
    float s, e;
    two_sum(x.hi, y.hi, s, e);
    e += x.lo + y.lo;
    float h, l;
    quick_two_sum(s, e, h, l);
    return dfl(h, l);
}
__host__ __device__ __forceinline__ dfl operator-(dfl x) { return dfl(-x.hi, -x.lo); }
__host__ __device__ __forceinline__ dfl operator-(dfl x, dfl y) { return x + dfl(-y.hi, -y.lo); }
__host__ __device__ __forceinline__ dfl operator*(dfl x, dfl y) {
#if defined(__CUDA_ARCH__)
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
#else
    const float p = x.hi * y.hi;
    float e = std::fma(x.hi, y.hi, -p);
    e = std::fma(x.hi, y.lo, e);
    e = std::fma(x.lo, y.hi, e);
#endif
    float h, l;
    quick_two_sum(p, e, h, l);
    return dfl(h, l);
}
__host__ __device__ __forceinline__ dfl& operator+=(dfl& x, dfl y) {
    x = x + y;
    return x;
}
__host__ __device__ __forceinline__ dfl& operator-=(dfl& x, dfl y) {
    x = x - y;
    return x;
}

// x1 y1 + x2 y2 as one double-float: the exact high products summed by
// TwoSum, then their rounding errors, the TwoSum error and the four cross
// terms folded into one float and the pair renormalised (the product
// counterpart of the sum above: absolute error O(2^-47 (|x1 y1| + |x2 y2|)),
// 19 FP32 operations where two products and a sum take 25).  The device
// form uses the round-to-nearest intrinsics so that no multiply is
// contracted into an addition.
__host__ __device__ __forceinline__ dfl dot2(dfl x1, dfl y1, dfl x2, dfl y2) {
#if defined(__CUDA_ARCH__)
    const float p1 = __fmul_rn(x1.hi, y1.hi), p2 = __fmul_rn(x2.hi, y2.hi);
    float s, t;
    two_sum(p1, p2, s, t);
    float l = __fadd_rn(__fmaf_rn(x1.hi, y1.hi, -p1), __fmaf_rn(x2.hi, y2.hi, -p2));
    l = __fadd_rn(l, t);
    l = __fmaf_rn(x1.hi, y1.lo, l);
    l = __fmaf_rn(x1.lo, y1.hi, l);
    l = __fmaf_rn(x2.hi, y2.lo, l);
    l = __fmaf_rn(x2.lo, y2.hi, l);
#else
    const float p1 = x1.hi * y1.hi, p2 = x2.hi * y2.hi;
    float s, t;
    two_sum(p1, p2, s, t);
    float l = std::fma(x1.hi, y1.hi, -p1) + std::fma(x2.hi, y2.hi, -p2);
    l += t;
    l = std::fma(x1.hi, y1.lo, l);
    l = std::fma(x1.lo, y1.hi, l);
    l = std::fma(x2.hi, y2.lo, l);
    l = std::fma(x2.lo, y2.hi, l);
#endif
    float h, e;
    quick_two_sum(s, l, h, e);
    return dfl(h, e);
}

// Complex double-float: 16-byte aligned, so that one vector load or store
// moves a whole element.
template <> struct __align__(16) cplx<dfl> { dfl x, y; };
using cdf = cplx<dfl>;

// Complex sums and differences.  On the device the real and the imaginary
// part go through the same steps side by side as packed FP32x2 instructions
// (each lane rounds to nearest, like the scalar operation), which halves the
// instruction count of the FFT butterflies; elsewhere the scalar operations
// above.  A difference x - y is formed as x + (-y) with the
// negations folded into the steps: every value is the one the scalar sum of
// x and -y gives.
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
namespace dfp {
__device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b = fma(b, -1, a): exact negation, one rounding
__device__ __forceinline__ float2 sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 his(cdf a) { return make_float2(a.x.hi, a.y.hi); }
__device__ __forceinline__ float2 los(cdf a) { return make_float2(a.x.lo, a.y.lo); }
// renormalised double-floats (h, l) per lane from s + e
__device__ __forceinline__ cdf quick(float2 s, float2 e) {
    const float2 h = add(s, e);
    const float2 l = sub(e, sub(h, s));
    return cdf{dfl(h.x, l.x), dfl(h.y, l.y)};
}
// the sum (xh + xl) + (yh + yl) per lane: TwoSum of the high parts, the
// error and both low parts folded into one float, renormalised
__device__ __forceinline__ cdf sum(float2 xh, float2 xl, float2 yh, float2 yl) {
    const float2 s = add(xh, yh);
    const float2 bb = sub(s, xh);
    float2 e = add(sub(xh, sub(s, bb)), sub(yh, bb));
    e = add(e, add(xl, yl));
    return quick(s, e);
}
// (xh + xl) - (yh + yl) per lane, the same steps on -y
__device__ __forceinline__ cdf diff(float2 xh, float2 xl, float2 yh, float2 yl) {
    const float2 s = sub(xh, yh);
    const float2 bb = sub(s, xh);
    float2 e = sub(sub(xh, sub(s, bb)), add(yh, bb));
    e = add(e, sub(xl, yl));
    return quick(s, e);
}
}  // namespace dfp
#endif

__host__ __device__ __forceinline__ cdf operator+(cdf a, cdf b) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
    return dfp::sum(dfp::his(a), dfp::los(a), dfp::his(b), dfp::los(b));
#else
    return cdf{a.x + b.x, a.y + b.y};
#endif
}
__host__ __device__ __forceinline__ cdf operator-(cdf a, cdf b) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
    return dfp::diff(dfp::his(a), dfp::los(a), dfp::his(b), dfp::los(b));
#else
    return cdf{a.x - b.x, a.y - b.y};
#endif
}
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
// a w_8 or a w_8^3 (see the generic root8): the sum or difference of a and
// -+i a in packed form, then the packed product with 1/sqrt2
__device__ __forceinline__ cdf root8(cdf a, bool inv, bool three) {
    const dfl h = dfl(0.70710678118654752440);
    // i' a with i' = +i (inverse) or -i (forward)
    const float2 rh = inv ? make_float2(-a.y.hi, a.x.hi) : make_float2(a.y.hi, -a.x.hi);
    const float2 rl = inv ? make_float2(-a.y.lo, a.x.lo) : make_float2(a.y.lo, -a.x.lo);
    const cdf r = three ? dfp::diff(rh, rl, dfp::his(a), dfp::los(a)) : dfp::sum(dfp::his(a), dfp::los(a), rh, rl);
    const float2 hh = make_float2(h.hi, h.hi), hl = make_float2(h.lo, h.lo);
    const float2 xh = dfp::his(r), xl = dfp::los(r);
    const float2 p = __fmul2_rn(hh, xh);
    float2 e = __ffma2_rn(hh, xh, make_float2(-p.x, -p.y));
    e = __ffma2_rn(hh, xl, e);
    e = __ffma2_rn(hl, xh, e);
    return dfp::quick(p, e);
}
#endif

// complex product: each part one two-term dot product
__host__ __device__ __forceinline__ cdf operator*(cdf a, cdf b) {
    return cdf{dot2(a.x, b.x, -a.y, b.y), dot2(a.x, b.y, a.y, b.x)};
}

// complex double-float from / to complex double
__host__ __device__ __forceinline__ cdf to_cdf(c64 a) { return cdf{dfl(a.x), dfl(a.y)}; }
__host__ __device__ __forceinline__ c64 to_c64(cdf a) { return c64{to_double(a.x), to_double(a.y)}; }

}  // namespace vie
