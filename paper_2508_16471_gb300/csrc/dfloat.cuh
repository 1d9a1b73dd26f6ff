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
// the two cross terms.
//
// GB300 runs FP32 at about 64 times its FP64 rate, so an FFT in double-float
// arithmetic (roughly 10 FP32 operations per FP64 operation) outruns the
// same transform in FP64 while matching its accuracy within a few units of
// 2^-47.  Nothing here may be reassociated: the library is built without
// fast-math, and no products appear in the additions for FMA contraction to
// merge.
#pragma once

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
    const float p = x.hi * y.hi;
#if defined(__CUDA_ARCH__)
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
#else
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

using cdf = cplx<dfl>;

// complex double-float from / to complex double
__host__ __device__ __forceinline__ cdf to_cdf(c64 a) { return cdf{dfl(a.x), dfl(a.y)}; }
__host__ __device__ __forceinline__ c64 to_c64(cdf a) { return c64{to_double(a.x), to_double(a.y)}; }

}  // namespace vie
