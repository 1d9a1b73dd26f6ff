// Shared device/host helpers of the VIE library: complex arithmetic on
// float2/double2-like structs, error plumbing, launch accounting.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>

#include "../../include/vie.h"

namespace vie {

// True the first time it is asked, per flag, for the current device (one bit
// per device, ordinals below 64): kernel attributes such as the dynamic
// shared-memory limit are set per device.
inline bool first_on_device(std::atomic<unsigned long long>& done) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return true;
    }
    const unsigned long long bit = 1ull << dev;
    return (done.fetch_or(bit) & bit) == 0;
}


template <typename T> struct cplx { T x, y; };
template <> struct __align__(8) cplx<float> { float x, y; };
template <> struct __align__(16) cplx<double> { double x, y; };

using c32 = cplx<float>;
using c64 = cplx<double>;

template <typename T> __host__ __device__ __forceinline__ cplx<T> mk(T a, T b) { return {a, b}; }
template <typename T> __host__ __device__ __forceinline__ cplx<T> operator+(cplx<T> a, cplx<T> b) {
    return {a.x + b.x, a.y + b.y};
}
template <typename T> __host__ __device__ __forceinline__ cplx<T> operator-(cplx<T> a, cplx<T> b) {
    return {a.x - b.x, a.y - b.y};
}
// FP32 complex sums and differences as one packed FP32x2 instruction on the
// device (round to nearest, the same result per part as two scalar adds).
__host__ __device__ __forceinline__ cplx<float> operator+(cplx<float> a, cplx<float> b) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
    const float2 r = __fadd2_rn(make_float2(a.x, a.y), make_float2(b.x, b.y));
    return {r.x, r.y};
#else
    return {a.x + b.x, a.y + b.y};
#endif
}
__host__ __device__ __forceinline__ cplx<float> operator-(cplx<float> a, cplx<float> b) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
    // a - b = fma(b, -1, a): exact negation, one rounding
    const float2 r = __ffma2_rn(make_float2(b.x, b.y), make_float2(-1.0f, -1.0f), make_float2(a.x, a.y));
    return {r.x, r.y};
#else
    return {a.x - b.x, a.y - b.y};
#endif
}
template <typename T> __host__ __device__ __forceinline__ cplx<T> operator*(cplx<T> a, cplx<T> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T> __host__ __device__ __forceinline__ cplx<T> operator*(T s, cplx<T> a) {
    return {s * a.x, s * a.y};
}
template <typename T> __host__ __device__ __forceinline__ cplx<T> conjg(cplx<T> a) { return {a.x, -a.y}; }
// a * conj(b)
template <typename T> __host__ __device__ __forceinline__ cplx<T> mulc(cplx<T> a, cplx<T> b) {
    return {a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}
template <typename T> __host__ __device__ __forceinline__ T abs2(cplx<T> a) { return a.x * a.x + a.y * a.y; }

template <typename To, typename Ti> __host__ __device__ __forceinline__ cplx<To> cvt(cplx<Ti> a) {
    return {(To)a.x, (To)a.y};
}

// ---- error plumbing -------------------------------------------------------
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* where);

#define VIE_CUDA(call)                                                    \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) return ::vie::cuda_fail(e_, #call);        \
    } while (0)

#define VIE_TRY(call)                  \
    do {                               \
        int s_ = (call);               \
        if (s_ != VIE_OK) return s_;   \
    } while (0)

// launches of library kernels (host-side counter)
void count_launch(long long n = 1);

// optional per-kernel event timing (vie_timer_*)
enum TimerId {
    TMR_ZFWD = 0, TMR_YFWD, TMR_XFUSED, TMR_YINV, TMR_ZINV, TMR_DOTS, TMR_REDUCE, TMR_UPDATE,
    TMR_FINISH, TMR_SCALE, TMR_XUPDATE, TMR_RESIDUAL, TMR_START, TMR_RHS, TMR_OTHER, TMR_MV64, TMR_REORTH, TMR_MVDF, TMR_SWEEP, TMR_FFGEMM, TMR_FFOTHER,
    TMR_COUNT
};
bool tmr_enabled();
// bytes (and events, counted as launches with no time) known only after a host synchronisation
void tmr_add(int id, double bytes, long long count);
void tmr_begin(int id, cudaStream_t s);
void tmr_end(int id, cudaStream_t s, double bytes = 0.0);

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace vie
