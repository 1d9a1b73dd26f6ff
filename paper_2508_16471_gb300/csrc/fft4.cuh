// Register-resident "four-step" FFT for power-of-two lengths L = R1 * R2
// (R1 >= R2, both <= 32), used by the FP32 fast path of the operator.
//
// With n = n1 R2 + n2 and k = k1 + R1 k2:
//   X[k1 + R1 k2] = sum_{n2} w_R2^{n2 k2} ( w_L^{n2 k1} sum_{n1} w_R1^{n1 k1} x[n1 R2 + n2] )
// Step 1 (one thread per n2): R1-point DFT of the stride-R2 subsequence held in
// registers, then the twiddle w_L^{n2 k1}; the R1 x R2 intermediate goes
// through shared memory once; step 2 (one thread per k1): R2-point DFT.  The
// inverse runs the same steps in reverse order with conjugate roots.  Data
// enter and leave through registers straight from/to global memory.
#pragma once

#include "fft.cuh"

namespace vie {

#define VIE_C32_1 0.98078528040323044913
#define VIE_C32_3 0.83146961230254523708
#define VIE_C32_5 0.55557023301960222474
#define VIE_C32_7 0.19509032201612826785

// w_32^k = exp(-+ 2 pi i k / 32), k = 0..15
template <typename T, bool INV> __device__ __forceinline__ cplx<T> w32(int k) {
    const T c[9] = {(T)1.0, (T)VIE_C32_1, (T)VIE_COS_PI8, (T)VIE_C32_3, (T)VIE_SQRT1_2,
                    (T)VIE_C32_5, (T)VIE_SIN_PI8, (T)VIE_C32_7, (T)0.0};
    // angle 2 pi k / 32 for k in [0, 16): cos = c[k] (k <= 8) or -c[16-k]; sin = c[8-k] (k <= 8) or c[k-8]
    T cs, sn;
    if (k <= 8) {
        cs = c[k];
        sn = c[8 - k];
    } else {
        cs = -c[16 - k];
        sn = c[k - 8];
    }
    return INV ? cplx<T>{cs, sn} : cplx<T>{cs, -sn};
}

template <typename T, bool INV> __device__ __forceinline__ void dft32(cplx<T>* a) {
    cplx<T> E[16], O[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        E[k] = a[2 * k];
        O[k] = a[2 * k + 1];
    }
    dft16<T, INV>(E);
    dft16<T, INV>(O);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        cplx<T> t = w32<T, INV>(k) * O[k];
        a[k] = E[k] + t;
        a[k + 16] = E[k] - t;
    }
}

template <typename T, int R, bool INV> __device__ __forceinline__ void dftp2(cplx<T>* a) {
    if constexpr (R == 1) {
    } else if constexpr (R == 2) dft2<T, INV>(a[0], a[1]);
    else if constexpr (R == 4) dft4<T, INV>(a[0], a[1], a[2], a[3]);
    else if constexpr (R == 8) dft8<T, INV>(a);
    else if constexpr (R == 16) dft16<T, INV>(a);
    else dft32<T, INV>(a);
}

// Factorisations used by the fast path.
template <int L> struct Fac;
template <> struct Fac<16> { static constexpr int R1 = 4, R2 = 4; };
template <> struct Fac<32> { static constexpr int R1 = 8, R2 = 4; };
template <> struct Fac<64> { static constexpr int R1 = 8, R2 = 8; };
template <> struct Fac<128> { static constexpr int R1 = 16, R2 = 8; };
template <> struct Fac<256> { static constexpr int R1 = 16, R2 = 16; };
template <> struct Fac<512> { static constexpr int R1 = 32, R2 = 16; };



}  // namespace vie
