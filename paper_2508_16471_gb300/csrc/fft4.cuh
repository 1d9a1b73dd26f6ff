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
        cplx<T> t = rootmul<T, 32, INV>(O[k], k);
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

// R-point DFT whose inputs a[R/2 .. R) are zero (the zero-padded half):
// X[2m] = DFT_{R/2}(a)[m], X[2m+1] = DFT_{R/2}(a[n] w_R^n)[m]; reads a[0..R/2),
// writes a[0..R).
template <typename T, int R, bool INV> __device__ __forceinline__ void dftp2_half_in(cplx<T>* a) {
    if constexpr (R == 1) {
    } else if constexpr (R == 2) {
        a[1] = a[0];
    } else {
        constexpr int H = R / 2;
        cplx<T> E[H], O[H];
#pragma unroll
        for (int n = 0; n < H; ++n) {
            E[n] = a[n];
            O[n] = rootmul<T, R, INV>(a[n], n);
        }
        dftp2<T, H, INV>(E);
        dftp2<T, H, INV>(O);
#pragma unroll
        for (int m = 0; m < H; ++m) {
            a[2 * m] = E[m];
            a[2 * m + 1] = O[m];
        }
    }
}

// R-point DFT of which only the outputs X[0 .. R/2) are wanted (the crop):
// X[n] = E[n] + w_R^n O[n] with E, O the DFTs of the even and odd inputs;
// writes a[0..R/2).
template <typename T, int R, bool INV> __device__ __forceinline__ void dftp2_half_out(cplx<T>* a) {
    if constexpr (R == 1) {
    } else if constexpr (R == 2) {
        a[0] = a[0] + a[1];
    } else {
        constexpr int H = R / 2;
        cplx<T> E[H], O[H];
#pragma unroll
        for (int n = 0; n < H; ++n) {
            E[n] = a[2 * n];
            O[n] = a[2 * n + 1];
        }
        dftp2<T, H, INV>(E);
        dftp2<T, H, INV>(O);
#pragma unroll
        for (int n = 0; n < H; ++n) a[n] = E[n] + rootmul<T, R, INV>(O[n], n);
    }
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
