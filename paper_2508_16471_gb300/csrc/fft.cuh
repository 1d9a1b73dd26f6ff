// Shared-memory mixed-radix Stockham FFT engine (radices 16, 8, 4, 2, 3, 5, 7).
//
// The zero-padded convolution of Sec. II-C needs many short 1-D transforms
// (lengths P = smallest 2,3,5,7-smooth size >= 2n-1) along each grid axis.
// A CTA holds a tile of `nl` lines in shared memory in "column" layout:
// element p of line l lives at s[p * ld + l].  Each Stockham stage of radix R
// reads R elements of stride L/R into registers, applies the stage twiddles,
// performs an R-point DFT in registers and writes the results in autosorted
// position; two buffers alternate between stages.  Twiddles are precomputed
// on the host in FP64 (rounded once to the working precision) and staged in
// shared memory, or read from global memory (through L1) for lengths whose
// tables would crowd the line buffers out of shared memory.
//
// Forward transforms use exp(-2 pi i j k / L), inverse exp(+2 pi i j k / L),
// both unnormalised.
#pragma once

#include "common.cuh"

namespace vie {

constexpr int FFT_MAX_STAGES = 10;
constexpr int FFT_MAX_L = 8192;

struct FFTPlan {
    int L;
    int nst;
    int R[FFT_MAX_STAGES];
    int Ns[FFT_MAX_STAGES];
    int twoff[FFT_MAX_STAGES];
    int twlen;  // total twiddle entries
    // division by the stage span Ns and by L as a multiply-high:
    // x / d = umulhi(x, ceil(2^32 / d)) for x d < 2^32 (0 when d = 1)
    unsigned int nsmag[FFT_MAX_STAGES];
    unsigned int lmag;
};

// x / d for the divisors of a plan (d >= 1, x d < 2^32)
__device__ __forceinline__ int div_mag(int x, int d, unsigned int mag) {
    return d == 1 ? x : (int)__umulhi((unsigned int)x, mag);
}
// log2 of a power of two
__device__ __forceinline__ int log2_p2(int v) { return __ffs(v) - 1; }

// ---- small DFTs in registers ----------------------------------------------
// multiply by -i (forward) or +i (inverse)
template <typename T, bool INV> __device__ __forceinline__ cplx<T> mul_mi(cplx<T> a) {
    return INV ? cplx<T>{-a.y, a.x} : cplx<T>{a.y, -a.x};
}

template <typename T, bool INV> __device__ __forceinline__ void dft2(cplx<T>& a0, cplx<T>& a1) {
    cplx<T> t = a0;
    a0 = t + a1;
    a1 = t - a1;
}

template <typename T, bool INV>
__device__ __forceinline__ void dft4(cplx<T>& a0, cplx<T>& a1, cplx<T>& a2, cplx<T>& a3) {
    cplx<T> t0 = a0 + a2, t1 = a0 - a2, t2 = a1 + a3, t3 = mul_mi<T, INV>(a1 - a3);
    a0 = t0 + t2;
    a2 = t0 - t2;
    a1 = t1 + t3;
    a3 = t1 - t3;
}

#define VIE_SQRT1_2 0.70710678118654752440
#define VIE_COS_PI8 0.92387953251128675613
#define VIE_SIN_PI8 0.38268343236508977173

// cos(2 pi m / 32) for m = 0..8 (the first octant; the rest by symmetry)
template <typename T> __device__ __forceinline__ T cos32(int m) {
    switch (m) {
        case 0: return (T)1.0;
        case 1: return (T)0.98078528040323044913;
        case 2: return (T)VIE_COS_PI8;
        case 3: return (T)0.83146961230254523708;
        case 4: return (T)VIE_SQRT1_2;
        case 5: return (T)0.55557023301960222474;
        case 6: return (T)VIE_SIN_PI8;
        case 7: return (T)0.19509032201612826785;
        default: return (T)0.0;
    }
}

// a (1 -+ i) / sqrt2 = a w_8 (three = false) or a (-1 -+ i) / sqrt2 = a w_8^3
// (three = true); the lower sign for the inverse.  Types with a faster form
// overload it.
template <typename T> __device__ __forceinline__ cplx<T> root8(cplx<T> a, bool inv, bool three) {
    const T h = (T)VIE_SQRT1_2;
    if (!three)
        return inv ? cplx<T>{h * (a.x - a.y), h * (a.x + a.y)} : cplx<T>{h * (a.x + a.y), h * (a.y - a.x)};
    return inv ? cplx<T>{-h * (a.x + a.y), h * (a.x - a.y)} : cplx<T>{h * (a.y - a.x), -h * (a.x + a.y)};
}

// a * w_N^k, w_N = exp(-+ 2 pi i / N), N a divisor of 32, 0 <= k < N.  Used
// with k known after unrolling: the multiples of pi/4 reduce to sign swaps
// or one shared scaling, instead of a full complex product with 0 / +-1
// entries that IEEE rules (signed zeros, NaN) forbid the compiler to drop.
template <typename T, int N, bool INV> __device__ __forceinline__ cplx<T> rootmul(cplx<T> a, int k) {
    const T h = (T)VIE_SQRT1_2;
    if (k == 0) return a;
    if (4 * k == N) return mul_mi<T, INV>(a);
    if (2 * k == N) return cplx<T>{-a.x, -a.y};
    if (4 * k == 3 * N) return mul_mi<T, !INV>(a);
    if (8 * k == N) return root8(a, INV, false);
    if (8 * k == 3 * N) return root8(a, INV, true);
    // general root: angle 2 pi m / 32, m = 32 k / N in (0, 32)
    const int m = k * (32 / N);
    const int q = m & 7, oct = m >> 3;  // octant and offset within it
    T c = cos32<T>(q), sn = cos32<T>(8 - q);  // cos and sin of 2 pi q / 32
    T cs, si;
    switch (oct) {
        case 0: cs = c; si = sn; break;
        case 1: cs = -sn; si = c; break;
        case 2: cs = -c; si = -sn; break;
        default: cs = sn; si = -c; break;
    }
    const cplx<T> w = INV ? cplx<T>{cs, si} : cplx<T>{cs, -si};
    return w * a;
}

template <typename T, bool INV> __device__ __forceinline__ void dft8(cplx<T>* a) {
    // even / odd split: E = DFT4(a0,a2,a4,a6), O = DFT4(a1,a3,a5,a7)
    cplx<T> e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
    cplx<T> o0 = a[1], o1 = a[3], o2 = a[5], o3 = a[7];
    dft4<T, INV>(e0, e1, e2, e3);
    dft4<T, INV>(o0, o1, o2, o3);
    cplx<T> E[4] = {e0, e1, e2, e3}, O[4] = {o0, o1, o2, o3};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        cplx<T> t = rootmul<T, 8, INV>(O[k], k);
        a[k] = E[k] + t;
        a[k + 4] = E[k] - t;
    }
}

template <typename T, bool INV> __device__ __forceinline__ void dft16(cplx<T>* a) {
    cplx<T> E[8], O[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        E[k] = a[2 * k];
        O[k] = a[2 * k + 1];
    }
    dft8<T, INV>(E);
    dft8<T, INV>(O);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        cplx<T> t = rootmul<T, 16, INV>(O[k], k);
        a[k] = E[k] + t;
        a[k + 8] = E[k] - t;
    }
}

template <typename T, bool INV> __device__ __forceinline__ void dft3(cplx<T>* a) {
    const T s3 = (T)0.86602540378443864676;
    cplx<T> t = a[1] + a[2], d = a[1] - a[2];
    cplx<T> m = {a[0].x - (T)0.5 * t.x, a[0].y - (T)0.5 * t.y};
    // forward: y1 = m - i s3 d, y2 = m + i s3 d
    cplx<T> r = mul_mi<T, INV>(d);
    a[0] = a[0] + t;
    a[1] = {m.x + s3 * r.x, m.y + s3 * r.y};
    a[2] = {m.x - s3 * r.x, m.y - s3 * r.y};
}

// direct DFT for the odd radices 5 and 7: y_q = sum_t a_t exp(-+ 2 pi i t q / R)
template <int R> struct OddRoots;
template <> struct OddRoots<5> {
    __device__ static double c(int k) {
        const double v[5] = {1.0, 0.30901699437494742410, -0.80901699437494742410,
                             -0.80901699437494742410, 0.30901699437494742410};
        return v[k];
    }
    __device__ static double s(int k) {
        const double v[5] = {0.0, 0.95105651629515357212, 0.58778525229247312917,
                             -0.58778525229247312917, -0.95105651629515357212};
        return v[k];
    }
};
template <> struct OddRoots<7> {
    __device__ static double c(int k) {
        const double v[7] = {1.0, 0.62348980185873353053, -0.22252093395631440429,
                             -0.90096886790241912624, -0.90096886790241912624,
                             -0.22252093395631440429, 0.62348980185873353053};
        return v[k];
    }
    __device__ static double s(int k) {
        const double v[7] = {0.0, 0.78183148246802980871, 0.97492791218182360702,
                             0.43388373911755812048, -0.43388373911755812048,
                             -0.97492791218182360702, -0.78183148246802980871};
        return v[k];
    }
};

template <typename T, int R, bool INV> __device__ __forceinline__ void dft_odd(cplx<T>* a) {
    cplx<T> y[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
        cplx<T> acc = a[0];
#pragma unroll
        for (int t = 1; t < R; ++t) {
            const int k = (t * q) % R;
            const T c = (T)OddRoots<R>::c(k);
            const T s = INV ? (T)OddRoots<R>::s(k) : -(T)OddRoots<R>::s(k);
            acc.x += a[t].x * c - a[t].y * s;
            acc.y += a[t].x * s + a[t].y * c;
        }
        y[q] = acc;
    }
#pragma unroll
    for (int q = 0; q < R; ++q) a[q] = y[q];
}

template <typename T, int R, bool INV> __device__ __forceinline__ void dft(cplx<T>* a) {
    if constexpr (R == 2) dft2<T, INV>(a[0], a[1]);
    else if constexpr (R == 4) dft4<T, INV>(a[0], a[1], a[2], a[3]);
    else if constexpr (R == 8) dft8<T, INV>(a);
    else if constexpr (R == 16) dft16<T, INV>(a);
    else if constexpr (R == 3) dft3<T, INV>(a);
    else dft_odd<T, R, INV>(a);
}

// ---- one Stockham stage over nl lines in column layout ---------------------
// nl is a power of two (the lines or columns of the tile); Ns is divided by
// its multiply-high constant.
template <typename T, int R, bool INV>
__device__ __forceinline__ void stockham_stage(const cplx<T>* __restrict__ in, cplx<T>* __restrict__ out,
                                               int L, int Ns, unsigned int nsmag, int nl, int ld,
                                               const cplx<T>* __restrict__ tw) {
    const int nbf = L / R;
    const int total = nbf * nl;
    const int nlsh = log2_p2(nl);
    for (int b = threadIdx.x; b < total; b += blockDim.x) {
        const int l = b & (nl - 1);
        const int j = b >> nlsh;
        cplx<T> a[R];
#pragma unroll
        for (int t = 0; t < R; ++t) a[t] = in[(j + t * nbf) * ld + l];
        const int jq = div_mag(j, Ns, nsmag);
        const int k = j - jq * Ns;
        if (Ns > 1) {
            const cplx<T>* w = tw + k * (R - 1);
#pragma unroll
            for (int t = 1; t < R; ++t) {
                cplx<T> wt = w[t - 1];
                if (INV) wt.y = -wt.y;
                a[t] = a[t] * wt;
            }
        }
        dft<T, R, INV>(a);
        const int base = jq * Ns * R + k;
#pragma unroll
        for (int t = 0; t < R; ++t) out[(base + t * Ns) * ld + l] = a[t];
    }
}

// Full transform of nl lines; data starts in `a`, `b` is scratch of the same
// size.  Returns the buffer holding the result.  Must be called by the whole
// CTA; ends with a __syncthreads().
template <typename T, bool INV>
__device__ cplx<T>* fft_tile(cplx<T>* a, cplx<T>* b, const FFTPlan& p, const cplx<T>* tw, int nl, int ld) {
    cplx<T>* in = a;
    cplx<T>* out = b;
    for (int s = 0; s < p.nst; ++s) {
        const cplx<T>* t = tw + p.twoff[s];
        const int Ns = p.Ns[s];
        const unsigned int mg = p.nsmag[s];
        switch (p.R[s]) {
            case 16: stockham_stage<T, 16, INV>(in, out, p.L, Ns, mg, nl, ld, t); break;
            case 8: stockham_stage<T, 8, INV>(in, out, p.L, Ns, mg, nl, ld, t); break;
            case 4: stockham_stage<T, 4, INV>(in, out, p.L, Ns, mg, nl, ld, t); break;
            case 2: stockham_stage<T, 2, INV>(in, out, p.L, Ns, mg, nl, ld, t); break;
            case 3: stockham_stage<T, 3, INV>(in, out, p.L, Ns, mg, nl, ld, t); break;
            case 5: stockham_stage<T, 5, INV>(in, out, p.L, Ns, mg, nl, ld, t); break;
            default: stockham_stage<T, 7, INV>(in, out, p.L, Ns, mg, nl, ld, t); break;
        }
        __syncthreads();
        cplx<T>* tmp = in;
        in = out;
        out = tmp;
    }
    return in;
}

// The same stages over three tiles at once (the three field components of
// the fused x pass), each with its own scratch: three times the butterflies
// per stage barrier, so narrow tiles keep every thread busy.  Tile c starts
// at a + c cs (its scratch at b + c cs); the return value says where the
// results are (0: a, 1: b).
template <typename T, int R, bool INV>
__device__ __forceinline__ void stockham_stage3(const cplx<T>* __restrict__ in, cplx<T>* __restrict__ out, int cs,
                                                int L, int Ns, unsigned int nsmag, int nl, int ld,
                                                const cplx<T>* __restrict__ tw) {
    const int nbf = L / R;
    const int per = nbf * nl;
    const int nlsh = log2_p2(nl);
    for (int b3 = threadIdx.x; b3 < 3 * per; b3 += blockDim.x) {
        const int c = b3 >= per ? (b3 >= 2 * per ? 2 : 1) : 0;
        const int b = b3 - c * per;
        const int l = b & (nl - 1);
        const int j = b >> nlsh;
        cplx<T> a[R];
#pragma unroll
        for (int t = 0; t < R; ++t) a[t] = in[c * cs + (j + t * nbf) * ld + l];
        const int jq = div_mag(j, Ns, nsmag);
        const int k = j - jq * Ns;
        if (Ns > 1) {
            const cplx<T>* w = tw + k * (R - 1);
#pragma unroll
            for (int t = 1; t < R; ++t) {
                cplx<T> wt = w[t - 1];
                if (INV) wt.y = -wt.y;
                a[t] = a[t] * wt;
            }
        }
        dft<T, R, INV>(a);
        const int base = jq * Ns * R + k;
#pragma unroll
        for (int t = 0; t < R; ++t) out[c * cs + (base + t * Ns) * ld + l] = a[t];
    }
}

template <typename T, bool INV>
__device__ int fft_tile3(cplx<T>* a, cplx<T>* b, int cs, const FFTPlan& p, const cplx<T>* tw, int nl, int ld) {
    int cur = 0;
    for (int s = 0; s < p.nst; ++s) {
        const cplx<T>* in = cur ? b : a;
        cplx<T>* out = cur ? a : b;
        const cplx<T>* t = tw + p.twoff[s];
        const int Ns = p.Ns[s];
        const unsigned int mg = p.nsmag[s];
        switch (p.R[s]) {
            case 16: stockham_stage3<T, 16, INV>(in, out, cs, p.L, Ns, mg, nl, ld, t); break;
            case 8: stockham_stage3<T, 8, INV>(in, out, cs, p.L, Ns, mg, nl, ld, t); break;
            case 4: stockham_stage3<T, 4, INV>(in, out, cs, p.L, Ns, mg, nl, ld, t); break;
            case 2: stockham_stage3<T, 2, INV>(in, out, cs, p.L, Ns, mg, nl, ld, t); break;
            case 3: stockham_stage3<T, 3, INV>(in, out, cs, p.L, Ns, mg, nl, ld, t); break;
            case 5: stockham_stage3<T, 5, INV>(in, out, cs, p.L, Ns, mg, nl, ld, t); break;
            default: stockham_stage3<T, 7, INV>(in, out, cs, p.L, Ns, mg, nl, ld, t); break;
        }
        __syncthreads();
        cur ^= 1;
    }
    return cur;
}

template <typename T>
__device__ __forceinline__ void load_twiddles(cplx<T>* dst, const cplx<T>* __restrict__ src, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// host side: plan construction and twiddle table (FP64, rounded to T on copy)
bool make_plan(int L, FFTPlan* p);
void plan_twiddles(const FFTPlan& p, double* re_im /* [2*twlen] */);

}  // namespace vie
