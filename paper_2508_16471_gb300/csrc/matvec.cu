// FFT-accelerated operator y = w - chi (K * w) on the compact body-voxel
// layout (Sec. II-C: uniform voxels give a Toeplitz/convolution structure, so
// the matrix-vector product is a zero-padded FFT convolution, O(N log N)).
//
// Data flow for a batch of RHS (grid n0 x n1 x n2 = x, y, z; padded P):
//   pass 1  k_zfwd    gather w from the body list, pad z: n2 -> P2, FFT z
//                     -> A [slot][3][n0][n1][P2]
//   pass 2  k_axis    FFT y, pad n1 -> P1              -> B [slot][3][n0][P1][P2]
//   pass 3  k_xfused  FFT x (pad n0 -> P0), 3x3 spectral multiply with the
//                     kernel octant, inverse FFT x, keep n0 rows (in place on B)
//   pass 4  k_axis    inverse FFT y, keep n1 rows      -> A
//   pass 5  k_zinv    inverse FFT z, keep n2, epilogue y = w - chi * u scattered
//                     to the body list
// The 1/(P0 P1 P2) normalisation is folded into the kernel spectrum.
//
// Kernel spectrum: K(m) (Eq. dyadicG sampled on voxel offsets, ball-averaged,
// plus the self term) is embedded in a periodic P0 x P1 x P2 array, transformed
// once in FP64 with the same FFT engine, and one octant (P/2+1 per axis) per
// tensor component is kept: K_ij(m) is even or odd in each axis, so its
// transform is too, and the other octants follow by sign flips.
#include <atomic>
#include <algorithm>
#include <cmath>
#include <cstring>

#include <type_traits>

#include "vie_internal.cuh"

namespace vie {

// ---------------------------------------------------------------------------
// plans
// ---------------------------------------------------------------------------
bool make_plan(int L, FFTPlan* p) {
    if (L < 1 || L > FFT_MAX_L) return false;
    std::memset(p, 0, sizeof(*p));
    p->L = L;
    int r = L, Ns = 1, off = 0;
    const int order[] = {16, 8, 4, 2, 3, 5, 7};
    for (int R : order) {
        while (r % R == 0) {
            if (p->nst >= FFT_MAX_STAGES) return false;
            p->R[p->nst] = R;
            p->Ns[p->nst] = Ns;
            p->twoff[p->nst] = off;
            off += Ns * (R - 1);
            Ns *= R;
            r /= R;
            p->nst++;
        }
    }
    if (r != 1) return false;
    p->twlen = off;
    // multiply-high divisors (exact for x d < 2^32; here x < 2^18 and d <= 8192)
    auto mag = [](int d) -> unsigned int {
        return d <= 1 ? 0u : (unsigned int)((((unsigned long long)1 << 32) + (unsigned long long)d - 1) / d);
    };
    for (int s = 0; s < p->nst; ++s) p->nsmag[s] = mag(p->Ns[s]);
    p->lmag = mag(L);
    return true;
}

void plan_twiddles(const FFTPlan& p, double* reim) {
    for (int s = 0; s < p.nst; ++s) {
        const int R = p.R[s], Ns = p.Ns[s];
        for (int k = 0; k < Ns; ++k)
            for (int t = 1; t < R; ++t) {
                const double ang = -2.0 * M_PI * (double)(t * k) / (double)(Ns * R);
                const int i = p.twoff[s] + k * (R - 1) + (t - 1);
                reim[2 * i] = std::cos(ang);
                reim[2 * i + 1] = std::sin(ang);
            }
    }
}

int smooth_size(int m) {
    int v = std::max(1, m);
    for (;; ++v) {
        int r = v;
        for (int q : {2, 3, 5, 7})
            while (r % q == 0) r /= q;
        if (r == 1) return v;
    }
}

static int upload_twiddles(Operator& op, AxisFFT& a) {
    const int n = std::max(1, a.plan.twlen);
    std::vector<double> t(2 * n, 0.0);
    plan_twiddles(a.plan, t.data());
    std::vector<float> tf(2 * n);
    for (int i = 0; i < 2 * n; ++i) tf[i] = (float)t[i];
    VIE_TRY(dev_alloc(op, (void**)&a.tw64, sizeof(c64) * n));
    VIE_TRY(dev_alloc(op, (void**)&a.tw32, sizeof(c32) * n));
    VIE_CUDA(cudaMemcpy(a.tw64, t.data(), sizeof(c64) * n, cudaMemcpyHostToDevice));
    VIE_CUDA(cudaMemcpy(a.tw32, tf.data(), sizeof(c32) * n, cudaMemcpyHostToDevice));
    std::vector<cdf> td(n);
    for (int i = 0; i < n; ++i) td[i] = cdf{dfl(t[2 * i]), dfl(t[2 * i + 1])};
    VIE_TRY(dev_alloc(op, (void**)&a.twdf, sizeof(cdf) * n));
    VIE_CUDA(cudaMemcpy(a.twdf, td.data(), sizeof(cdf) * n, cudaMemcpyHostToDevice));
    if (fast_length(a.plan.L)) {
        // four-step twiddles w_L^{k1 n2} in two orders: TA[k1][n2] then TB[n2][k1]
        const int L = a.plan.L;
        int R1 = 0, R2 = 0;
        fast_factors(L, &R1, &R2);
        std::vector<float> r(4 * L);
        for (int k1 = 0; k1 < R1; ++k1)
            for (int n2 = 0; n2 < R2; ++n2) {
                const double ang = -2.0 * M_PI * (double)((k1 * n2) % L) / (double)L;
                const float c = (float)std::cos(ang), sn = (float)std::sin(ang);
                r[2 * (k1 * R2 + n2)] = c;
                r[2 * (k1 * R2 + n2) + 1] = sn;
                r[2 * (L + n2 * R1 + k1)] = c;
                r[2 * (L + n2 * R1 + k1) + 1] = sn;
            }
        VIE_TRY(dev_alloc(op, (void**)&a.roots32, sizeof(c32) * 2 * L));
        VIE_CUDA(cudaMemcpy(a.roots32, r.data(), sizeof(c32) * 2 * L, cudaMemcpyHostToDevice));
    }
    return VIE_OK;
}

// Padded length of one axis: the next power of two >= 2n-1 when it costs at
// most 15 % more points than the smallest 2,3,5,7-smooth length (the power of
// two runs on the register four-step kernels), else the smooth length.
int padded_len(int m) {
    const int sm = smooth_size(m);
    int p2 = 1;
    while (p2 < m) p2 *= 2;
    return (p2 <= 512 && p2 * 100 <= sm * 115) ? p2 : sm;
}
int padded_size(int n) { return padded_len(2 * n - 1); }

static int check_tiles(const Operator& op);

int op_init_axes(Operator& op) {
    for (int a = 0; a < 3; ++a) {
        // D2 takes differences of the convolution one cell beyond the grid: P >= 2n
        const int need = op.disc ? 2 * op.n[a] : 2 * op.n[a] - 1;
        op.P[a] = op.P_fixed[a] > 0 ? op.P_fixed[a] : padded_len(need);
        if (op.P[a] < need) return fail(VIE_EINVAL, "padded length below the convolution's span");
        op.H[a] = op.P[a] / 2 + 1;
        if (!make_plan(op.P[a], &op.ax[a].plan))
            return fail(VIE_EINVAL, "padded FFT size " + std::to_string(op.P[a]) + " exceeds the engine limit (8192)");
        VIE_TRY(upload_twiddles(op, op.ax[a]));
    }
    return check_tiles(op);
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ cplx<T> czero() { return cplx<T>{(T)0, (T)0}; }
// vectors in memory (TI) to the arithmetic type (T) and back: the identity,
// or double <-> double-float for the F32X2 operator
template <typename T, typename TI> __device__ __forceinline__ cplx<T> ld_as(const cplx<TI>* p, long long i) {
    if constexpr (std::is_same<T, TI>::value) return p[i];
    else return to_cdf(p[i]);
}
template <typename T, typename TI> __device__ __forceinline__ void st_as(cplx<TI>* p, long long i, cplx<T> v) {
    if constexpr (std::is_same<T, TI>::value) p[i] = v;
    else p[i] = to_c64(v);
}
// multiply-high constant of a runtime divisor d >= 1 (div_mag(x, d, .) exact for x d < 2^32)
__device__ __forceinline__ unsigned int mag_of(int d) {
    return d <= 1 ? 0u : (unsigned int)((0x100000000ull + (unsigned long long)d - 1) / (unsigned long long)d);
}

// Generic contiguous lines: in [count][n_in] -> out [count][n_out], length L.
// Twiddles: staged in shared memory when `stw`, else read from `twg` directly.
// Lines are padded to NL + 1 columns against bank conflicts when NL > 1.
__host__ __device__ __forceinline__ int lines_ld(int NL) { return NL > 1 ? NL + 1 : 1; }

template <typename T>
__device__ __forceinline__ cplx<T>* tw_setup(unsigned char* smraw, const cplx<T>* __restrict__ twg,
                                             const FFTPlan& plan, int stw, const cplx<T>** tw) {
    cplx<T>* s = reinterpret_cast<cplx<T>*>(smraw);
    if (!stw) {
        *tw = twg;
        return s;
    }
    load_twiddles(s, twg, plan.twlen);
    *tw = s;
    return s + ((plan.twlen + 1) & ~1);
}

template <typename T, bool INV>
__global__ void k_lines(const cplx<T>* in, cplx<T>* out, long long count, int n_in,
                        int n_out, FFTPlan plan, const cplx<T>* __restrict__ twg, int NL, int stw) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const cplx<T>* tw;
    const int L = plan.L;
    const int ld = lines_ld(NL);
    cplx<T>* bA = tw_setup<T>(smraw, twg, plan, stw, &tw);
    cplx<T>* bB = bA + L * ld;
    const long long line0 = (long long)blockIdx.x * NL;
    for (int e = threadIdx.x; e < NL * L; e += blockDim.x) {
        const int l = div_mag(e, L, plan.lmag), p = e - l * L;
        const long long line = line0 + l;
        cplx<T> v = czero<T>();
        if (line < count && p < n_in) v = in[line * n_in + p];
        bA[p * ld + l] = v;
    }
    __syncthreads();
    cplx<T>* r = fft_tile<T, INV>(bA, bB, plan, tw, NL, ld);
    const unsigned int omag = mag_of(n_out);
    for (int e = threadIdx.x; e < NL * n_out; e += blockDim.x) {
        const int l = div_mag(e, n_out, omag), p = e - l * n_out;
        const long long line = line0 + l;
        if (line < count) out[line * n_out + p] = r[p * ld + l];
    }
}

// Middle-axis transform: in [outer][n_in][inner] -> out [outer][n_out][inner].
template <typename T, bool INV>
__global__ void k_axis(const cplx<T>* in, cplx<T>* out, long long inner, int n_in,
                       int n_out, FFTPlan plan, const cplx<T>* __restrict__ twg, int TW, int stw) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const cplx<T>* tw;
    const int L = plan.L;
    cplx<T>* bA = tw_setup<T>(smraw, twg, plan, stw, &tw);
    cplx<T>* bB = bA + L * TW;
    const long long ntile = (inner + TW - 1) / TW;
    const long long o = blockIdx.x / ntile;
    const long long i0 = (blockIdx.x - o * ntile) * TW;
    const int twsh = log2_p2(TW);
    for (int e = threadIdx.x; e < L * TW; e += blockDim.x) {
        const int p = e >> twsh, t = e & (TW - 1);
        cplx<T> v = czero<T>();
        if (p < n_in && i0 + t < inner) v = in[(o * n_in + p) * inner + i0 + t];
        bA[p * TW + t] = v;
    }
    __syncthreads();
    cplx<T>* r = fft_tile<T, INV>(bA, bB, plan, tw, TW, TW);
    for (int e = threadIdx.x; e < n_out * TW; e += blockDim.x) {
        const int p = e >> twsh, t = e & (TW - 1);
        if (i0 + t < inner) out[(o * n_out + p) * inner + i0 + t] = r[p * TW + t];
    }
}

// Pass 1: gather compact w, zero-pad z, forward FFT along z.
template <typename T, typename TI>
__global__ void k_zfwd(const cplx<TI>* __restrict__ w, long long w_rstride, const int* __restrict__ list,
                       const int* __restrict__ idx_map, cplx<T>* __restrict__ A, int n0, int n1, int n2,
                       long long Nb, long long nlines, FFTPlan plan, const cplx<T>* __restrict__ twg, int NL,
                       int stw, long long idx_stride) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const cplx<T>* tw;
    const int L = plan.L;
    const int ld = lines_ld(NL);
    cplx<T>* bA = tw_setup<T>(smraw, twg, plan, stw, &tw);
    cplx<T>* bB = bA + L * ld;
    const long long line0 = (long long)blockIdx.x * NL;
    const long long plane = (long long)n0 * n1;
    for (int e = threadIdx.x; e < NL * L; e += blockDim.x) {
        const int l = div_mag(e, L, plan.lmag), p = e - l * L;
        const long long line = line0 + l;
        cplx<T> v = czero<T>();
        if (line < nlines && p < n2) {
            const long long sc = line / plane;
            const long long xy = line - sc * plane;
            const int slot = (int)(sc / 3), c = (int)(sc - (sc / 3) * 3);
            const int vi = idx_map[(long long)list[slot] * idx_stride + xy * n2 + p];
            if (vi >= 0) v = ld_as<T, TI>(w, (long long)list[slot] * w_rstride + c * Nb + vi);
        }
        bA[p * ld + l] = v;
    }
    __syncthreads();
    cplx<T>* r = fft_tile<T, false>(bA, bB, plan, tw, NL, ld);
    for (int e = threadIdx.x; e < NL * L; e += blockDim.x) {
        const int l = div_mag(e, L, plan.lmag), p = e - l * L;
        const long long line = line0 + l;
        if (line < nlines) A[line * L + p] = r[p * ld + l];
    }
}

// Pass 5: inverse FFT along z, crop, epilogue y = w - chi u on body voxels.
template <typename T, typename TI>
__global__ void k_zinv(const cplx<T>* __restrict__ A, const cplx<TI>* __restrict__ w, long long w_rstride,
                       cplx<TI>* __restrict__ y, long long y_rstride, const int* __restrict__ list,
                       const int* __restrict__ idx_map, const T* __restrict__ chi, int n0, int n1, int n2,
                       long long Nb, long long nlines, FFTPlan plan, const cplx<T>* __restrict__ twg, int NL,
                       long long chi_cs, int stw, long long idx_stride) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const cplx<T>* tw;
    const int L = plan.L;
    const int ld = lines_ld(NL);
    cplx<T>* bA = tw_setup<T>(smraw, twg, plan, stw, &tw);
    cplx<T>* bB = bA + L * ld;
    const long long line0 = (long long)blockIdx.x * NL;
    const long long plane = (long long)n0 * n1;
    for (int e = threadIdx.x; e < NL * L; e += blockDim.x) {
        const int l = div_mag(e, L, plan.lmag), p = e - l * L;
        const long long line = line0 + l;
        cplx<T> v = czero<T>();
        if (line < nlines) v = A[line * L + p];
        bA[p * ld + l] = v;
    }
    __syncthreads();
    cplx<T>* r = fft_tile<T, true>(bA, bB, plan, tw, NL, ld);
    const unsigned int n2mag = mag_of(n2);
    for (int e = threadIdx.x; e < NL * n2; e += blockDim.x) {
        const int l = div_mag(e, n2, n2mag), p = e - l * n2;
        const long long line = line0 + l;
        if (line >= nlines) continue;
        const long long sc = line / plane;
        const long long xy = line - sc * plane;
        const int slot = (int)(sc / 3), c = (int)(sc - (sc / 3) * 3);
        const long long rr = list[slot];
        const int vi = idx_map[rr * idx_stride + xy * n2 + p];
        if (vi < 0) continue;
        const cplx<T> u = r[p * ld + l];
        const cplx<T> wv = ld_as<T, TI>(w, rr * w_rstride + c * Nb + vi);
        const T ch = chi[c * chi_cs + vi];
        st_as<T, TI>(y, rr * y_rstride + c * Nb + vi, cplx<T>{wv.x - ch * u.x, wv.y - ch * u.y});
    }
}

// Pass 3: FFT x, spectral multiply by the 3x3 symmetric kernel, inverse FFT x.
// B [slot][3][n0][inner], inner = P1 * P2; updated in place for x < n0.
// Two CTAs per SM: the transform stages are separated by CTA barriers, so a
// second resident CTA keeps the (FP64-bound) pipes busy while one waits.
// Threads of the generic fused x pass: 256, or 192 for double-float, whose
// tile width (100 KB over six L x TW buffers of 16-byte elements: TW L = 1024)
// gives its joint three-component radix-16 stages 3 (L/16) TW = 192
// butterflies, and whose registers then fit without spilling at two CTAs per SM.
template <typename T> struct XG { static constexpr int NT = std::is_same<T, dfl>::value ? 192 : 256; };

template <typename T>
__global__ void __launch_bounds__(XG<T>::NT, 2) k_xfused(cplx<T>* __restrict__ B, int n0, long long inner, int P0, int P1, int P2,
                         const cplx<T>* __restrict__ khat, int H0, int H1, int H2, FFTPlan plan,
                         const cplx<T>* __restrict__ twg, int TW, const cplx<T>* __restrict__ dtab, int dstride,
                         T ksq, int stw, int joint) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const cplx<T>* tw;
    const int L = plan.L;  // == P0
    // three component tiles and one scratch (joint = 0), or three scratch tiles
    // and stages over the three components at once (joint = 1)
    cplx<T>* D[6];
    D[0] = tw_setup<T>(smraw, twg, plan, stw, &tw);
    for (int i = 1; i < (joint ? 6 : 4); ++i) D[i] = D[i - 1] + L * TW;
    // slots vary fastest across the grid, so the CTAs running at one time
    // share few column tiles and their kernel entries stay in L2
    const long long ntile = (inner + TW - 1) / TW;
    const long long nsl = gridDim.x / ntile;
    const long long tile = blockIdx.x / nsl;
    const long long slot = blockIdx.x - tile * nsl;
    const long long i0 = tile * TW;
    cplx<T>* base = B + slot * 3 * (long long)n0 * inner;
    const int twsh = log2_p2(TW);
    for (int e = threadIdx.x; e < 3 * L * TW; e += blockDim.x) {
        const int cp = e >> twsh, t = e & (TW - 1);  // cp = c L + p
        const int c = div_mag(cp, L, plan.lmag), p = cp - c * L;
        cplx<T> v = czero<T>();
        if (p < n0 && i0 + t < inner) v = base[((long long)c * n0 + p) * inner + i0 + t];
        D[c][p * TW + t] = v;
    }
    __syncthreads();
    cplx<T>* cur[3] = {D[0], D[1], D[2]};
    cplx<T>* scr = D[3];
    bool flip = false;  // joint: the components' data sit in D[3..5]
    if (joint) {
        flip = fft_tile3<T, false>(D[0], D[3], L * TW, plan, tw, TW, TW) != 0;
        if (flip)
            for (int c = 0; c < 3; ++c) cur[c] = D[3 + c];
    } else {
        for (int c = 0; c < 3; ++c) {
            cplx<T>* r = fft_tile<T, false>(cur[c], scr, plan, tw, TW, TW);
            if (r != cur[c]) {
                scr = cur[c];
                cur[c] = r;
            }
        }
    }
    // spectral multiply (a thread keeps its column: blockDim is a multiple of TW)
    const long long HH = (long long)H0 * H1 * H2;
    const long long iic = i0 + (threadIdx.x & (TW - 1));
    const int kyc = (int)(iic / P2), kzc = (int)(iic - (iic / P2) * P2);
    for (int e = threadIdx.x; e < L * TW; e += blockDim.x) {
        const int p = e >> twsh;
        const long long ii = iic;
        if (ii >= inner) continue;
        const int ky = kyc, kz = kzc;
        const int kx = p;
        const bool flx = 2 * kx > P0, fly = 2 * ky > P1, flz = 2 * kz > P2;
        const int fx = flx ? P0 - kx : kx, fy = fly ? P1 - ky : ky, fz = flz ? P2 - kz : kz;
        const long long o = ((long long)fx * H1 + fy) * H2 + fz;
        if (dtab) {
            // D2: U_a = G (k^2 W_a + d+_a sum_b d-_b W_b), G scalar and even
            const cplx<T> g = khat[o];
            const cplx<T> dxp = dtab[kx], dxm = dtab[dstride + kx];
            const cplx<T> dyp = dtab[2 * dstride + ky], dym = dtab[3 * dstride + ky];
            const cplx<T> dzp = dtab[4 * dstride + kz], dzm = dtab[5 * dstride + kz];
            const cplx<T> a = cur[0][e], b = cur[1][e], cc = cur[2][e];
            const cplx<T> sd = dxm * a + dym * b + dzm * cc;
            cur[0][e] = g * (ksq * a + dxp * sd);
            cur[1][e] = g * (ksq * b + dyp * sd);
            cur[2][e] = g * (ksq * cc + dzp * sd);
            continue;
        }
        cplx<T> kxx = khat[o], kxy = khat[HH + o], kxz = khat[2 * HH + o];
        cplx<T> kyy = khat[3 * HH + o], kyz = khat[4 * HH + o], kzz = khat[5 * HH + o];
        if (flx ^ fly) kxy = cplx<T>{-kxy.x, -kxy.y};
        if (flx ^ flz) kxz = cplx<T>{-kxz.x, -kxz.y};
        if (fly ^ flz) kyz = cplx<T>{-kyz.x, -kyz.y};
        const cplx<T> a = cur[0][e], b = cur[1][e], cc = cur[2][e];
        cur[0][e] = kxx * a + kxy * b + kxz * cc;
        cur[1][e] = kxy * a + kyy * b + kyz * cc;
        cur[2][e] = kxz * a + kyz * b + kzz * cc;
    }
    __syncthreads();
    if (joint) {
        if (fft_tile3<T, true>(flip ? D[3] : D[0], flip ? D[0] : D[3], L * TW, plan, tw, TW, TW))
            for (int c = 0; c < 3; ++c) cur[c] = (flip ? D[0] : D[3]) + c * L * TW;
    } else {
        for (int c = 0; c < 3; ++c) {
            cplx<T>* r = fft_tile<T, true>(cur[c], scr, plan, tw, TW, TW);
            if (r != cur[c]) {
                scr = cur[c];
                cur[c] = r;
            }
        }
    }
    const unsigned int n0mag = mag_of(n0);
    for (int e = threadIdx.x; e < 3 * n0 * TW; e += blockDim.x) {
        const int cp = e >> twsh, t = e & (TW - 1);  // cp = c n0 + p
        const int c = div_mag(cp, n0, n0mag), p = cp - c * n0;
        if (i0 + t < inner) base[((long long)c * n0 + p) * inner + i0 + t] = cur[c][p * TW + t];
    }
}

// out[i] = nearest double-float of in[i] (complex arrays convert part by part)
__global__ void k_to_dfl(const double* __restrict__ in, dfl* __restrict__ out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = dfl(in[i]);
}
static int to_dfl(const double* in, dfl* out, long long n, cudaStream_t s) {
    if (n <= 0) return VIE_OK;
    k_to_dfl<<<(unsigned)std::min<long long>(4096, (n + 255) / 256), 256, 0, s>>>(in, out, n);
    count_launch();
    VIE_CUDA(cudaGetLastError());
    return VIE_OK;
}

// Periodic embedding of component q of the discrete kernel K(m) (FP64);
// q = 0..5 for xx, xy, xz, yy, yz, zz.
__global__ void k_kernel_circulant(c64* __restrict__ Kc, int q, int n0, int n1, int n2, int P0, int P1, int P2,
                                   double h, double k0, double coef, double self_re, double self_im) {
    const long long tot = (long long)P0 * P1 * P2;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
         i += (long long)gridDim.x * blockDim.x) {
        const int p2 = (int)(i % P2);
        const long long r0 = i / P2;
        const int p1 = (int)(r0 % P1);
        const int p0 = (int)(r0 / P1);
        int m[3];
        bool ok = true;
        const int pp[3] = {p0, p1, p2}, nn[3] = {n0, n1, n2}, PP[3] = {P0, P1, P2};
        for (int a = 0; a < 3; ++a) {
            if (pp[a] <= nn[a] - 1) m[a] = pp[a];
            else if (pp[a] >= PP[a] - nn[a] + 1) m[a] = pp[a] - PP[a];
            else ok = false;
        }
        c64 out = {0, 0};
        const int I[6] = {0, 0, 0, 1, 1, 2}, J[6] = {0, 1, 2, 1, 2, 2};
        if (ok) {
            if (m[0] == 0 && m[1] == 0 && m[2] == 0) {
                if (I[q] == J[q]) out = c64{self_re, self_im};
            } else {
                const double R[3] = {m[0] * h, m[1] * h, m[2] * h};
                const double r = sqrt(R[0] * R[0] + R[1] * R[1] + R[2] * R[2]);
                const double kr = k0 * r;
                double s, c;
                sincos(kr, &s, &c);
                const double gi = coef / (4.0 * M_PI * r);
                const c64 g = {gi * c, gi * s};
                const double ikr = 1.0 / kr, ikr2 = ikr * ikr;
                const c64 A = {1.0 - ikr2, ikr};
                const c64 Bc = {-1.0 + 3.0 * ikr2, -3.0 * ikr};
                const double u[3] = {R[0] / r, R[1] / r, R[2] / r};
                c64 t = {Bc.x * u[I[q]] * u[J[q]], Bc.y * u[I[q]] * u[J[q]]};
                if (I[q] == J[q]) t = t + A;
                out = g * t;
            }
        }
        Kc[i] = out;
    }
}

// D2 scalar kernel on the full periodic index range (m = p or p - P per axis)
__global__ void k_scalar_circulant(c64* __restrict__ Kc, int P0, int P1, int P2, double h, double k0, double coef,
                                   double g0r, double g0i) {
    const long long tot = (long long)P0 * P1 * P2;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
         i += (long long)gridDim.x * blockDim.x) {
        const int p2 = (int)(i % P2);
        const long long r0 = i / P2;
        const int p1 = (int)(r0 % P1), p0 = (int)(r0 / P1);
        const int m0 = 2 * p0 <= P0 ? p0 : p0 - P0, m1 = 2 * p1 <= P1 ? p1 : p1 - P1, m2 = 2 * p2 <= P2 ? p2 : p2 - P2;
        if (m0 == 0 && m1 == 0 && m2 == 0) {
            Kc[i] = c64{g0r, g0i};
        } else {
            const double r = h * sqrt((double)m0 * m0 + (double)m1 * m1 + (double)m2 * m2);
            double s, c;
            sincos(k0 * r, &s, &c);
            const double gi = coef / (4.0 * M_PI * r);
            Kc[i] = c64{gi * c, gi * s};
        }
    }
}

// keep the octant (P/2 + 1 per axis) of one transformed component, scaled
__global__ void k_octant(const c64* __restrict__ Kc, c64* __restrict__ o64, c32* __restrict__ o32, int P0, int P1,
                         int P2, int H0, int H1, int H2, double scale) {
    const long long HH = (long long)H0 * H1 * H2;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < HH;
         i += (long long)gridDim.x * blockDim.x) {
        const int fz = (int)(i % H2);
        const int fy = (int)((i / H2) % H1);
        const int fx = (int)(i / ((long long)H1 * H2));
        const c64 v = Kc[((long long)fx * P1 + fy) * P2 + fz];
        const c64 s = {v.x * scale, v.y * scale};
        o64[i] = s;
        o32[i] = c32{(float)s.x, (float)s.y};
    }
}

// ---------------------------------------------------------------------------
// number of z lines (x, y) with at least one body voxel
__global__ void k_line_count(const int* __restrict__ idx_map, long long nl, int n2, long long* __restrict__ count) {
    const long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (l >= nl) return;
    const int* im = idx_map + l * n2;
    for (int z = 0; z < n2; ++z)
        if (im[z] >= 0) {
            atomicAdd((unsigned long long*)count, 1ull);
            return;
        }
}

// body compaction: idx_map, vox, chi from a device eps grid
// ---------------------------------------------------------------------------
constexpr int SCAN_B = 1024;

// unknown at voxel i: D1 where eps > 1; D2 (face unknowns on the +a faces)
// where the cell or one of its +x/+y/+z neighbours has eps > 1
__device__ __forceinline__ int body_flag(const double* __restrict__ eps, long long i, int n1, int n2, int disc,
                                         long long N) {
    if (eps[i] > 1.0) return 1;
    if (!disc) return 0;
    const int k = (int)(i % n2), j = (int)((i / n2) % n1);
    const long long x = i / ((long long)n1 * n2);
    const long long n0 = N / ((long long)n1 * n2);
    return (x + 1 < n0 && eps[i + (long long)n1 * n2] > 1.0) || (j + 1 < n1 && eps[i + n2] > 1.0) ||
           (k + 1 < n2 && eps[i + 1] > 1.0);
}

__global__ void k_body_count(const double* __restrict__ eps, long long N, int* __restrict__ bcount,
                             int* __restrict__ err, int n1, int n2, int disc) {
    __shared__ int ws[32];
    const long long i = (long long)blockIdx.x * SCAN_B + threadIdx.x;
    int f = 0;
    if (i < N) {
        const double e = eps[i];
        if (!(e >= 1.0) || !isfinite(e)) atomicOr(err, 1);
        else f = body_flag(eps, i, n1, n2, disc, N);
    }
    int s = __syncthreads_count(f);
    (void)ws;
    if (threadIdx.x == 0) bcount[blockIdx.x] = s;
}

// single-CTA exclusive scan of the block counts; writes total to *total
__global__ void k_scan_blocks(int* __restrict__ bcount, int nb, long long* __restrict__ total) {
    __shared__ int carry;
    __shared__ int wsum[32];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += blockDim.x) {
        const int i = base + threadIdx.x;
        int v = i < nb ? bcount[i] : 0;
        // inclusive warp scan
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if ((threadIdx.x & 31) >= o) x += y;
        }
        if ((threadIdx.x & 31) == 31) wsum[threadIdx.x >> 5] = x;
        __syncthreads();
        if (threadIdx.x < 32) {
            int s = threadIdx.x < (blockDim.x >> 5) ? wsum[threadIdx.x] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, s, o);
                if (threadIdx.x >= o) s += y;
            }
            wsum[threadIdx.x] = s;
        }
        __syncthreads();
        const int wpre = (threadIdx.x >> 5) ? wsum[(threadIdx.x >> 5) - 1] : 0;
        const int excl = carry + wpre + x - v;
        if (i < nb) bcount[i] = excl;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

// D1: chi[v] = eps - 1; D2: chi[a Nb + v] = (chi(cell) + chi(cell + e_a)) / 2
__global__ void k_body_write(const double* __restrict__ eps, long long N, const int* __restrict__ boff,
                             int* __restrict__ idx_map, int* __restrict__ vox, float* __restrict__ chi32,
                             double* __restrict__ chi64, int n1, int n2, int disc, long long Nb) {
    __shared__ int wsum[32];
    const long long i = (long long)blockIdx.x * SCAN_B + threadIdx.x;
    const double e = i < N ? eps[i] : 1.0;
    const int f = i < N ? body_flag(eps, i, n1, n2, disc, N) : 0;
    int x = f;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) >= o) x += y;
    }
    if ((threadIdx.x & 31) == 31) wsum[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
        int s = wsum[threadIdx.x];
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (threadIdx.x >= o) s += y;
        }
        wsum[threadIdx.x] = s;
    }
    __syncthreads();
    const int excl = boff[blockIdx.x] + ((threadIdx.x >> 5) ? wsum[(threadIdx.x >> 5) - 1] : 0) + x - f;
    if (i < N) {
        idx_map[i] = f ? excl : -1;
        if (f) {
            vox[excl] = (int)i;
            if (!disc) {
                chi32[excl] = (float)(e - 1.0);
                chi64[excl] = e - 1.0;
            } else {
                const int k = (int)(i % n2), j = (int)((i / n2) % n1);
                const long long x = i / ((long long)n1 * n2);
                const long long n0 = N / ((long long)n1 * n2);
                const double nb[3] = {x + 1 < n0 ? eps[i + (long long)n1 * n2] : 1.0, j + 1 < n1 ? eps[i + n2] : 1.0,
                                      k + 1 < n2 ? eps[i + 1] : 1.0};
                for (int a = 0; a < 3; ++a) {
                    const double c = 0.5 * ((e - 1.0) + (nb[a] - 1.0));
                    chi32[a * Nb + excl] = (float)c;
                    chi64[a * Nb + excl] = c;
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static const size_t SMEM_CAP = 200 * 1024;

template <typename KernelT> static int allow_smem(KernelT k) {
    VIE_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_CAP));
    return VIE_OK;
}

// Threads per CTA of a generic FFT pass.  Short transforms keep 256.  Transforms
// longer than 1024 points hold one or two lines per CTA, so the CTA is widened
// to as many threads as the register file allows for the CTAs that fit by
// shared memory (at most 512): more warps hide the stage barriers and each
// stage takes fewer sequential butterflies per thread.
// Threads of a generic line or column pass.  Double-float tiles are narrow
// (16-byte elements), so 256 threads would leave most of them idle at every
// stage: there the CTA gets one thread per butterfly of its widest stage
// ((L / largest radix) x lines, a multiple of 32, 64 to 256).
template <typename T, typename KernelT>
static int fft_threads(KernelT k, const FFTPlan& p, int nl, size_t smem) {
    const int L = p.L;
    if (std::is_same<T, dfl>::value && L <= 1024) {
        int rmax = 2;
        for (int st = 0; st < p.nst; ++st) rmax = std::max(rmax, p.R[st]);
        const int bf = (L / rmax) * nl;
        return std::max(64, std::min(256, (bf + 31) / 32 * 32));
    }
    if (L <= 1024) return 256;
    cudaFuncAttributes a;
    if (cudaFuncGetAttributes(&a, k) != cudaSuccess || a.numRegs <= 0) {
        cudaGetLastError();
        return 256;
    }
    const int ctas = std::max(1, (int)((227 * 1024) / std::max<size_t>(smem + 1024, 1)));
    int t = 65536 / (ctas * a.numRegs);
    t = std::min(512, std::min(a.maxThreadsPerBlock, t)) / 32 * 32;
    return std::max(256, t);
}

static int pow2_floor(int v) {
    int p = 1;
    while (p * 2 <= v) p *= 2;
    return p;
}

template <typename T> static size_t tw_bytes(const FFTPlan& p) {
    return sizeof(cplx<T>) * (size_t)((p.twlen + 1) & ~1);
}

// Launch shape of a generic FFT pass: lines (or columns) per CTA, whether the
// twiddle table is staged in shared memory, and the dynamic shared memory.
// The table is staged while the whole CTA stays within half of an SM's shared
// memory (two resident CTAs); longer transforms read it through L1 instead.
struct TileCfg {
    int w = 1;
    int stw = 1;
    size_t smem = 0;
    bool ok = false;
    bool joint = false;  // fused x pass: stages over the three components at once
};
static const size_t SMEM_STAGE = 100 * 1024;
template <typename T> static TileCfg finish_cfg(const FFTPlan& p, int w, size_t data) {
    TileCfg c;
    c.w = w;
    c.stw = tw_bytes<T>(p) + data <= SMEM_STAGE ? 1 : 0;
    c.smem = data + (c.stw ? tw_bytes<T>(p) : 0);
    c.ok = c.smem <= SMEM_CAP;
    return c;
}

// contiguous-line kernels: two buffers of L x lines_ld(NL)
template <typename T> static TileCfg lines_cfg(const FFTPlan& p) {
    const int budget = 48 * 1024;
    int nl = budget / (2 * (int)sizeof(cplx<T>) * std::max(p.L, 1)) - 1;
    nl = std::max(1, std::min(32, pow2_floor(std::max(1, nl))));
    return finish_cfg<T>(p, nl, 2 * sizeof(cplx<T>) * (size_t)p.L * lines_ld(nl));
}
// strided-axis kernels: two buffers of L x TW; TW is raised to one 32-byte
// sector of adjacent columns where that fits, so the strided rows coalesce
template <typename T> static TileCfg axis_cfg(const FFTPlan& p, long long inner) {
    const int budget = 64 * 1024;
    const size_t row = 2 * sizeof(cplx<T>) * (size_t)std::max(p.L, 1);
    int tw = (int)(budget / row);
    tw = std::max(1, std::min(32, pow2_floor(std::max(1, tw))));
    const int sector = 32 / (int)sizeof(cplx<T>);
    while (tw < sector && row * (size_t)(2 * tw) <= SMEM_CAP) tw *= 2;
    while (tw > 1 && tw / 2 >= inner) tw /= 2;
    return finish_cfg<T>(p, tw, row * tw);
}
// fused x pass: six buffers of L x TW (three components, three scratch: the
// joint three-component stages) when that leaves at least four columns per
// tile, else four (three components and one scratch, components in turn)
template <typename T> static TileCfg xfused_cfg(const FFTPlan& p, long long inner) {
    const int budget = 100 * 1024;
    for (int nbuf : {6, 4}) {
        int tw = (nbuf == 6 ? budget : 96 * 1024) / (nbuf * (int)sizeof(cplx<T>) * std::max(p.L, 1));
        tw = std::max(1, std::min(32, pow2_floor(std::max(1, tw))));
        while (tw > 1 && tw / 2 >= inner) tw /= 2;
        if (nbuf == 6 && tw < 4 && tw < inner) continue;
        TileCfg c = finish_cfg<T>(p, tw, nbuf * sizeof(cplx<T>) * (size_t)p.L * tw);
        c.joint = nbuf == 6;
        if (c.ok || nbuf == 4) return c;
    }
    return TileCfg();
}

// Every generic pass must fit in shared memory at FP64 (the larger element).
// The fused x pass holds three components of a column at once, so the first
// axis has the tightest limit (3200 points at FP64): long grids put their
// longest axis last.
static int check_tiles(const Operator& op) {
    if (!xfused_cfg<double>(op.ax[0].plan, (long long)op.P[1] * op.P[2]).ok)
        return fail(VIE_EINVAL, "padded length " + std::to_string(op.P[0]) +
                                    " of the first axis is too long for the fused x pass (order the axes "
                                    "shortest first)");
    if (!axis_cfg<double>(op.ax[1].plan, op.P[2]).ok || !lines_cfg<double>(op.ax[2].plan).ok)
        return fail(VIE_EINVAL, "padded FFT length does not fit in shared memory");
    return VIE_OK;
}

template <typename T> static const cplx<T>* twp(const AxisFFT& a);
template <> const c32* twp<float>(const AxisFFT& a) { return a.tw32; }
template <> const c64* twp<double>(const AxisFFT& a) { return a.tw64; }
template <> const cdf* twp<dfl>(const AxisFFT& a) { return a.twdf; }
template <typename T> static const cplx<T>* dtp(const Operator& op);
template <> const c32* dtp<float>(const Operator& op) { return op.dtab32; }
template <> const c64* dtp<double>(const Operator& op) { return op.dtab64; }
template <> const cdf* dtp<dfl>(const Operator& op) { return op.dtabdf; }

template <typename T, bool INV>
static int launch_lines(const cplx<T>* in, cplx<T>* out, long long count, int n_in, int n_out, const FFTPlan& p,
                        const cplx<T>* tw, cudaStream_t s) {
    static std::atomic<unsigned long long> init{0};  // repeated attribute calls from racing threads are harmless
    if (first_on_device(init)) VIE_TRY(allow_smem(k_lines<T, INV>));
    const TileCfg c = lines_cfg<T>(p);
    if (!c.ok) return fail(VIE_EINVAL, "FFT length " + std::to_string(p.L) + " does not fit in shared memory");
    const long long grid = (count + c.w - 1) / c.w;
    if (grid <= 0) return VIE_OK;
    const int nt = fft_threads<T>(k_lines<T, INV>, p, c.w, c.smem);
    k_lines<T, INV><<<(unsigned)grid, nt, c.smem, s>>>(in, out, count, n_in, n_out, p, tw, c.w, c.stw);
    count_launch();
    VIE_CUDA(cudaGetLastError());
    return VIE_OK;
}

template <typename T, bool INV>
static int launch_axis(const cplx<T>* in, cplx<T>* out, long long outer, int n_in, int n_out, long long inner,
                       const FFTPlan& p, const cplx<T>* tw, cudaStream_t s, int tid = TMR_OTHER) {
    const double bytes = (double)sizeof(cplx<T>) * outer * inner * (double)(n_in + n_out);
    static std::atomic<unsigned long long> init{0};  // repeated attribute calls from racing threads are harmless
    if (first_on_device(init)) VIE_TRY(allow_smem(k_axis<T, INV>));
    const TileCfg c = axis_cfg<T>(p, inner);
    if (!c.ok) return fail(VIE_EINVAL, "FFT length " + std::to_string(p.L) + " does not fit in shared memory");
    const long long grid = outer * ((inner + c.w - 1) / c.w);
    if (grid <= 0) return VIE_OK;
    const int nt = fft_threads<T>(k_axis<T, INV>, p, c.w, c.smem);
    tmr_begin(tid, s);
    k_axis<T, INV><<<(unsigned)grid, nt, c.smem, s>>>(in, out, inner, n_in, n_out, p, tw, c.w, c.stw);
    tmr_end(tid, s, bytes);
    count_launch();
    VIE_CUDA(cudaGetLastError());
    return VIE_OK;
}

int fft_lines_device(const void* in, void* out, int L, int count, int inverse, int prec, cudaStream_t s) {
    FFTPlan p;
    if (!make_plan(L, &p)) return fail(VIE_EINVAL, "FFT length must be 2,3,5,7-smooth and <= 8192");
    const int n = std::max(1, p.twlen);
    std::vector<double> t(2 * n, 0.0);
    plan_twiddles(p, t.data());
    void* dtw = nullptr;
    int st = VIE_OK;
    if (prec == VIE_PREC_FP64) {
        VIE_CUDA(cudaMalloc(&dtw, sizeof(c64) * n));
        VIE_CUDA(cudaMemcpy(dtw, t.data(), sizeof(c64) * n, cudaMemcpyHostToDevice));
        st = inverse ? launch_lines<double, true>((const c64*)in, (c64*)out, count, L, L, p, (const c64*)dtw, s)
                     : launch_lines<double, false>((const c64*)in, (c64*)out, count, L, L, p, (const c64*)dtw, s);
    } else {
        std::vector<float> tf(2 * n);
        for (int i = 0; i < 2 * n; ++i) tf[i] = (float)t[i];
        VIE_CUDA(cudaMalloc(&dtw, sizeof(c32) * n));
        VIE_CUDA(cudaMemcpy(dtw, tf.data(), sizeof(c32) * n, cudaMemcpyHostToDevice));
        st = inverse ? launch_lines<float, true>((const c32*)in, (c32*)out, count, L, L, p, (const c32*)dtw, s)
                     : launch_lines<float, false>((const c32*)in, (c32*)out, count, L, L, p, (const c32*)dtw, s);
    }
    cudaError_t e = cudaStreamSynchronize(s);
    cudaFree(dtw);
    if (st != VIE_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e, "fft_lines");
    return VIE_OK;
}

// D2 difference symbols per axis, forward-transform convention e^{-i kappa j}:
// forward difference f(c+1) - f(c) -> (e^{i kappa} - 1)/h, backward
// f(c) - f(c-1) -> (1 - e^{-i kappa})/h, kappa = 2 pi q / P.
static int build_diff_tables(Operator& op) {
    const int ds = std::max(op.P[0], std::max(op.P[1], op.P[2]));
    std::vector<c64> t(6 * (size_t)ds, c64{0, 0});
    for (int a = 0; a < 3; ++a)
        for (int q = 0; q < op.P[a]; ++q) {
            const double kap = 2.0 * M_PI * q / op.P[a];
            const double c = std::cos(kap), s = std::sin(kap);
            t[(2 * a) * (size_t)ds + q] = c64{(c - 1.0) / op.h, s / op.h};       // (e^{ik} - 1)/h
            t[(2 * a + 1) * (size_t)ds + q] = c64{(1.0 - c) / op.h, s / op.h};   // (1 - e^{-ik})/h
        }
    std::vector<c32> tf(t.size());
    for (size_t i = 0; i < t.size(); ++i) tf[i] = c32{(float)t[i].x, (float)t[i].y};
    std::vector<cdf> td(t.size());
    for (size_t i = 0; i < t.size(); ++i) td[i] = cdf{dfl(t[i].x), dfl(t[i].y)};
    if (op.dtab64) dev_free(op, op.dtab64, sizeof(c64) * 6 * (size_t)op.dstride);
    if (op.dtab32) dev_free(op, op.dtab32, sizeof(c32) * 6 * (size_t)op.dstride);
    if (op.dtabdf) dev_free(op, op.dtabdf, sizeof(cdf) * 6 * (size_t)op.dstride);
    op.dtab64 = nullptr;
    op.dtab32 = nullptr;
    op.dtabdf = nullptr;
    op.dstride = ds;
    VIE_TRY(dev_alloc(op, (void**)&op.dtab64, sizeof(c64) * t.size()));
    VIE_TRY(dev_alloc(op, (void**)&op.dtab32, sizeof(c32) * t.size()));
    VIE_TRY(dev_alloc(op, (void**)&op.dtabdf, sizeof(cdf) * t.size()));
    VIE_CUDA(cudaMemcpy(op.dtab64, t.data(), sizeof(c64) * t.size(), cudaMemcpyHostToDevice));
    VIE_CUDA(cudaMemcpy(op.dtab32, tf.data(), sizeof(c32) * t.size(), cudaMemcpyHostToDevice));
    VIE_CUDA(cudaMemcpy(op.dtabdf, td.data(), sizeof(cdf) * t.size(), cudaMemcpyHostToDevice));
    return VIE_OK;
}

int op_build_kernel(Operator& op) {
    const int P0 = op.P[0], P1 = op.P[1], P2 = op.P[2];
    const long long PP = (long long)P0 * P1 * P2;
    const double a = op.h * std::cbrt(3.0 / (4.0 * M_PI));
    const double ka = op.k0 * a;
    double kap;
    if (ka < 1e-3) kap = 1.0 - ka * ka / 10.0 + ka * ka * ka * ka / 280.0;
    else kap = 3.0 * (std::sin(ka) - ka * std::cos(ka)) / (ka * ka * ka);
    const double coef = kap * op.k0 * op.k0 * op.h * op.h * op.h;
    // self term: 2/3((1 - i ka) e^{i ka} - 1) - 1/3
    const double cr = std::cos(ka), sr = std::sin(ka);
    const double self_re = (2.0 / 3.0) * ((cr + ka * sr) - 1.0) - 1.0 / 3.0;
    const double self_im = (2.0 / 3.0) * (sr - ka * cr);
    const int nc = op.disc ? 1 : 6;  // D2: one scalar kernel
    if (op.disc) VIE_TRY(build_diff_tables(op));
    const long long HH = (long long)op.H[0] * op.H[1] * op.H[2];
    VIE_TRY(dev_alloc(op, (void**)&op.khat64, sizeof(c64) * 6 * HH));
    VIE_TRY(dev_alloc(op, (void**)&op.khat32, sizeof(c32) * 6 * HH));
    VIE_TRY(dev_alloc(op, (void**)&op.khatdf, sizeof(cdf) * 6 * HH));
    // one component at a time through a single FP64 periodic array
    c64* Kc = nullptr;
    VIE_TRY(dev_alloc(op, (void**)&Kc, sizeof(c64) * PP));
    int st = VIE_OK;
    for (int q = 0; q < nc && st == VIE_OK; ++q) {
        if (op.disc) {
            // D2: G_h(m) = kappa h^3 g(m h), G_h(0) = ((1 - i ka) e^{i ka} - 1) / k^2 on the whole periodic range
            const double g0r = ((cr + ka * sr) - 1.0) / (op.k0 * op.k0), g0i = (sr - ka * cr) / (op.k0 * op.k0);
            k_scalar_circulant<<<1184, 256, 0, op.stream>>>(Kc, P0, P1, P2, op.h, op.k0, coef / (op.k0 * op.k0), g0r,
                                                            g0i);
        } else {
            k_kernel_circulant<<<1184, 256, 0, op.stream>>>(Kc, q, op.n[0], op.n[1], op.n[2], P0, P1, P2, op.h, op.k0,
                                                            coef, self_re, self_im);
        }
        count_launch();
        if (cudaGetLastError() != cudaSuccess) st = fail(VIE_EDEVICE, "kernel build launch failed");
        // 3-D FFT, in place: z (contiguous lines), y, x
        if (st == VIE_OK)
            st = launch_lines<double, false>(Kc, Kc, (long long)P0 * P1, P2, P2, op.ax[2].plan, op.ax[2].tw64,
                                             op.stream);
        if (st == VIE_OK)
            st = launch_axis<double, false>(Kc, Kc, (long long)P0, P1, P1, P2, op.ax[1].plan, op.ax[1].tw64,
                                            op.stream);
        if (st == VIE_OK)
            st = launch_axis<double, false>(Kc, Kc, 1, P0, P0, (long long)P1 * P2, op.ax[0].plan, op.ax[0].tw64,
                                            op.stream);
        if (st == VIE_OK) {
            k_octant<<<1184, 256, 0, op.stream>>>(Kc, op.khat64 + q * HH, op.khat32 + q * HH, P0, P1, P2, op.H[0],
                                                  op.H[1], op.H[2], 1.0 / (double)PP);
            count_launch();
            if (cudaGetLastError() != cudaSuccess) st = fail(VIE_EDEVICE, "octant launch failed");
        }
    }
    if (st == VIE_OK) st = to_dfl((const double*)op.khat64, (dfl*)op.khatdf, 2LL * nc * HH, op.stream);
    cudaError_t e = cudaStreamSynchronize(op.stream);
    dev_free(op, Kc, sizeof(c64) * PP);
    if (st != VIE_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e, "kernel spectrum build");
    return VIE_OK;
}

int op_set_body_device(Operator& op, const double* eps) {
    const long long N = op.N;
    const int nb = (int)((N + SCAN_B - 1) / SCAN_B);
    int* bcount = nullptr;
    int* err = nullptr;
    long long* total = nullptr;
    VIE_CUDA(cudaMalloc(&bcount, sizeof(int) * (nb + 1)));
    VIE_CUDA(cudaMalloc(&err, sizeof(int)));
    VIE_CUDA(cudaMalloc(&total, sizeof(long long)));
    VIE_CUDA(cudaMemsetAsync(err, 0, sizeof(int), op.stream));
    k_body_count<<<nb, SCAN_B, 0, op.stream>>>(eps, N, bcount, err, op.n[1], op.n[2], op.disc);
    k_scan_blocks<<<1, 1024, 0, op.stream>>>(bcount, nb, total);
    count_launch(2);
    int herr = 0;
    long long Nb = 0;
    VIE_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, op.stream));
    VIE_CUDA(cudaMemcpyAsync(&Nb, total, sizeof(long long), cudaMemcpyDeviceToHost, op.stream));
    VIE_CUDA(cudaStreamSynchronize(op.stream));
    int st = VIE_OK;
    if (herr) st = fail(VIE_EINVAL, "eps_r must be finite and >= 1 everywhere");
    else if (Nb == 0) st = fail(VIE_EINVAL, "the body is empty (no voxel with eps_r > 1)");
    if (st == VIE_OK) {
        const long long nchi_old = op.chi_cs ? 3 * op.Nb : op.Nb;
        if (op.vox) dev_free(op, op.vox, sizeof(int) * op.Nb);
        if (op.chi32) dev_free(op, op.chi32, sizeof(float) * nchi_old);
        if (op.chi64) dev_free(op, op.chi64, sizeof(double) * nchi_old);
        if (op.chidf) dev_free(op, op.chidf, sizeof(dfl) * nchi_old);
        op.vox = nullptr;
        op.chi32 = nullptr;
        op.chi64 = nullptr;
        op.chidf = nullptr;
        if (!op.idx_map) st = dev_alloc(op, (void**)&op.idx_map, sizeof(int) * N);
        if (st == VIE_OK) st = dev_alloc(op, (void**)&op.vox, sizeof(int) * Nb);
        const long long nchi = op.disc ? 3 * Nb : Nb;
        if (st == VIE_OK) st = dev_alloc(op, (void**)&op.chi32, sizeof(float) * nchi);
        if (st == VIE_OK) st = dev_alloc(op, (void**)&op.chi64, sizeof(double) * nchi);
        if (st == VIE_OK) st = dev_alloc(op, (void**)&op.chidf, sizeof(dfl) * nchi);
        if (st == VIE_OK) {
            op.Nb = Nb;
            op.chi_cs = op.disc ? Nb : 0;
            k_body_write<<<nb, SCAN_B, 0, op.stream>>>(eps, N, bcount, op.idx_map, op.vox, op.chi32, op.chi64,
                                                       op.n[1], op.n[2], op.disc, Nb);
            count_launch();
            // fraction of z lines that hold a body voxel (the z-inverse pass reads only those)
            const long long nl = (long long)op.n[0] * op.n[1];
            cudaMemsetAsync(total, 0, sizeof(long long), op.stream);
            k_line_count<<<ceil_div(nl, 256), 256, 0, op.stream>>>(op.idx_map, nl, op.n[2], total);
            count_launch();
            long long nz = nl;
            cudaMemcpyAsync(&nz, total, sizeof(long long), cudaMemcpyDeviceToHost, op.stream);
            st = to_dfl(op.chi64, op.chidf, nchi, op.stream);
            cudaError_t e = cudaStreamSynchronize(op.stream);
            if (st == VIE_OK && e != cudaSuccess) st = cuda_fail(e, "body compaction");
            op.line_frac = nl > 0 ? (double)nz / (double)nl : 1.0;
        }
    }
    cudaFree(bcount);
    cudaFree(err);
    cudaFree(total);
    return st;
}

int op_reserve(Operator& op, int prec, int nrhs) {
    MatvecWork& W = op.work[prec];
    const size_t esz = prec ? sizeof(c64) : sizeof(c32);
    const long long perA = 3LL * op.n[0] * op.n[1] * op.P[2];
    const long long perB = 3LL * op.n[0] * op.P[1] * op.P[2];
    // The workspace of a precision takes up to 24 GB, or up to 45 % of the device memory that is free (counting
    // what it already holds) when that is more: on large grids two or more RHS per launch amortise the kernel
    // octant tile of the fused x pass.  Larger batches run in chunks of `cap` RHS.
    if (W.cap >= nrhs) return VIE_OK;
    double limit = 24e9;
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) == cudaSuccess)
        limit = std::max(limit, 0.45 * ((double)fr + (double)esz * (perA + perB) * W.cap));
    else
        cudaGetLastError();
    int cap = std::max(1, std::min(nrhs, (int)(limit / ((perA + perB) * (double)esz))));
    if (W.cap >= cap) return VIE_OK;
    if (W.A) dev_free(op, W.A, esz * perA * W.cap);
    if (W.B) dev_free(op, W.B, esz * perB * W.cap);
    W.A = W.B = nullptr;
    W.cap = 0;
    VIE_TRY(dev_alloc(op, &W.A, esz * perA * cap));
    VIE_TRY(dev_alloc(op, &W.B, esz * perB * cap));
    W.cap = cap;
    return VIE_OK;
}

int op_set_list(Operator& op, const int* host_list, int nr) {
    if (nr > op.list_cap) {
        if (op.d_list) dev_free(op, op.d_list, sizeof(int) * op.list_cap);
        op.d_list = nullptr;
        const int cap = std::max(nr, 64);
        VIE_TRY(dev_alloc(op, (void**)&op.d_list, sizeof(int) * cap));
        op.list_cap = cap;
    }
    VIE_CUDA(cudaMemcpyAsync(op.d_list, host_list, sizeof(int) * nr, cudaMemcpyHostToDevice, op.stream));
    op.h_list.assign(host_list, host_list + nr);
    return VIE_OK;
}

// T: arithmetic (float, double or double-float); TI: the vectors' scalar in
// memory (T, or double for double-float)
template <typename T, typename TI>
static int apply_t(Operator& op, const cplx<TI>* w, long long wr, cplx<TI>* y, long long yr, const int* d_list,
                   int nr) {
    constexpr bool F32 = std::is_same<T, float>::value, DF = std::is_same<T, dfl>::value;
    const int pi = F32 ? 0 : 1;  // work arrays: double and double-float elements are both 16 bytes
    VIE_TRY(op_reserve(op, pi, nr));
    MatvecWork& W = op.work[pi];
    static std::atomic<unsigned long long> init{0};  // repeated attribute calls from racing threads are harmless
    if (first_on_device(init)) {
        VIE_TRY(allow_smem(k_zfwd<T, TI>));
        VIE_TRY(allow_smem(k_zinv<T, TI>));
        VIE_TRY(allow_smem(k_xfused<T>));
    }
    const int n0 = op.n[0], n1 = op.n[1], n2 = op.n[2];
    const int P0 = op.P[0], P1 = op.P[1], P2 = op.P[2];
    cplx<T>* A = (cplx<T>*)W.A;
    cplx<T>* B = (cplx<T>*)W.B;
    const cplx<T>* kh;
    const T* chi;
    if constexpr (DF) {
        kh = (const cplx<T>*)op.khatdf;
        chi = (const T*)op.chidf;
    } else if constexpr (!F32) {
        kh = (const cplx<T>*)op.khat64;
        chi = (const T*)op.chi64;
    } else {
        kh = (const cplx<T>*)op.khat32;
        chi = (const T*)op.chi32;
    }
    const double E = sizeof(cplx<T>);
    const double EI = sizeof(cplx<TI>);
    const long long cst = comp_stride(op);  // component stride of w and y
    const double lineA = 3.0 * n0 * n1 * P2 * E;  // one slot of A
    const double lineB = 3.0 * n0 * P1 * P2 * E;  // one slot of B
    const double vec = 3.0 * op.Nb * EI;          // one compact vector
    // FP64 and double-float passes are timed under one id each (ALU-bound, kept apart from the FP32 roofline)
    auto tid = [](int id) { return F32 ? id : (DF ? (int)TMR_MVDF : (int)TMR_MV64); };
    for (int s0 = 0; s0 < nr; s0 += W.cap) {
        const int ns = std::min(W.cap, nr - s0);
        const int* list = d_list + s0;
        const bool fz = F32 && op.fft_path == 0 && fast_length(P2);
        const bool fy = F32 && op.fft_path == 0 && fast_length(P1);
        const bool fx = F32 && op.fft_path == 0 && fast_length(P0);
        // pass 1
        if (fz) {
            const long long nlines = (long long)ns * 3 * n0 * n1;
            tmr_begin(tid(TMR_ZFWD), op.stream);
            VIE_TRY(fast_zfwd((const c32*)w, wr, list, op.idx_map, (c32*)A, n0, n1, n2, cst, nlines, P2,
                              op.ax[2].roots32, op.stream, op.idx_stride));
            tmr_end(tid(TMR_ZFWD), op.stream, ns * (vec + lineA) + 4.0 * op.N);
            count_launch();
            VIE_CUDA(cudaGetLastError());
        } else {
            const FFTPlan& p = op.ax[2].plan;
            const TileCfg c = lines_cfg<T>(p);
            const long long nlines = (long long)ns * 3 * n0 * n1;
            const int nt = fft_threads<T>(k_zfwd<T, TI>, p, c.w, c.smem);
            tmr_begin(tid(TMR_ZFWD), op.stream);
            k_zfwd<T, TI><<<(unsigned)((nlines + c.w - 1) / c.w), nt, c.smem, op.stream>>>(
                w, wr, list, op.idx_map, A, n0, n1, n2, cst, nlines, p, twp<T>(op.ax[2]), c.w, c.stw,
                op.idx_stride);
            tmr_end(tid(TMR_ZFWD), op.stream, ns * (vec + lineA) + 4.0 * op.N);
            count_launch();
            VIE_CUDA(cudaGetLastError());
        }
        // pass 2
        if (fy) {
            tmr_begin(tid(TMR_YFWD), op.stream);
            VIE_TRY(fast_axis((const c32*)A, (c32*)B, (long long)ns * 3 * n0, n1, P1, P2, P1, op.ax[1].roots32, false,
                              op.stream));
            tmr_end(tid(TMR_YFWD), op.stream, (double)ns * (lineA + lineB));
            count_launch();
            VIE_CUDA(cudaGetLastError());
        } else {
            VIE_TRY((launch_axis<T, false>(A, B, (long long)ns * 3 * n0, n1, P1, P2, op.ax[1].plan, twp<T>(op.ax[1]),
                                           op.stream, tid(TMR_YFWD))));
        }
        // pass 3
        if (fx) {
            tmr_begin(tid(TMR_XFUSED), op.stream);
            D2Spec d2;
            d2.dtab = op.dtab32;
            d2.dstride = op.dstride;
            d2.k2 = (float)(op.k0 * op.k0);
            VIE_TRY(fast_xfused((c32*)B, n0, (long long)P1 * P2, P0, P1, P2, (const c32*)kh, op.H, op.ax[0].roots32, ns,
                                op.stream, op.disc ? &d2 : nullptr));
            tmr_end(tid(TMR_XFUSED), op.stream, 2.0 * ns * lineB + 6.0 * op.H[0] * op.H[1] * op.H[2] * E);
            count_launch();
            VIE_CUDA(cudaGetLastError());
        } else {
            const FFTPlan& p = op.ax[0].plan;
            const long long inner = (long long)P1 * P2;
            const TileCfg c = xfused_cfg<T>(p, inner);
            const long long grid = (long long)ns * ((inner + c.w - 1) / c.w);
            tmr_begin(tid(TMR_XFUSED), op.stream);
            k_xfused<T><<<(unsigned)grid, XG<T>::NT, c.smem, op.stream>>>(
                B, n0, inner, P0, P1, P2, kh, op.H[0], op.H[1], op.H[2], p, twp<T>(op.ax[0]), c.w,
                op.disc ? dtp<T>(op) : nullptr, op.dstride, (T)(op.k0 * op.k0), c.stw, c.joint ? 1 : 0);
            tmr_end(tid(TMR_XFUSED), op.stream, 2.0 * ns * lineB + 6.0 * op.H[0] * op.H[1] * op.H[2] * E);
            count_launch();
            VIE_CUDA(cudaGetLastError());
        }
        // pass 4
        if (fy) {
            tmr_begin(tid(TMR_YINV), op.stream);
            VIE_TRY(fast_axis((const c32*)B, (c32*)A, (long long)ns * 3 * n0, P1, n1, P2, P1, op.ax[1].roots32, true,
                              op.stream));
            tmr_end(tid(TMR_YINV), op.stream, (double)ns * (lineA + lineB));
            count_launch();
            VIE_CUDA(cudaGetLastError());
        } else {
            VIE_TRY((launch_axis<T, true>(B, A, (long long)ns * 3 * n0, P1, n1, P2, op.ax[1].plan, twp<T>(op.ax[1]),
                                          op.stream, tid(TMR_YINV))));
        }
        // pass 5
        if (fz) {
            const long long nlines = (long long)ns * 3 * n0 * n1;
            tmr_begin(tid(TMR_ZINV), op.stream);
            VIE_TRY(fast_zinv((const c32*)A, (const c32*)w, wr, (c32*)y, yr, list, op.idx_map, (const float*)chi, n0, n1,
                              n2, cst, nlines, P2, op.ax[2].roots32, op.stream, op.chi_cs, op.idx_stride));
            tmr_end(tid(TMR_ZINV), op.stream, ns * (lineA * op.line_frac + 2.0 * vec) + op.Nb * sizeof(T) + 4.0 * op.N);
            count_launch();
            VIE_CUDA(cudaGetLastError());
        } else {
            const FFTPlan& p = op.ax[2].plan;
            const TileCfg c = lines_cfg<T>(p);
            const long long nlines = (long long)ns * 3 * n0 * n1;
            const int nt = fft_threads<T>(k_zinv<T, TI>, p, c.w, c.smem);
            tmr_begin(tid(TMR_ZINV), op.stream);
            k_zinv<T, TI><<<(unsigned)((nlines + c.w - 1) / c.w), nt, c.smem, op.stream>>>(
                A, w, wr, y, yr, list, op.idx_map, chi, n0, n1, n2, cst, nlines, p, twp<T>(op.ax[2]), c.w,
                op.chi_cs, c.stw, op.idx_stride);
            tmr_end(tid(TMR_ZINV), op.stream, ns * (lineA * op.line_frac + 2.0 * vec) + op.Nb * sizeof(T) + 4.0 * op.N);
            count_launch();
            VIE_CUDA(cudaGetLastError());
        }
    }
    return VIE_OK;
}

int op_apply(Operator& op, int prec, const void* w, long long wr, void* y, long long yr, const int* d_list, int nr) {
    if (nr <= 0) return VIE_OK;
    if (op.batch) {
        if (d_list != op.d_list) return fail(VIE_EINVAL, "a batch operator takes the list set by op_set_list");
        return batch_apply(op, prec, w, wr, y, yr, nr);
    }
    if (prec == VIE_PREC_FP64) return apply_t<double, double>(op, (const c64*)w, wr, (c64*)y, yr, d_list, nr);
    if (prec == VIE_PREC_F32X2) return apply_t<dfl, double>(op, (const c64*)w, wr, (c64*)y, yr, d_list, nr);
    return apply_t<float, float>(op, (const c32*)w, wr, (c32*)y, yr, d_list, nr);
}

int op_replan(Operator& op, const int P[3]) {
    VIE_CUDA(cudaStreamSynchronize(op.stream));
    for (int a = 0; a < 3; ++a) {
        AxisFFT& x = op.ax[a];
        const int n = std::max(1, x.plan.twlen);
        dev_free(op, x.tw64, sizeof(c64) * n);
        dev_free(op, x.tw32, sizeof(c32) * n);
        dev_free(op, x.roots32, sizeof(c32) * 2 * x.plan.L);
        dev_free(op, x.twdf, sizeof(cdf) * n);
        x.tw64 = nullptr;
        x.tw32 = nullptr;
        x.roots32 = nullptr;
        x.twdf = nullptr;
    }
    const long long HH = (long long)op.H[0] * op.H[1] * op.H[2];
    dev_free(op, op.khat64, sizeof(c64) * 6 * HH);
    dev_free(op, op.khat32, sizeof(c32) * 6 * HH);
    dev_free(op, op.khatdf, sizeof(cdf) * 6 * HH);
    op.khat64 = nullptr;
    op.khat32 = nullptr;
    op.khatdf = nullptr;
    for (int p = 0; p < 2; ++p) {
        MatvecWork& W = op.work[p];
        const size_t esz = p ? sizeof(c64) : sizeof(c32);
        dev_free(op, W.A, esz * 3LL * op.n[0] * op.n[1] * op.P[2] * W.cap);
        dev_free(op, W.B, esz * 3LL * op.n[0] * op.P[1] * op.P[2] * W.cap);
        W = MatvecWork();
    }
    for (int a = 0; a < 3; ++a) op.P_fixed[a] = P[a];
    VIE_TRY(op_init_axes(op));
    return op_build_kernel(op);
}

void op_free(Operator& op) {
    cudaFree(op.ff_ws);
    op.ff_ws = nullptr;
    op.ff_ws_bytes = 0;
    for (int a = 0; a < 3; ++a) {
        cudaFree(op.ax[a].tw32);
        cudaFree(op.ax[a].tw64);
        cudaFree(op.ax[a].roots32);
        cudaFree(op.ax[a].twdf);
        op.ax[a].tw32 = nullptr;
        op.ax[a].tw64 = nullptr;
        op.ax[a].roots32 = nullptr;
        op.ax[a].twdf = nullptr;
    }
    cudaFree(op.khat32);
    cudaFree(op.khat64);
    cudaFree(op.khatdf);
    cudaFree(op.dtab32);
    cudaFree(op.dtab64);
    cudaFree(op.dtabdf);
    op.dtab32 = nullptr;
    op.dtab64 = nullptr;
    op.dtabdf = nullptr;
    op.khatdf = nullptr;
    cudaFree(op.idx_map);
    cudaFree(op.vox);
    cudaFree(op.chi32);
    cudaFree(op.chi64);
    cudaFree(op.chidf);
    op.chidf = nullptr;
    for (int p = 0; p < 2; ++p) {
        cudaFree(op.work[p].A);
        cudaFree(op.work[p].B);
        op.work[p] = MatvecWork();
    }
    cudaFree(op.d_list);
    op.khat32 = nullptr;
    op.khat64 = nullptr;
    op.idx_map = nullptr;
    op.vox = nullptr;
    op.chi32 = nullptr;
    op.chi64 = nullptr;
    op.d_list = nullptr;
    op.bytes = 0;
}

}  // namespace vie
