// FP32 fast path of the operator passes for power-of-two padded lengths
// (16 .. 512): register-resident four-step FFTs (fft4.cuh) with a single
// shared-memory exchange per transform, loads and stores straight between
// registers and global memory.  Same data layouts and semantics as the
// generic passes in matvec.cu, which remain the path for other lengths and
// for FP64.
//
// Twiddles w_L^{k1 n2} come from two tables of L entries staged in shared
// memory, TA[k1][n2] for the forward step (threads indexed by n2) and
// TB[n2][k1] for the inverse step (threads indexed by k1), so that lanes of a
// warp read consecutive words.
#include "fft4.cuh"
#include "vie_internal.cuh"

namespace vie {

bool fast_length(int L) { return L == 16 || L == 32 || L == 64 || L == 128 || L == 256 || L == 512; }

void fast_factors(int L, int* R1, int* R2) {
    switch (L) {
        case 16: *R1 = Fac<16>::R1; *R2 = Fac<16>::R2; break;
        case 32: *R1 = Fac<32>::R1; *R2 = Fac<32>::R2; break;
        case 64: *R1 = Fac<64>::R1; *R2 = Fac<64>::R2; break;
        case 128: *R1 = Fac<128>::R1; *R2 = Fac<128>::R2; break;
        case 256: *R1 = Fac<256>::R1; *R2 = Fac<256>::R2; break;
        default: *R1 = Fac<512>::R1; *R2 = Fac<512>::R2; break;
    }
}

namespace {

constexpr int AX_TW = 16;  // columns per CTA, strided-axis passes
constexpr int XF_TW = 8;   // columns per CTA, fused x pass (3 components)

__device__ __forceinline__ c32 z32() { return c32{0.f, 0.f}; }

__device__ __forceinline__ void stage_table(c32* dst, const c32* __restrict__ g, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = g[i];
}

template <bool INV> __device__ __forceinline__ c32 tw(const c32* t, int i) {
    c32 w = t[i];
    if (INV) w.y = -w.y;
    return w;
}

// ---- strided axis: in [outer][n_in][inner] -> out [outer][n_out][inner] ------
// HALF: the forward input (n_in) or the inverse output (n_out) spans at most
// L/2 rows, so the radix-R1 step next to it is a half DFT.
template <int L, bool INV, bool HALF>
__global__ void __launch_bounds__(Fac<L>::R2 * AX_TW) k_axis_r(const c32* __restrict__ in, c32* __restrict__ out,
                                                               long long inner, int n_in, int n_out,
                                                               const c32* __restrict__ tw4) {
    constexpr int R1 = Fac<L>::R1, R2 = Fac<L>::R2, TW = AX_TW, NT = R2 * TW;
    constexpr int SR = R2 * TW;  // row stride of the R1 x R2 x TW exchange
    extern __shared__ __align__(16) unsigned char smraw[];
    c32* T = reinterpret_cast<c32*>(smraw);  // TA (forward) or TB (inverse)
    c32* S = T + L;
    stage_table(T, tw4 + (INV ? L : 0), L);
    const long long ntile = (inner + TW - 1) / TW;
    const long long o = blockIdx.x / ntile;
    const long long i0 = (blockIdx.x - o * ntile) * TW;
    const int t = threadIdx.x % TW, n2 = threadIdx.x / TW;
    __syncthreads();
    if (!INV) {
        c32 a[R1];
        const bool ok = i0 + t < inner;
#pragma unroll
        for (int n1 = 0; n1 < (HALF ? R1 / 2 : R1); ++n1) {
            const int p = n1 * R2 + n2;
            a[n1] = (ok && p < n_in) ? in[(o * n_in + p) * inner + i0 + t] : z32();
        }
        if (HALF) dftp2_half_in<float, R1, false>(a);
        else dftp2<float, R1, false>(a);
#pragma unroll
        for (int k1 = 1; k1 < R1; ++k1) a[k1] = a[k1] * tw<false>(T, k1 * R2 + n2);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) S[k1 * SR + n2 * TW + t] = a[k1];
        __syncthreads();
        for (int it = threadIdx.x; it < R1 * TW; it += NT) {
            const int k1 = it / TW, tt = it % TW;
            c32 b[R2];
#pragma unroll
            for (int q = 0; q < R2; ++q) b[q] = S[k1 * SR + q * TW + tt];
            dftp2<float, R2, false>(b);
            if (i0 + tt < inner) {
#pragma unroll
                for (int k2 = 0; k2 < R2; ++k2) {
                    const int p = k1 + R1 * k2;
                    if (p < n_out) out[(o * n_out + p) * inner + i0 + tt] = b[k2];
                }
            }
        }
    } else {
        for (int it = threadIdx.x; it < R1 * TW; it += NT) {
            const int k1 = it / TW, tt = it % TW;
            const bool ok = i0 + tt < inner;
            c32 b[R2];
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) {
                const int p = k1 + R1 * k2;
                b[k2] = (ok && p < n_in) ? in[(o * n_in + p) * inner + i0 + tt] : z32();
            }
            dftp2<float, R2, true>(b);
#pragma unroll
            for (int q = 0; q < R2; ++q) S[k1 * SR + q * TW + tt] = b[q] * tw<true>(T, q * R1 + k1);
        }
        __syncthreads();
        c32 a[R1];
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) a[k1] = S[k1 * SR + n2 * TW + t];
        if (HALF) dftp2_half_out<float, R1, true>(a);
        else dftp2<float, R1, true>(a);
        if (i0 + t < inner) {
#pragma unroll
            for (int n1 = 0; n1 < (HALF ? R1 / 2 : R1); ++n1) {
                const int p = n1 * R2 + n2;
                if (p < n_out) out[(o * n_out + p) * inner + i0 + t] = a[n1];
            }
        }
    }
}

// ---- fused x pass: forward FFT x, 3x3 spectral multiply, inverse FFT x ------
// One CTA per tile of XF_TW (y, z)-frequency columns; it stages the kernel
// octant rows of its columns in shared memory once (x-folded, y/z signs
// applied) and loops over all RHS slots.  The x support of the data is
// n0 <= L/2 rows (zero padding) and only those rows are written back (crop),
// so the first forward and the last inverse radix-R1 steps take the half
// DFTs.  For L <= 256 the global loads of the next slot are issued before the
// arithmetic of the current one (register double buffering), so their
// latency overlaps the FFTs.
template <int L> struct XF {
    static constexpr int R1 = Fac<L>::R1, R2 = Fac<L>::R2, TW = XF_TW, NT = R2 * TW;
    static constexpr int SR = R2 * TW + 8;  // padded exchange row (conflict-free half-warps)
    static constexpr int SC = R1 * SR;      // one component
    static constexpr int HX = L / 2 + 1;    // folded x rows of the kernel tile
    static constexpr int HR = R1 / 2;       // non-zero input rows per thread
    static constexpr bool PF = L <= 256;    // prefetch the next slot
    static constexpr size_t smem = sizeof(c32) * (2 * L + 6 * (size_t)HX * TW + 3 * (size_t)SC);
    // D2: the x difference symbols (2 L) and the column ones (4 TW) follow
    static constexpr size_t smem_d2 = smem + sizeof(c32) * (2 * L + 4 * TW);
};

// D2 (rooftop discretisation): the kernel tile holds the scalar G only and the
// multiply is U_a = G (k^2 W_a + d+_a (d-_x W_x + d-_y W_y + d-_z W_z)).
template <int L, bool D2>
__global__ void __launch_bounds__(XF<L>::NT) k_xfused_r(c32* __restrict__ B, int n0, long long inner, int P1,
                                                       int P2, const c32* __restrict__ khat, int H0, int H1, int H2,
                                                       const c32* __restrict__ tw4, int nslots,
                                                       const c32* __restrict__ dtab, int dstride, float ksq) {
    constexpr int R1 = XF<L>::R1, R2 = XF<L>::R2, TW = XF<L>::TW, NT = XF<L>::NT;
    constexpr int SR = XF<L>::SR, SC = XF<L>::SC, HX = XF<L>::HX, HR = XF<L>::HR;
    constexpr bool PF = XF<L>::PF;
    extern __shared__ __align__(16) unsigned char smraw[];
    c32* TA = reinterpret_cast<c32*>(smraw);
    c32* TB = TA + L;
    c32* Kt = TB + L;          // [6][HX][TW]
    c32* S = Kt + 6 * HX * TW;  // [3][R1][SR]
    c32* DX = S + 3 * SC;       // D2: [2][L] x symbols (+, -)
    c32* DC = DX + 2 * L;       // D2: [4][TW] column symbols y+, y-, z+, z-
    stage_table(TA, tw4, 2 * L);
    if (D2) {
        for (int q = threadIdx.x; q < L; q += NT) {
            DX[q] = dtab[q];
            DX[L + q] = dtab[dstride + q];
        }
        if (threadIdx.x < TW) {
            const long long ii = (long long)blockIdx.x * TW + threadIdx.x;
            c32 v[4] = {z32(), z32(), z32(), z32()};
            if (ii < inner) {
                const int ky = (int)(ii / P2), kz = (int)(ii - (ii / P2) * P2);
                v[0] = dtab[2 * dstride + ky];
                v[1] = dtab[3 * dstride + ky];
                v[2] = dtab[4 * dstride + kz];
                v[3] = dtab[5 * dstride + kz];
            }
            for (int q = 0; q < 4; ++q) DC[q * TW + threadIdx.x] = v[q];
        }
    }
    const long long i0 = (long long)blockIdx.x * TW;
    const long long HH = (long long)H0 * H1 * H2;
    // kernel tile: rows fx = 0..L/2 of the 6 components for this CTA's columns.
    // Per column: the folded (y, z) offset in the octant and the y/z parities
    // (xy odd in y, xz odd in z, yz odd in y and z), then batched loads.
    __shared__ long long coff[TW];
    __shared__ unsigned char cneg[TW];  // bit q set: negate component q
    if (threadIdx.x < TW) {
        const long long ii = i0 + threadIdx.x;
        long long off = -1;
        unsigned char ng = 0;
        if (ii < inner) {
            const int ky = (int)(ii / P2), kz = (int)(ii - (ii / P2) * P2);
            const bool fly = 2 * ky > P1, flz = 2 * kz > P2;
            off = (long long)(fly ? P1 - ky : ky) * H2 + (flz ? P2 - kz : kz);
            ng = D2 ? 0 : (unsigned char)((fly ? 2 : 0) | (flz ? 4 : 0) | ((fly ^ flz) ? 16 : 0));
        }
        coff[threadIdx.x] = off;
        cneg[threadIdx.x] = ng;
    }
    __syncthreads();
    {
        constexpr int NE = (D2 ? 1 : 6) * HX * TW, U = 8;
        const long long rowst = (long long)H1 * H2;
        for (int e0 = 0; e0 < NE; e0 += U * NT) {
            c32 v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int e = e0 + u * NT + threadIdx.x;
                v[u] = z32();
                if (e < NE) {
                    const int tt = e % TW, fx = (e / TW) % HX, q = e / (TW * HX);
                    const long long off = coff[tt];
                    if (off >= 0) v[u] = khat[q * HH + fx * rowst + off];
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int e = e0 + u * NT + threadIdx.x;
                if (e < NE) {
                    const int tt = e % TW, q = e / (TW * HX);
                    c32 w = v[u];
                    if ((cneg[tt] >> q) & 1) w = c32{-w.x, -w.y};
                    Kt[e] = w;
                }
            }
        }
    }
    const int t = threadIdx.x % TW, n2 = threadIdx.x / TW;
    const bool okt = i0 + t < inner;
    const long long cs = (long long)n0 * inner;        // component stride
    const long long rs = (long long)R2 * inner;        // stride between a thread's rows
    c32* const col = B + (long long)n2 * inner + i0 + t;  // row n2 of this thread's column, slot 0, component 0
    c32 pre[3][HR];
    auto load = [&](int slot) {
        const c32* q = col + (long long)slot * 3 * cs;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int n1 = 0; n1 < HR; ++n1)
                pre[c][n1] = (okt && n1 * R2 + n2 < n0) ? q[c * cs + n1 * rs] : z32();
    };
    if (PF) load(0);
    __syncthreads();
    for (int slot = 0; slot < nslots; ++slot) {
        c32* base = B + (long long)slot * 3 * cs;
        c32 a[3][R1];
        if (!PF) load(slot);
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int n1 = 0; n1 < HR; ++n1) a[c][n1] = pre[c][n1];
        if (PF && slot + 1 < nslots) load(slot + 1);
#pragma unroll
        for (int c = 0; c < 3; ++c) dftp2_half_in<float, R1, false>(a[c]);
#pragma unroll
        for (int k1 = 1; k1 < R1; ++k1) {
            const c32 w = tw<false>(TA, k1 * R2 + n2);
#pragma unroll
            for (int c = 0; c < 3; ++c) a[c][k1] = a[c][k1] * w;
        }
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int k1 = 0; k1 < R1; ++k1) S[c * SC + k1 * SR + n2 * TW + t] = a[c][k1];
        __syncthreads();
        for (int it = threadIdx.x; it < R1 * TW; it += NT) {
            const int k1 = it / TW, tt = it % TW;
            c32 bx[R2], by[R2], bz[R2];
#pragma unroll
            for (int q = 0; q < R2; ++q) {
                bx[q] = S[0 * SC + k1 * SR + q * TW + tt];
                by[q] = S[1 * SC + k1 * SR + q * TW + tt];
                bz[q] = S[2 * SC + k1 * SR + q * TW + tt];
            }
            dftp2<float, R2, false>(bx);
            dftp2<float, R2, false>(by);
            dftp2<float, R2, false>(bz);
            // kx = k1 + R1 k2 folds to L - kx above L/2: for k2 < R2/2 never, for
            // k2 > R2/2 always, for k2 = R2/2 unless k1 = 0
            const c32* kp = Kt + k1 * TW + tt;        // row kx
            const c32* km = Kt + (L - k1) * TW + tt;  // row L - kx (plus R1 k2 rows)
            if (D2) {
                const c32 dyp = DC[tt], dym = DC[TW + tt], dzp = DC[2 * TW + tt], dzm = DC[3 * TW + tt];
#pragma unroll
                for (int k2 = 0; k2 < R2; ++k2) {
                    const bool flx = 2 * k2 > R2 || (2 * k2 == R2 && k1 > 0);
                    const c32 g = *(flx ? km - R1 * k2 * TW : kp + R1 * k2 * TW);
                    const int kx = k1 + R1 * k2;
                    const c32 dxp = DX[kx], dxm = DX[L + kx];
                    const c32 a0 = bx[k2], b0 = by[k2], c0 = bz[k2];
                    const c32 sdiv = dxm * a0 + dym * b0 + dzm * c0;
                    bx[k2] = g * (ksq * a0 + dxp * sdiv);
                    by[k2] = g * (ksq * b0 + dyp * sdiv);
                    bz[k2] = g * (ksq * c0 + dzp * sdiv);
                }
            } else
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) {
                const bool flx = 2 * k2 > R2 || (2 * k2 == R2 && k1 > 0);
                const c32* kt = flx ? km - R1 * k2 * TW : kp + R1 * k2 * TW;
                c32 kxx = kt[0], kxy = kt[HX * TW], kxz = kt[2 * HX * TW];
                const c32 kyy = kt[3 * HX * TW], kyz = kt[4 * HX * TW], kzz = kt[5 * HX * TW];
                if (flx) {
                    kxy = c32{-kxy.x, -kxy.y};
                    kxz = c32{-kxz.x, -kxz.y};
                }
                const c32 a0 = bx[k2], b0 = by[k2], c0 = bz[k2];
                bx[k2] = kxx * a0 + kxy * b0 + kxz * c0;
                by[k2] = kxy * a0 + kyy * b0 + kyz * c0;
                bz[k2] = kxz * a0 + kyz * b0 + kzz * c0;
            }
            dftp2<float, R2, true>(bx);
            dftp2<float, R2, true>(by);
            dftp2<float, R2, true>(bz);
#pragma unroll
            for (int q = 0; q < R2; ++q) {
                const c32 w = tw<true>(TB, q * R1 + k1);
                S[0 * SC + k1 * SR + q * TW + tt] = bx[q] * w;
                S[1 * SC + k1 * SR + q * TW + tt] = by[q] * w;
                S[2 * SC + k1 * SR + q * TW + tt] = bz[q] * w;
            }
        }
        __syncthreads();
        if (okt) {
#pragma unroll 1
            for (int c = 0; c < 3; ++c) {
                c32 o[R1];
#pragma unroll
                for (int k1 = 0; k1 < R1; ++k1) o[k1] = S[c * SC + k1 * SR + n2 * TW + t];
                dftp2_half_out<float, R1, true>(o);
                c32* q = base + c * cs + (long long)n2 * inner + i0 + t;
#pragma unroll
                for (int n1 = 0; n1 < HR; ++n1)
                    if (n1 * R2 + n2 < n0) q[n1 * rs] = o[n1];
            }
        }
        __syncthreads();
    }
}

// ---- z passes on contiguous lines (gather from / scatter to the body list) ---
constexpr int Z_THREADS = 256;

template <int L>
__global__ void __launch_bounds__(Z_THREADS) k_zfwd_r(const c32* __restrict__ w, long long w_rstride,
                                                      const int* __restrict__ list, const int* __restrict__ idx_map,
                                                      c32* __restrict__ A, int n0, int n1, int n2, long long Nb,
                                                      long long nlines, const c32* __restrict__ tw4,
                                                      long long idx_stride) {
    constexpr int R1 = Fac<L>::R1, R2 = Fac<L>::R2;
    constexpr int NL = Z_THREADS / R2;
    constexpr int RS = R2 + 1;  // padded row
    extern __shared__ __align__(16) unsigned char smraw[];
    c32* TA = reinterpret_cast<c32*>(smraw);
    c32* S = TA + L;
    stage_table(TA, tw4, L);
    const long long line0 = (long long)blockIdx.x * NL;
    const long long plane = (long long)n0 * n1;
    const int q2 = threadIdx.x % R2, l = threadIdx.x / R2;
    const long long line = line0 + l;
    c32 a[R1];
    bool any = false;
    if (line < nlines) {
        const long long sc = line / plane;
        const long long xy = line - sc * plane;
        const int slot = (int)(sc / 3), c = (int)(sc - (sc / 3) * 3);
        const c32* wr = w + (long long)list[slot] * w_rstride + c * Nb;
        const int* im = idx_map + (long long)list[slot] * idx_stride + xy * n2;
#pragma unroll
        for (int n1i = 0; n1i < R1 / 2; ++n1i) {  // n2 <= L/2: the upper half is padding
            const int z = n1i * R2 + q2;
            c32 v = z32();
            if (z < n2) {
                const int vi = im[z];
                if (vi >= 0) {
                    v = wr[vi];
                    any = true;
                }
            }
            a[n1i] = v;
        }
    } else {
#pragma unroll
        for (int n1i = 0; n1i < R1 / 2; ++n1i) a[n1i] = z32();
    }
    if (!__syncthreads_or(any)) {
        // no body voxel on this CTA's lines: their spectra are zero
        for (long long i = threadIdx.x; i < (long long)NL * L; i += Z_THREADS)
            if (line0 + i / L < nlines) A[line0 * L + i] = z32();
        return;
    }
    dftp2_half_in<float, R1, false>(a);
#pragma unroll
    for (int k1 = 1; k1 < R1; ++k1) a[k1] = a[k1] * tw<false>(TA, k1 * R2 + q2);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) S[(l * R1 + k1) * RS + q2] = a[k1];
    __syncthreads();
    for (int it = threadIdx.x; it < NL * R1; it += Z_THREADS) {
        const int k1 = it % R1, ll = it / R1;
        c32 b[R2];
#pragma unroll
        for (int q = 0; q < R2; ++q) b[q] = S[(ll * R1 + k1) * RS + q];
        dftp2<float, R2, false>(b);
        const long long ln = line0 + ll;
        if (ln < nlines) {
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) A[ln * L + k1 + R1 * k2] = b[k2];
        }
    }
}

template <int L>
__global__ void __launch_bounds__(Z_THREADS) k_zinv_r(const c32* __restrict__ A, const c32* __restrict__ w,
                                                      long long w_rstride, c32* __restrict__ y, long long y_rstride,
                                                      const int* __restrict__ list, const int* __restrict__ idx_map,
                                                      const float* __restrict__ chi, int n0, int n1, int n2,
                                                      long long Nb, long long nlines, const c32* __restrict__ tw4,
                                                      long long chi_cs, long long idx_stride) {
    constexpr int R1 = Fac<L>::R1, R2 = Fac<L>::R2;
    constexpr int NL = Z_THREADS / R2;
    constexpr int RS = R2 + 1;
    extern __shared__ __align__(16) unsigned char smraw[];
    c32* TB = reinterpret_cast<c32*>(smraw);
    c32* S = TB + L;
    const long long line0 = (long long)blockIdx.x * NL;
    // this thread's voxel indices of the scatter (read first: a CTA whose lines
    // hold no body voxel has nothing to write and skips its transforms)
    const int q2 = threadIdx.x % R2, l = threadIdx.x / R2;
    const long long line = line0 + l;
    const long long plane = (long long)n0 * n1;
    const long long sc = line / plane;
    const long long xy = line - sc * plane;
    const int slot = (int)(sc / 3), c = (int)(sc - (sc / 3) * 3);
    const long long rr = line < nlines ? list[slot] : 0;
    int vis[R1 / 2];
    bool any = false;
    {
        const int* im = idx_map + rr * idx_stride + xy * n2;
#pragma unroll
        for (int n1i = 0; n1i < R1 / 2; ++n1i) {
            const int z = n1i * R2 + q2;
            vis[n1i] = (line < nlines && z < n2) ? im[z] : -1;
            any |= vis[n1i] >= 0;
        }
    }
    stage_table(TB, tw4 + L, L);
    if (!__syncthreads_or(any)) return;
    for (int it = threadIdx.x; it < NL * R1; it += Z_THREADS) {
        const int k1 = it % R1, ll = it / R1;
        const long long ln = line0 + ll;
        c32 b[R2];
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) b[k2] = ln < nlines ? A[ln * L + k1 + R1 * k2] : z32();
        dftp2<float, R2, true>(b);
#pragma unroll
        for (int q = 0; q < R2; ++q) S[(ll * R1 + k1) * RS + q] = b[q] * tw<true>(TB, q * R1 + k1);
    }
    __syncthreads();
    if (line >= nlines) return;
    c32 a[R1];
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) a[k1] = S[(l * R1 + k1) * RS + q2];
    dftp2_half_out<float, R1, true>(a);  // only z < n2 <= L/2 is kept
    const c32* wr = w + rr * w_rstride + c * Nb;
    c32* yr = y + rr * y_rstride + c * Nb;
#pragma unroll
    for (int n1i = 0; n1i < R1 / 2; ++n1i) {
        const int z = n1i * R2 + q2;
        if (z < n2) {
            const int vi = vis[n1i];
            if (vi >= 0) {
                const c32 u = a[n1i];
                const c32 wv = wr[vi];
                const float ch = chi[c * chi_cs + vi];
                yr[vi] = c32{wv.x - ch * u.x, wv.y - ch * u.y};
            }
        }
    }
}

// ---- multi-body passes: one launch over slots of different bodies ----------
// A slot is one RHS of one body; all slots of a launch share the padded
// sizes (the template lengths) but each has its own grid n, voxel map,
// contrast, kernel spectrum, vectors and work areas (MSlot, vie_internal.cuh).
// Slots of a body are consecutive.  Each CTA of the z and y passes belongs
// to one slot (found by binary search over the slots' first CTA); the fused
// x pass walks the slots of its column tile and restages the kernel tile
// when the body changes.
__device__ __forceinline__ int slot_of(const MSlot* __restrict__ sl, int ns, long long blk, int which) {
    int lo = 0, hi = ns - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const long long b0 = which ? sl[mid].yb0 : sl[mid].zb0;
        if (b0 <= blk) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int L>
__global__ void __launch_bounds__(Z_THREADS) k_zfwd_m(const MSlot* __restrict__ sl, int ns, c32* __restrict__ A,
                                                      long long cst, const c32* __restrict__ tw4) {
    constexpr int R1 = Fac<L>::R1, R2 = Fac<L>::R2;
    constexpr int NL = Z_THREADS / R2;
    constexpr int RS = R2 + 1;
    extern __shared__ __align__(16) unsigned char smraw[];
    c32* TA = reinterpret_cast<c32*>(smraw);
    c32* S = TA + L;
    stage_table(TA, tw4, L);
    const int si = slot_of(sl, ns, blockIdx.x, 0);
    const MSlot d = sl[si];
    const long long plane = (long long)d.n0 * d.n1;
    const long long nlines = 3 * plane;
    const long long line0 = (long long)(blockIdx.x - d.zb0) * NL;
    const int q2 = threadIdx.x % R2, l = threadIdx.x / R2;
    const long long line = line0 + l;
    c32 a[R1];
    if (line < nlines) {
        const int c = (int)(line / plane);
        const long long xy = line - c * plane;
        const c32* wr = d.w + c * cst;
        const int* im = d.idx + xy * d.n2;
#pragma unroll
        for (int n1i = 0; n1i < R1 / 2; ++n1i) {
            const int z = n1i * R2 + q2;
            c32 v = z32();
            if (z < d.n2) {
                const int vi = im[z];
                if (vi >= 0) v = wr[vi];
            }
            a[n1i] = v;
        }
    } else {
#pragma unroll
        for (int n1i = 0; n1i < R1 / 2; ++n1i) a[n1i] = z32();
    }
    __syncthreads();
    dftp2_half_in<float, R1, false>(a);
#pragma unroll
    for (int k1 = 1; k1 < R1; ++k1) a[k1] = a[k1] * tw<false>(TA, k1 * R2 + q2);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) S[(l * R1 + k1) * RS + q2] = a[k1];
    __syncthreads();
    c32* Ad = A + d.a_off;
    for (int it = threadIdx.x; it < NL * R1; it += Z_THREADS) {
        const int k1 = it % R1, ll = it / R1;
        c32 b[R2];
#pragma unroll
        for (int q = 0; q < R2; ++q) b[q] = S[(ll * R1 + k1) * RS + q];
        dftp2<float, R2, false>(b);
        const long long ln = line0 + ll;
        if (ln < nlines) {
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) Ad[ln * L + k1 + R1 * k2] = b[k2];
        }
    }
}

template <int L>
__global__ void __launch_bounds__(Z_THREADS) k_zinv_m(const MSlot* __restrict__ sl, int ns, const c32* __restrict__ A,
                                                      long long cst, const c32* __restrict__ tw4) {
    constexpr int R1 = Fac<L>::R1, R2 = Fac<L>::R2;
    constexpr int NL = Z_THREADS / R2;
    constexpr int RS = R2 + 1;
    extern __shared__ __align__(16) unsigned char smraw[];
    c32* TB = reinterpret_cast<c32*>(smraw);
    c32* S = TB + L;
    stage_table(TB, tw4 + L, L);
    const int si = slot_of(sl, ns, blockIdx.x, 0);
    const MSlot d = sl[si];
    const long long plane = (long long)d.n0 * d.n1;
    const long long nlines = 3 * plane;
    const long long line0 = (long long)(blockIdx.x - d.zb0) * NL;
    const c32* Ad = A + d.a_off;
    __syncthreads();
    for (int it = threadIdx.x; it < NL * R1; it += Z_THREADS) {
        const int k1 = it % R1, ll = it / R1;
        const long long ln = line0 + ll;
        c32 b[R2];
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) b[k2] = ln < nlines ? Ad[ln * L + k1 + R1 * k2] : z32();
        dftp2<float, R2, true>(b);
#pragma unroll
        for (int q = 0; q < R2; ++q) S[(ll * R1 + k1) * RS + q] = b[q] * tw<true>(TB, q * R1 + k1);
    }
    __syncthreads();
    const int q2 = threadIdx.x % R2, l = threadIdx.x / R2;
    const long long line = line0 + l;
    if (line >= nlines) return;
    c32 a[R1];
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) a[k1] = S[(l * R1 + k1) * RS + q2];
    dftp2_half_out<float, R1, true>(a);
    const int c = (int)(line / plane);
    const long long xy = line - c * plane;
    const c32* wr = d.w + c * cst;
    c32* yr = d.y + c * cst;
    const int* im = d.idx + xy * d.n2;
#pragma unroll
    for (int n1i = 0; n1i < R1 / 2; ++n1i) {
        const int z = n1i * R2 + q2;
        if (z < d.n2) {
            const int vi = im[z];
            if (vi >= 0) {
                const c32 u = a[n1i];
                const c32 wv = wr[vi];
                const float ch = d.chi[vi];
                yr[vi] = c32{wv.x - ch * u.x, wv.y - ch * u.y};
            }
        }
    }
}

// y pass over slots: forward A[slot] [3 n0][n1][P2] -> B[slot] [3 n0][P1][P2],
// inverse B -> A (the half transforms: n1 <= L/2 always holds here)
template <int L, bool INV>
__global__ void __launch_bounds__(Fac<L>::R2 * AX_TW) k_axis_m(const MSlot* __restrict__ sl, int ns,
                                                               c32* __restrict__ A, c32* __restrict__ B,
                                                               long long inner, const c32* __restrict__ tw4) {
    constexpr int R1 = Fac<L>::R1, R2 = Fac<L>::R2, TW = AX_TW, NT = R2 * TW;
    constexpr int SR = R2 * TW;
    extern __shared__ __align__(16) unsigned char smraw[];
    c32* T = reinterpret_cast<c32*>(smraw);
    c32* S = T + L;
    stage_table(T, tw4 + (INV ? L : 0), L);
    const int si = slot_of(sl, ns, blockIdx.x, 1);
    const MSlot d = sl[si];
    const long long ntile = (inner + TW - 1) / TW;
    const long long lb = blockIdx.x - d.yb0;
    const long long o = lb / ntile;
    const long long i0 = (lb - o * ntile) * TW;
    const int n_in = INV ? L : d.n1, n_out = INV ? d.n1 : L;
    const c32* in = INV ? B + d.b_off : A + d.a_off;
    c32* out = INV ? A + d.a_off : B + d.b_off;
    const int t = threadIdx.x % TW, n2 = threadIdx.x / TW;
    __syncthreads();
    if (!INV) {
        c32 a[R1];
        const bool ok = i0 + t < inner;
#pragma unroll
        for (int n1 = 0; n1 < R1 / 2; ++n1) {
            const int p = n1 * R2 + n2;
            a[n1] = (ok && p < n_in) ? in[(o * n_in + p) * inner + i0 + t] : z32();
        }
        dftp2_half_in<float, R1, false>(a);
#pragma unroll
        for (int k1 = 1; k1 < R1; ++k1) a[k1] = a[k1] * tw<false>(T, k1 * R2 + n2);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) S[k1 * SR + n2 * TW + t] = a[k1];
        __syncthreads();
        for (int it = threadIdx.x; it < R1 * TW; it += NT) {
            const int k1 = it / TW, tt = it % TW;
            c32 b[R2];
#pragma unroll
            for (int q = 0; q < R2; ++q) b[q] = S[k1 * SR + q * TW + tt];
            dftp2<float, R2, false>(b);
            if (i0 + tt < inner) {
#pragma unroll
                for (int k2 = 0; k2 < R2; ++k2) out[(o * n_out + k1 + R1 * k2) * inner + i0 + tt] = b[k2];
            }
        }
    } else {
        for (int it = threadIdx.x; it < R1 * TW; it += NT) {
            const int k1 = it / TW, tt = it % TW;
            const bool ok = i0 + tt < inner;
            c32 b[R2];
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) b[k2] = ok ? in[(o * n_in + k1 + R1 * k2) * inner + i0 + tt] : z32();
            dftp2<float, R2, true>(b);
#pragma unroll
            for (int q = 0; q < R2; ++q) S[k1 * SR + q * TW + tt] = b[q] * tw<true>(T, q * R1 + k1);
        }
        __syncthreads();
        c32 a[R1];
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) a[k1] = S[k1 * SR + n2 * TW + t];
        dftp2_half_out<float, R1, true>(a);
        if (i0 + t < inner) {
#pragma unroll
            for (int n1 = 0; n1 < R1 / 2; ++n1) {
                const int p = n1 * R2 + n2;
                if (p < n_out) out[(o * n_out + p) * inner + i0 + t] = a[n1];
            }
        }
    }
}

// fused x pass over slots (D1): per column tile, every slot in turn; the
// kernel tile is restaged whenever the slot's body (spectrum) changes
template <int L>
__global__ void __launch_bounds__(XF<L>::NT) k_xfused_m(const MSlot* __restrict__ sl, int ns, c32* __restrict__ B,
                                                        long long inner, int P1, int P2, int H0, int H1, int H2,
                                                        const c32* __restrict__ tw4) {
    constexpr int R1 = XF<L>::R1, R2 = XF<L>::R2, TW = XF<L>::TW, NT = XF<L>::NT;
    constexpr int SR = XF<L>::SR, SC = XF<L>::SC, HX = XF<L>::HX, HR = XF<L>::HR;
    extern __shared__ __align__(16) unsigned char smraw[];
    c32* TA = reinterpret_cast<c32*>(smraw);
    c32* TB = TA + L;
    c32* Kt = TB + L;           // [6][HX][TW]
    c32* S = Kt + 6 * HX * TW;  // [3][R1][SR]
    stage_table(TA, tw4, 2 * L);
    const long long i0 = (long long)blockIdx.x * TW;
    const long long HH = (long long)H0 * H1 * H2;
    __shared__ long long coff[TW];
    __shared__ unsigned char cneg[TW];
    if (threadIdx.x < TW) {
        const long long ii = i0 + threadIdx.x;
        long long off = -1;
        unsigned char ng = 0;
        if (ii < inner) {
            const int ky = (int)(ii / P2), kz = (int)(ii - (ii / P2) * P2);
            const bool fly = 2 * ky > P1, flz = 2 * kz > P2;
            off = (long long)(fly ? P1 - ky : ky) * H2 + (flz ? P2 - kz : kz);
            ng = (unsigned char)((fly ? 2 : 0) | (flz ? 4 : 0) | ((fly ^ flz) ? 16 : 0));
        }
        coff[threadIdx.x] = off;
        cneg[threadIdx.x] = ng;
    }
    const int t = threadIdx.x % TW, n2 = threadIdx.x / TW;
    const bool okt = i0 + t < inner;
    const long long rs = (long long)R2 * inner;
    const c32* khat_cur = nullptr;
    for (int slot = 0; slot < ns; ++slot) {
        const MSlot d = sl[slot];
        if (d.khat != khat_cur) {  // a new body: stage its kernel tile
            __syncthreads();       // the previous body's tile is no longer read
            constexpr int NE = 6 * HX * TW;
            const long long rowst = (long long)H1 * H2;
            for (int e = threadIdx.x; e < NE; e += NT) {
                const int tt = e % TW, fx = (e / TW) % HX, qq = e / (TW * HX);
                const long long off = coff[tt];
                c32 w = off >= 0 ? d.khat[qq * HH + fx * rowst + off] : z32();
                if ((cneg[tt] >> qq) & 1) w = c32{-w.x, -w.y};
                Kt[e] = w;
            }
            khat_cur = d.khat;
        }
        __syncthreads();
        const int n0 = d.n0;
        const long long cs = (long long)n0 * inner;
        c32* base = B + d.b_off;
        c32* col = base + (long long)n2 * inner + i0 + t;
        c32 a[3][R1];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int n1 = 0; n1 < HR; ++n1) a[c][n1] = (okt && n1 * R2 + n2 < n0) ? col[c * cs + n1 * rs] : z32();
#pragma unroll
        for (int c = 0; c < 3; ++c) dftp2_half_in<float, R1, false>(a[c]);
#pragma unroll
        for (int k1 = 1; k1 < R1; ++k1) {
            const c32 w = tw<false>(TA, k1 * R2 + n2);
#pragma unroll
            for (int c = 0; c < 3; ++c) a[c][k1] = a[c][k1] * w;
        }
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int k1 = 0; k1 < R1; ++k1) S[c * SC + k1 * SR + n2 * TW + t] = a[c][k1];
        __syncthreads();
        for (int it = threadIdx.x; it < R1 * TW; it += NT) {
            const int k1 = it / TW, tt = it % TW;
            c32 bx[R2], by[R2], bz[R2];
#pragma unroll
            for (int q = 0; q < R2; ++q) {
                bx[q] = S[0 * SC + k1 * SR + q * TW + tt];
                by[q] = S[1 * SC + k1 * SR + q * TW + tt];
                bz[q] = S[2 * SC + k1 * SR + q * TW + tt];
            }
            dftp2<float, R2, false>(bx);
            dftp2<float, R2, false>(by);
            dftp2<float, R2, false>(bz);
            const c32* kp = Kt + k1 * TW + tt;
            const c32* km = Kt + (L - k1) * TW + tt;
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) {
                const bool flx = 2 * k2 > R2 || (2 * k2 == R2 && k1 > 0);
                const c32* kt = flx ? km - R1 * k2 * TW : kp + R1 * k2 * TW;
                c32 kxx = kt[0], kxy = kt[HX * TW], kxz = kt[2 * HX * TW];
                const c32 kyy = kt[3 * HX * TW], kyz = kt[4 * HX * TW], kzz = kt[5 * HX * TW];
                if (flx) {
                    kxy = c32{-kxy.x, -kxy.y};
                    kxz = c32{-kxz.x, -kxz.y};
                }
                const c32 a0 = bx[k2], b0 = by[k2], c0 = bz[k2];
                bx[k2] = kxx * a0 + kxy * b0 + kxz * c0;
                by[k2] = kxy * a0 + kyy * b0 + kyz * c0;
                bz[k2] = kxz * a0 + kyz * b0 + kzz * c0;
            }
            dftp2<float, R2, true>(bx);
            dftp2<float, R2, true>(by);
            dftp2<float, R2, true>(bz);
#pragma unroll
            for (int q = 0; q < R2; ++q) {
                const c32 w = tw<true>(TB, q * R1 + k1);
                S[0 * SC + k1 * SR + q * TW + tt] = bx[q] * w;
                S[1 * SC + k1 * SR + q * TW + tt] = by[q] * w;
                S[2 * SC + k1 * SR + q * TW + tt] = bz[q] * w;
            }
        }
        __syncthreads();
        if (okt) {
#pragma unroll 1
            for (int c = 0; c < 3; ++c) {
                c32 o[R1];
#pragma unroll
                for (int k1 = 0; k1 < R1; ++k1) o[k1] = S[c * SC + k1 * SR + n2 * TW + t];
                dftp2_half_out<float, R1, true>(o);
                c32* q = col + c * cs;
#pragma unroll
                for (int n1 = 0; n1 < HR; ++n1)
                    if (n1 * R2 + n2 < n0) q[n1 * rs] = o[n1];
            }
        }
    }
}

template <typename K> int set_smem(K k, size_t bytes) {
    if (bytes > 48 * 1024) VIE_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    return VIE_OK;
}

template <int L> int launch_axis_r(const c32* in, c32* out, long long outer, int n_in, int n_out, long long inner,
                                   const c32* tw4, bool inv, cudaStream_t s) {
    constexpr int NT = Fac<L>::R2 * AX_TW;
    const size_t sm = sizeof(c32) * (L + (size_t)L * AX_TW);
    const long long grid = outer * ((inner + AX_TW - 1) / AX_TW);
    const bool half = 2 * (inv ? n_out : n_in) <= L;
    if (inv) {
        if (half) {
            VIE_TRY(set_smem(k_axis_r<L, true, true>, sm));
            k_axis_r<L, true, true><<<(unsigned)grid, NT, sm, s>>>(in, out, inner, n_in, n_out, tw4);
        } else {
            VIE_TRY(set_smem(k_axis_r<L, true, false>, sm));
            k_axis_r<L, true, false><<<(unsigned)grid, NT, sm, s>>>(in, out, inner, n_in, n_out, tw4);
        }
    } else {
        if (half) {
            VIE_TRY(set_smem(k_axis_r<L, false, true>, sm));
            k_axis_r<L, false, true><<<(unsigned)grid, NT, sm, s>>>(in, out, inner, n_in, n_out, tw4);
        } else {
            VIE_TRY(set_smem(k_axis_r<L, false, false>, sm));
            k_axis_r<L, false, false><<<(unsigned)grid, NT, sm, s>>>(in, out, inner, n_in, n_out, tw4);
        }
    }
    return VIE_OK;
}

template <int L> int launch_xfused_r(c32* B, int n0, long long inner, int P1, int P2, const c32* kh, const int* H,
                                     const c32* tw4, int ns, cudaStream_t s, const D2Spec* d2) {
    const size_t sm = d2 ? XF<L>::smem_d2 : XF<L>::smem;
    if (sm > 227 * 1024) return fail(VIE_EINVAL, "fused x pass does not fit in shared memory");
    if (2 * n0 > L) return fail(VIE_EINVAL, "fused x pass: data rows exceed half the padded length");
    const long long grid = (inner + XF_TW - 1) / XF_TW;
    if (d2) {
        VIE_TRY(set_smem(k_xfused_r<L, true>, sm));
        k_xfused_r<L, true><<<(unsigned)grid, XF<L>::NT, sm, s>>>(B, n0, inner, P1, P2, kh, H[0], H[1], H[2], tw4, ns,
                                                                  d2->dtab, d2->dstride, d2->k2);
    } else {
        VIE_TRY(set_smem(k_xfused_r<L, false>, sm));
        k_xfused_r<L, false><<<(unsigned)grid, XF<L>::NT, sm, s>>>(B, n0, inner, P1, P2, kh, H[0], H[1], H[2], tw4,
                                                                   ns, nullptr, 0, 0.f);
    }
    return VIE_OK;
}

template <int L> int launch_zfwd_r(const c32* w, long long wr, const int* list, const int* idx, c32* A, int n0,
                                   int n1, int n2, long long Nb, long long nlines, const c32* tw4, cudaStream_t s,
                                   long long idx_stride) {
    constexpr int NL = Z_THREADS / Fac<L>::R2;
    const size_t sm = sizeof(c32) * (L + (size_t)NL * Fac<L>::R1 * (Fac<L>::R2 + 1));
    if (2 * n2 > L) return fail(VIE_EINVAL, "z pass: grid extent exceeds half the padded length");
    VIE_TRY(set_smem(k_zfwd_r<L>, sm));
    k_zfwd_r<L><<<(unsigned)((nlines + NL - 1) / NL), Z_THREADS, sm, s>>>(w, wr, list, idx, A, n0, n1, n2, Nb, nlines,
                                                                         tw4, idx_stride);
    return VIE_OK;
}

template <int L> int launch_zinv_r(const c32* A, const c32* w, long long wr, c32* y, long long yr, const int* list,
                                   const int* idx, const float* chi, int n0, int n1, int n2, long long Nb,
                                   long long nlines, const c32* tw4, cudaStream_t s, long long chi_cs,
                                   long long idx_stride) {
    constexpr int NL = Z_THREADS / Fac<L>::R2;
    const size_t sm = sizeof(c32) * (L + (size_t)NL * Fac<L>::R1 * (Fac<L>::R2 + 1));
    if (2 * n2 > L) return fail(VIE_EINVAL, "z pass: grid extent exceeds half the padded length");
    VIE_TRY(set_smem(k_zinv_r<L>, sm));
    k_zinv_r<L><<<(unsigned)((nlines + NL - 1) / NL), Z_THREADS, sm, s>>>(A, w, wr, y, yr, list, idx, chi, n0, n1,
                                                                         n2, Nb, nlines, tw4, chi_cs, idx_stride);
    return VIE_OK;
}

template <int L> int launch_multi(const MSlot* dsl, int ns, long long zblocks, long long yblocks, c32* A, c32* B,
                                   long long cst, int P1, int P2, const int* H, const c32* tw0, const c32* tw1,
                                   const c32* tw2, cudaStream_t s) {
    // all three axes share L here (cubic padded sizes)
    constexpr int NLz = Z_THREADS / Fac<L>::R2;
    const size_t smz = sizeof(c32) * (L + (size_t)NLz * Fac<L>::R1 * (Fac<L>::R2 + 1));
    const size_t smy = sizeof(c32) * (L + (size_t)L * AX_TW);
    const size_t smx = XF<L>::smem;
    const long long inner = (long long)P1 * P2;
    VIE_TRY(set_smem(k_zfwd_m<L>, smz));
    VIE_TRY(set_smem(k_zinv_m<L>, smz));
    VIE_TRY(set_smem(k_axis_m<L, false>, smy));
    VIE_TRY(set_smem(k_axis_m<L, true>, smy));
    VIE_TRY(set_smem(k_xfused_m<L>, smx));
    tmr_begin(TMR_ZFWD, s);
    k_zfwd_m<L><<<(unsigned)zblocks, Z_THREADS, smz, s>>>(dsl, ns, A, cst, tw2);
    tmr_end(TMR_ZFWD, s);
    tmr_begin(TMR_YFWD, s);
    k_axis_m<L, false><<<(unsigned)yblocks, Fac<L>::R2 * AX_TW, smy, s>>>(dsl, ns, A, B, P2, tw1);
    tmr_end(TMR_YFWD, s);
    tmr_begin(TMR_XFUSED, s);
    k_xfused_m<L><<<(unsigned)((inner + XF_TW - 1) / XF_TW), XF<L>::NT, smx, s>>>(dsl, ns, B, inner, P1, P2, H[0], H[1],
                                                                                 H[2], tw0);
    tmr_end(TMR_XFUSED, s);
    tmr_begin(TMR_YINV, s);
    k_axis_m<L, true><<<(unsigned)yblocks, Fac<L>::R2 * AX_TW, smy, s>>>(dsl, ns, A, B, P2, tw1);
    tmr_end(TMR_YINV, s);
    tmr_begin(TMR_ZINV, s);
    k_zinv_m<L><<<(unsigned)zblocks, Z_THREADS, smz, s>>>(dsl, ns, A, cst, tw2);
    tmr_end(TMR_ZINV, s);
    count_launch(5);
    VIE_CUDA(cudaGetLastError());
    return VIE_OK;
}

#define VIE_DISPATCH_L(Lv, CALL) \
    switch (Lv) {                \
        case 16: { constexpr int LL = 16; CALL; } break; \
        case 32: { constexpr int LL = 32; CALL; } break; \
        case 64: { constexpr int LL = 64; CALL; } break; \
        case 128: { constexpr int LL = 128; CALL; } break; \
        case 256: { constexpr int LL = 256; CALL; } break; \
        case 512: { constexpr int LL = 512; CALL; } break; \
        default: return fail(VIE_EINVAL, "fast FFT length not supported"); \
    }

}  // namespace

int fast_axis(const c32* in, c32* out, long long outer, int n_in, int n_out, long long inner, int L,
              const c32* tw4, bool inv, cudaStream_t s) {
    VIE_DISPATCH_L(L, VIE_TRY(launch_axis_r<LL>(in, out, outer, n_in, n_out, inner, tw4, inv, s)));
    return VIE_OK;
}

int fast_xfused(c32* B, int n0, long long inner, int L, int P1, int P2, const c32* kh, const int* H,
                const c32* tw4, int ns, cudaStream_t s, const D2Spec* d2) {
    VIE_DISPATCH_L(L, VIE_TRY(launch_xfused_r<LL>(B, n0, inner, P1, P2, kh, H, tw4, ns, s, d2)));
    return VIE_OK;
}

int fast_zfwd(const c32* w, long long wr, const int* list, const int* idx, c32* A, int n0, int n1, int n2,
              long long Nb, long long nlines, int L, const c32* tw4, cudaStream_t s, long long idx_stride) {
    VIE_DISPATCH_L(L, VIE_TRY(launch_zfwd_r<LL>(w, wr, list, idx, A, n0, n1, n2, Nb, nlines, tw4, s, idx_stride)));
    return VIE_OK;
}

int fast_zinv(const c32* A, const c32* w, long long wr, c32* y, long long yr, const int* list, const int* idx,
              const float* chi, int n0, int n1, int n2, long long Nb, long long nlines, int L, const c32* tw4,
              cudaStream_t s, long long chi_cs, long long idx_stride) {
    VIE_DISPATCH_L(L, VIE_TRY(launch_zinv_r<LL>(A, w, wr, y, yr, list, idx, chi, n0, n1, n2, Nb, nlines, tw4, s,
                                                chi_cs, idx_stride)));
    return VIE_OK;
}

int multi_lines_per_cta(int L) {
    int R1 = 0, R2 = 0;
    fast_factors(L, &R1, &R2);
    return Z_THREADS / R2;
}

int fast_multi_apply(const MSlot* dsl, int ns, long long zblocks, long long yblocks, c32* A, c32* B, long long cst,
                     int L, const int* H, const c32* tw0, const c32* tw1, const c32* tw2, cudaStream_t s) {
    switch (L) {
        case 32: return launch_multi<32>(dsl, ns, zblocks, yblocks, A, B, cst, L, L, H, tw0, tw1, tw2, s);
        case 64: return launch_multi<64>(dsl, ns, zblocks, yblocks, A, B, cst, L, L, H, tw0, tw1, tw2, s);
        case 128: return launch_multi<128>(dsl, ns, zblocks, yblocks, A, B, cst, L, L, H, tw0, tw1, tw2, s);
        case 256: return launch_multi<256>(dsl, ns, zblocks, yblocks, A, B, cst, L, L, H, tw0, tw1, tw2, s);
        default: return fail(VIE_EINVAL, "multi-body launches take cubic padded sizes 32, 64, 128 or 256");
    }
}

}  // namespace vie
