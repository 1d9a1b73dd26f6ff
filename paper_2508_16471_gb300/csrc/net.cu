// Learned initial guess: a 4-level 3-D U-Net trained and run on the device by
// the library's own kernels (forward, backward, Adam).
//
// Architecture (channels c0..c3, all 3x3x3 convolutions 'same' with bias and
// ReLU, 2x2x2 average pooling, nearest 2x upsampling, skip concatenations,
// 1x1x1 head to 6 channels):
//   enc0 7->c0->c0, enc1 c0->c1->c1, enc2 c1->c2->c2, bottleneck c2->c3->c3,
//   dec2 (c3+c2)->c2->c2, dec1 (c2+c1)->c1->c1, dec0 (c1+c0)->c0->c0, head.
// Activations are stored in S (float or bf16); every product and sum is FP32.
// Weights are FP32 masters (Adam updates them) with an S-rounded copy for the
// convolutions.  Layout [batch][channel][x][y][z] with explicit batch strides
// so that skip connections are written straight into concatenation buffers.
//
// Use in the solver: the network sees, on a grid coarsened by f per axis, the
// block-averaged contrast and the incident channel (polarisation and
// propagation direction, constant channels); it predicts the scattered part
// of the total field with the incident phase removed,
//   d(r) = (E_tot(r) - E_inc(r)) exp(-i k0 khat.r),
// averaged over each block's body voxels.  The initial current is
// x0 = chi (E_inc + d_pred exp(i k0 khat.r)) on the fine body voxels (nearest
// upsampling of d_pred).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <type_traits>
#include <vector>

#include "net.cuh"

namespace vie {

template <typename S> __device__ __forceinline__ float ldf(const S* p) { return (float)p[0]; }
template <> __device__ __forceinline__ float ldf<__nv_bfloat16>(const __nv_bfloat16* p) { return __bfloat162float(p[0]); }
template <typename S> __device__ __forceinline__ S tos(float v) { return (S)v; }
// weights as the storage type sees them (bf16 path: rounded to bf16)
template <typename S> __device__ __forceinline__ float wround(float v) { return v; }
template <> __device__ __forceinline__ float wround<__nv_bfloat16>(float v) { return __bfloat162float(__float2bfloat16(v)); }
template <> __device__ __forceinline__ __nv_bfloat16 tos<__nv_bfloat16>(float v) { return __float2bfloat16(v); }

constexpr int CONV_T = 128;  // voxels per CTA
constexpr int CONV_CO = 8;   // output channels per CTA
constexpr int CONV_CI = 32;  // input channels staged per pass

// y[b][co][v] = bias[co] + sum_{ci,k} w[co][ci][k] x[b][ci][v + off_k] (+ ReLU)
template <typename S>
__global__ void __launch_bounds__(CONV_T) k_conv(const S* __restrict__ x, long long xbs, const float* __restrict__ w,
                                                 const float* __restrict__ bias, S* __restrict__ y, long long ybs,
                                                 int Ci, int Co, int D, int ks, int relu) {
    __shared__ float ws[CONV_CO * CONV_CI * 27];
    const int V = D * D * D;
    const int v = blockIdx.x * CONV_T + threadIdx.x;
    const int co0 = blockIdx.y * CONV_CO;
    const int b = blockIdx.z;
    const int KK = ks * ks * ks;
    const int vx = v / (D * D), vy = (v / D) % D, vz = v % D;
    float acc[CONV_CO];
#pragma unroll
    for (int c = 0; c < CONV_CO; ++c) acc[c] = (bias && co0 + c < Co) ? bias[co0 + c] : 0.f;
    const S* xb = x + b * xbs;
    for (int ci0 = 0; ci0 < Ci; ci0 += CONV_CI) {
        const int nci = min(CONV_CI, Ci - ci0);
        __syncthreads();
        for (int e = threadIdx.x; e < CONV_CO * nci * KK; e += CONV_T) {
            const int c = e / (nci * KK), r = e % (nci * KK);
            const int ci = r / KK, k = r % KK;
            ws[(c * CONV_CI + ci) * 27 + k] =
                (co0 + c < Co) ? wround<S>(w[((long long)(co0 + c) * Ci + ci0 + ci) * KK + k]) : 0.f;
        }
        __syncthreads();
        if (v < V) {
            for (int ci = 0; ci < nci; ++ci) {
                const S* xc = xb + (long long)(ci0 + ci) * V;
                if (ks == 1) {
                    const float xv = ldf(xc + v);
#pragma unroll
                    for (int c = 0; c < CONV_CO; ++c) acc[c] += ws[(c * CONV_CI + ci) * 27] * xv;
                } else {
#pragma unroll
                    for (int k = 0; k < 27; ++k) {
                        const int ox = k / 9 - 1, oy = (k / 3) % 3 - 1, oz = k % 3 - 1;
                        const int X = vx + ox, Y = vy + oy, Z = vz + oz;
                        const bool in = X >= 0 && X < D && Y >= 0 && Y < D && Z >= 0 && Z < D;
                        const float xv = in ? ldf(xc + (X * D + Y) * D + Z) : 0.f;
#pragma unroll
                        for (int c = 0; c < CONV_CO; ++c) acc[c] += ws[(c * CONV_CI + ci) * 27 + k] * xv;
                    }
                }
            }
        }
    }
    if (v < V) {
#pragma unroll
        for (int c = 0; c < CONV_CO; ++c)
            if (co0 + c < Co) {
                float a = acc[c];
                if (relu) a = fmaxf(a, 0.f);
                y[b * ybs + (long long)(co0 + c) * V + v] = tos<S>(a);
            }
    }
}

// wt[ci][co][KK-1-k] = w[co][ci][k]  (transposed, offsets reversed: the data
// gradient of a convolution is a convolution with these weights)
__global__ void k_wflip(const float* __restrict__ w, float* __restrict__ wt, int Ci, int Co, int KK) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Co * Ci * KK) return;
    const int k = i % KK, ci = (i / KK) % Ci, co = i / (KK * Ci);
    wt[((long long)ci * Co + co) * KK + (KK - 1 - k)] = w[i];
}

// g[...] *= (a > 0): ReLU backward using the stored activation
template <typename S>
__global__ void k_relu_bwd(S* __restrict__ g, long long gbs, const S* __restrict__ a, long long abs_, int C, int V, int B) {
    const long long n = (long long)B * C * V;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(i / ((long long)C * V));
        const long long r = i - (long long)b * C * V;
        if (!(ldf(a + b * abs_ + r) > 0.f)) g[b * gbs + r] = tos<S>(0.f);
    }
}

// weight / bias gradients: gw[co][ci][k] += sum_{b,v in chunk} gy[b][co][v] x[b][ci][v+off_k]
template <typename S>
__global__ void k_wgrad(const S* __restrict__ gy, long long gbs, const S* __restrict__ x, long long xbs,
                        float* __restrict__ gw, float* __restrict__ gb, int Ci, int Co, int D, int ks, int B,
                        int chunk) {
    const int KK = ks * ks * ks;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int total = Co * Ci * KK;
    const int V = D * D * D;
    const long long v0 = (long long)blockIdx.y * chunk;
    const long long v1 = min((long long)B * V, v0 + chunk);
    if (idx < total) {
        const int k = idx % KK, ci = (idx / KK) % Ci, co = idx / (KK * Ci);
        const int ox = ks == 3 ? k / 9 - 1 : 0, oy = ks == 3 ? (k / 3) % 3 - 1 : 0, oz = ks == 3 ? k % 3 - 1 : 0;
        float acc = 0.f;
        for (long long t = v0; t < v1; ++t) {
            const int b = (int)(t / V);
            const int v = (int)(t - (long long)b * V);
            const int vx = v / (D * D), vy = (v / D) % D, vz = v % D;
            const int X = vx + ox, Y = vy + oy, Z = vz + oz;
            if (X < 0 || X >= D || Y < 0 || Y >= D || Z < 0 || Z >= D) continue;
            acc += ldf(gy + b * gbs + (long long)co * V + v) * ldf(x + b * xbs + (long long)ci * V + (X * D + Y) * D + Z);
        }
        atomicAdd(gw + idx, acc);
    }
    if (gb && idx < Co) {
        float s = 0.f;
        for (long long t = v0; t < v1; ++t) {
            const int b = (int)(t / V);
            const int v = (int)(t - (long long)b * V);
            s += ldf(gy + b * gbs + (long long)idx * V + v);
        }
        atomicAdd(gb + idx, s);
    }
}

// y[b][c][coarse] = mean of the 2x2x2 fine block (D = fine edge)
// gb[co] += sum over the batch and the voxels of gy[b][co][v] (grid: (Co, chunks))
template <typename S>
__global__ void k_bgrad(const S* __restrict__ gy, long long gbs, float* __restrict__ gb, int V, int B) {
    __shared__ float ws[8];
    const int co = blockIdx.x;
    const long long n = (long long)B * V;
    float acc = 0.f;
    for (long long t = blockIdx.y * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.y * blockDim.x) {
        const int b = (int)(t / V);
        acc += ldf(gy + b * gbs + (long long)co * V + (t - (long long)b * V));
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += ws[q];
        atomicAdd(gb + co, t);
    }
}

template <typename S>
__global__ void k_pool(const S* __restrict__ x, long long xbs, S* __restrict__ y, long long ybs, int C, int D, int B) {
    const int d = D / 2, Vc = d * d * d;
    const long long n = (long long)B * C * Vc;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int v = (int)(i % Vc);
        const int c = (int)((i / Vc) % C);
        const int b = (int)(i / ((long long)Vc * C));
        const int X = v / (d * d), Y = (v / d) % d, Z = v % d;
        const S* xc = x + b * xbs + (long long)c * D * D * D;
        float s = 0.f;
        for (int q = 0; q < 8; ++q)
            s += ldf(xc + ((2 * X + (q >> 2)) * D + 2 * Y + ((q >> 1) & 1)) * D + 2 * Z + (q & 1));
        y[b * ybs + (long long)c * Vc + v] = tos<S>(0.125f * s);
    }
}

// y (fine, edge D) = nearest upsample of x (coarse, edge D/2); if accumulate, y += ...
// mode 0: upsample forward;  mode 1: pool backward (y += g/8 upsampled)
template <typename S>
__global__ void k_up(const S* __restrict__ x, long long xbs, S* __restrict__ y, long long ybs, int C, int D, int B,
                     float scale, int accumulate) {
    const int d = D / 2, V = D * D * D;
    const long long n = (long long)B * C * V;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int v = (int)(i % V);
        const int c = (int)((i / V) % C);
        const int b = (int)(i / ((long long)V * C));
        const int X = v / (D * D) / 2, Y = (v / D) % D / 2, Z = v % D / 2;
        float val = scale * ldf(x + b * xbs + (long long)c * d * d * d + (X * d + Y) * d + Z);
        S* yp = y + b * ybs + (long long)c * V + v;
        if (accumulate) val += ldf(yp);
        *yp = tos<S>(val);
    }
}

// upsample backward: y (coarse) = sum over the 2x2x2 block of g (fine)
template <typename S>
__global__ void k_up_bwd(const S* __restrict__ g, long long gbs, S* __restrict__ y, long long ybs, int C, int D, int B) {
    const int d = D / 2, Vc = d * d * d;
    const long long n = (long long)B * C * Vc;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int v = (int)(i % Vc);
        const int c = (int)((i / Vc) % C);
        const int b = (int)(i / ((long long)Vc * C));
        const int X = v / (d * d), Y = (v / d) % d, Z = v % d;
        const S* gc = g + b * gbs + (long long)c * D * D * D;
        float s = 0.f;
        for (int q = 0; q < 8; ++q)
            s += ldf(gc + ((2 * X + (q >> 2)) * D + 2 * Y + ((q >> 1) & 1)) * D + 2 * Z + (q & 1));
        y[b * ybs + (long long)c * Vc + v] = tos<S>(s);
    }
}

// masked MSE: loss and gradient 2 m (y - t) / den
template <typename S>
__global__ void k_mse(const S* __restrict__ y, const float* __restrict__ t, const float* __restrict__ m,
                      S* __restrict__ g, int C, int V, int B, float inv_den, float* __restrict__ loss) {
    const long long n = (long long)B * C * V;
    float acc = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int v = (int)(i % V);
        const int b = (int)(i / ((long long)C * V));
        const float mm = m[(long long)b * V + v];
        const float d = (ldf(y + i) - t[i]) * mm;
        acc += d * d;
        g[i] = tos<S>(2.f * d * mm * inv_den);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc * inv_den);
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       long long n, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

template <typename S> __global__ void k_to_s(const float* __restrict__ a, S* __restrict__ b, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = tos<S>(a[i]);
}
template <typename S> __global__ void k_to_f(const S* __restrict__ a, float* __restrict__ b, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = ldf(a + i);
}

// ---------------------------------------------------------------------------
// host: the network object
// ---------------------------------------------------------------------------
static int grid1(long long n) { return (int)std::max(1LL, std::min(4096LL, (n + 255) / 256)); }

Net::~Net() {
    for (void* p : owned) cudaFree(p);
}

int Net::alloc(void** p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(VIE_ENOMEM, "network allocation failed");
    }
    owned.push_back(*p);
    return VIE_OK;
}

int Net::init(const int* ch, unsigned long long seed, int store_bf16, int cin_) {
    for (int i = 0; i < 4; ++i) c[i] = ch[i];
    bf16 = store_bf16;
    cin = cin_;
    const int c0 = c[0], c1 = c[1], c2 = c[2], c3 = c[3];
    const int spec[NL][3] = {{cin, c0, 3},       {c0, c0, 3}, {c0, c1, 3}, {c1, c1, 3}, {c1, c2, 3},
                             {c2, c2, 3},      {c2, c3, 3}, {c3, c3, 3}, {c3 + c2, c2, 3}, {c2, c2, 3},
                             {c2 + c1, c1, 3}, {c1, c1, 3}, {c1 + c0, c0, 3}, {c0, c0, 3}, {c0, 6, 1}};
    std::mt19937_64 rng(seed);
    std::normal_distribution<double> nd(0.0, 1.0);
    nparams = 0;
    for (int l = 0; l < NL; ++l) {
        L[l].ci = spec[l][0];
        L[l].co = spec[l][1];
        L[l].ks = spec[l][2];
        const int KK = L[l].ks * L[l].ks * L[l].ks;
        const long long nw = (long long)L[l].co * L[l].ci * KK;
        L[l].nw = nw;
        std::vector<float> hw(nw), hb(L[l].co, 0.f);
        const double sd = std::sqrt(2.0 / (L[l].ci * KK));
        for (long long i = 0; i < nw; ++i) hw[i] = (float)(nd(rng) * sd);
        VIE_TRY(alloc((void**)&L[l].w, 4 * nw));
        VIE_TRY(alloc((void**)&L[l].b, 4 * L[l].co));
        VIE_TRY(alloc((void**)&L[l].wt, 4 * nw));
        VIE_TRY(alloc((void**)&L[l].gw, 4 * nw));
        VIE_TRY(alloc((void**)&L[l].gb, 4 * L[l].co));
        VIE_TRY(alloc((void**)&L[l].mw, 4 * nw));
        VIE_TRY(alloc((void**)&L[l].vw, 4 * nw));
        VIE_TRY(alloc((void**)&L[l].mb, 4 * L[l].co));
        VIE_TRY(alloc((void**)&L[l].vb, 4 * L[l].co));
        VIE_CUDA(cudaMemcpy(L[l].w, hw.data(), 4 * nw, cudaMemcpyHostToDevice));
        VIE_CUDA(cudaMemcpy(L[l].b, hb.data(), 4 * L[l].co, cudaMemcpyHostToDevice));
        VIE_CUDA(cudaMemset(L[l].mw, 0, 4 * nw));
        VIE_CUDA(cudaMemset(L[l].vw, 0, 4 * nw));
        VIE_CUDA(cudaMemset(L[l].mb, 0, 4 * L[l].co));
        VIE_CUDA(cudaMemset(L[l].vb, 0, 4 * L[l].co));
        nparams += nw + L[l].co;
    }
    VIE_TRY(alloc((void**)&d_loss, 4));
    long long wbe = 16;
    for (int l = 0; l < NL; ++l)
        wbe = std::max(wbe, std::max(conv_tc_weight_elems(L[l].ci, L[l].co, L[l].ks),
                                     conv_tc_weight_elems(L[l].co, L[l].ci, L[l].ks)));
    VIE_TRY(alloc(&wB, 2 * wbe));
    VIE_TRY(alloc((void**)&d_err, sizeof(int)));
    VIE_CUDA(cudaMemset(d_err, 0, sizeof(int)));
    t = 0;
    return VIE_OK;
}

int Net::reserve(int B_, int D_) {
    if (B_ <= Bcap && D_ == D && act[0]) return VIE_OK;
    // release old activations
    for (int i = 0; i < NBUF; ++i) {
        if (act[i]) {
            for (size_t q = 0; q < owned.size(); ++q)
                if (owned[q] == act[i]) {
                    cudaFree(act[i]);
                    owned.erase(owned.begin() + q);
                    break;
                }
            act[i] = nullptr;
        }
        if (grd[i]) {
            for (size_t q = 0; q < owned.size(); ++q)
                if (owned[q] == grd[i]) {
                    cudaFree(grd[i]);
                    owned.erase(owned.begin() + q);
                    break;
                }
            grd[i] = nullptr;
        }
    }
    Bcap = B_;
    D = D_;
    const long long V0 = (long long)D * D * D, V1 = V0 / 8, V2 = V1 / 8, V3 = V2 / 8;
    const int c0 = c[0], c1 = c[1], c2 = c[2], c3 = c[3];
    // buffer channel counts and voxel counts
    const long long sizes[NBUF][2] = {
        {cin, V0},      // IN
        {c0, V0},       // E0A
        {c1 + c0, V0},  // CAT0: [up(d1) | s0]
        {c0, V1},       // P0
        {c1, V1},       // E1A
        {c2 + c1, V1},  // CAT1: [up(d2) | s1]
        {c1, V2},       // P1 (pooled s1)
        {c2, V2},       // E2A
        {c3 + c2, V2},  // CAT2: [up(bt) | s2]
        {c2, V3},       // P2
        {c3, V3},       // BA
        {c3, V3},       // BB (bottleneck out)
        {c2, V2},       // D2A
        {c2, V2},       // D2B
        {c1, V1},       // D1A
        {c1, V1},       // D1B
        {c0, V0},       // D0A
        {c0, V0},       // D0B
        {6, V0},        // OUT
    };
    const size_t es = bf16 ? 2 : 4;
    for (int i = 0; i < NBUF; ++i) {
        ch_[i] = (int)sizes[i][0];
        vox_[i] = sizes[i][1];
        VIE_TRY(alloc(&act[i], es * B_ * sizes[i][0] * sizes[i][1]));
        VIE_TRY(alloc(&grd[i], es * B_ * sizes[i][0] * sizes[i][1]));
    }
    // FP32 split-K accumulation for the small-grid tensor-core convolutions
    // (at most 2^25 floats; a layer that needs more is not split)
    if (acc32) {
        for (size_t q = 0; q < owned.size(); ++q)
            if (owned[q] == acc32) {
                cudaFree(acc32);
                owned.erase(owned.begin() + q);
                break;
            }
        acc32 = nullptr;
    }
    acc32_elems = std::min<long long>((long long)B_ * 256 * V0, 1LL << 25);
    VIE_TRY(alloc((void**)&acc32, sizeof(float) * acc32_elems));
    return VIE_OK;
}

template <typename S> int Net::conv_fwd(int l, int src, int src_c0, int dst, int dst_c0, int Dl, int B, int relu,
                                        cudaStream_t s) {
    const Layer& ly = L[l];
    const long long V = (long long)Dl * Dl * Dl;
    const S* x = (const S*)act[src] + (long long)src_c0 * V;
    S* y = (S*)act[dst] + (long long)dst_c0 * V;
    if constexpr (std::is_same_v<S, __nv_bfloat16>) {
        if (tc && conv_tc_fits(ly.ci, ly.co))
            return conv_tc_fwd(x, ch_[src] * V, ly.w, 0, ly.b, y, ch_[dst] * V, ly.ci, ly.co, Dl, ly.ks, relu, B,
                               (__nv_bfloat16*)wB, acc32, acc32_elems, d_err, s);
    }
    dim3 g((unsigned)((V + CONV_T - 1) / CONV_T), (ly.co + CONV_CO - 1) / CONV_CO, B);
    k_conv<S><<<g, CONV_T, 0, s>>>(x, ch_[src] * V, bly_w(l), ly.b, y, ch_[dst] * V, ly.ci, ly.co, Dl, ly.ks, relu);
    count_launch();
    VIE_CUDA(cudaGetLastError());
    return VIE_OK;
}

// weights used by the convolutions: FP32 masters rounded to S
const float* Net::bly_w(int l) const { return L[l].w; }

template <typename S> int Net::forward_t(int B, cudaStream_t s) {
    const int c0 = c[0], c1 = c[1], c2 = c[2], c3 = c[3];
    const int D0 = D, D1 = D / 2, D2 = D / 4, D3 = D / 8;
    auto pool = [&](int src, int src_c0, int C, int Dl, int dst) {
        const long long V = (long long)Dl * Dl * Dl;
        k_pool<S><<<grid1((long long)B * C * V / 8), 256, 0, s>>>((const S*)act[src] + (long long)src_c0 * V,
                                                                  ch_[src] * V, (S*)act[dst], ch_[dst] * V / 8, C, Dl,
                                                                  B);
        count_launch();
    };
    auto up = [&](int src, int C, int Dl, int dst) {  // Dl = fine edge
        const long long V = (long long)Dl * Dl * Dl;
        k_up<S><<<grid1((long long)B * C * V), 256, 0, s>>>((const S*)act[src], ch_[src] * V / 8, (S*)act[dst],
                                                            ch_[dst] * V, C, Dl, B, 1.f, 0);
        count_launch();
    };
    VIE_TRY(conv_fwd<S>(0, IN, 0, E0A, 0, D0, B, 1, s));
    VIE_TRY(conv_fwd<S>(1, E0A, 0, CAT0, c1, D0, B, 1, s));  // s0 -> CAT0[c1:]
    pool(CAT0, c1, c0, D0, P0);
    VIE_TRY(conv_fwd<S>(2, P0, 0, E1A, 0, D1, B, 1, s));
    VIE_TRY(conv_fwd<S>(3, E1A, 0, CAT1, c2, D1, B, 1, s));  // s1 -> CAT1[c2:]
    pool(CAT1, c2, c1, D1, P1);
    VIE_TRY(conv_fwd<S>(4, P1, 0, E2A, 0, D2, B, 1, s));
    VIE_TRY(conv_fwd<S>(5, E2A, 0, CAT2, c3, D2, B, 1, s));  // s2 -> CAT2[c3:]
    pool(CAT2, c3, c2, D2, P2);
    VIE_TRY(conv_fwd<S>(6, P2, 0, BA, 0, D3, B, 1, s));
    VIE_TRY(conv_fwd<S>(7, BA, 0, BB, 0, D3, B, 1, s));
    up(BB, c3, D2, CAT2);
    VIE_TRY(conv_fwd<S>(8, CAT2, 0, D2A, 0, D2, B, 1, s));
    VIE_TRY(conv_fwd<S>(9, D2A, 0, D2B, 0, D2, B, 1, s));
    up(D2B, c2, D1, CAT1);
    VIE_TRY(conv_fwd<S>(10, CAT1, 0, D1A, 0, D1, B, 1, s));
    VIE_TRY(conv_fwd<S>(11, D1A, 0, D1B, 0, D1, B, 1, s));
    up(D1B, c1, D0, CAT0);
    VIE_TRY(conv_fwd<S>(12, CAT0, 0, D0A, 0, D0, B, 1, s));
    VIE_TRY(conv_fwd<S>(13, D0A, 0, D0B, 0, D0, B, 1, s));
    VIE_TRY(conv_fwd<S>(14, D0B, 0, OUT, 0, D0, B, 0, s));
    VIE_CUDA(cudaGetLastError());
    return VIE_OK;
}

// gradient of layer l: g_out (in grd[dst] at channel dst_c0) -> weight grads and
// (if src_grad >= 0) data gradient into grd[src] at src_c0 (accumulate if acc)
template <typename S>
int Net::conv_bwd(int l, int src, int src_c0, int dst, int dst_c0, int Dl, int B, int relu, int want_dx,
                  cudaStream_t s) {
    const Layer& ly = L[l];
    const long long V = (long long)Dl * Dl * Dl;
    S* g = (S*)grd[dst] + (long long)dst_c0 * V;
    const long long gbs = ch_[dst] * V;
    if (relu) {
        k_relu_bwd<S><<<grid1((long long)B * ly.co * V), 256, 0, s>>>(g, gbs, (const S*)act[dst] + (long long)dst_c0 * V,
                                                                    gbs, ly.co, (int)V, B);
        count_launch();
    }
    const S* x = (const S*)act[src] + (long long)src_c0 * V;
    const int KK = ly.ks * ly.ks * ly.ks;
    if constexpr (std::is_same_v<S, __nv_bfloat16>) {
        if (tc && conv_tc_fits(ly.ci, ly.co)) {
            VIE_TRY(conv_tc_wgrad(g, gbs, x, ch_[src] * V, ly.gw, ly.ci, ly.co, Dl, ly.ks, B, d_err, s));
            const int chunks = (int)std::max<long long>(1, std::min<long long>(64, (long long)B * V / 4096));
            k_bgrad<S><<<dim3(ly.co, chunks), 256, 0, s>>>(g, gbs, ly.gb, (int)V, B);
            count_launch();
            if (want_dx)
                VIE_TRY(conv_tc_fwd(g, gbs, ly.w, 1, nullptr, (S*)grd[src] + (long long)src_c0 * V, ch_[src] * V,
                                    ly.co, ly.ci, Dl, ly.ks, 0, B, (__nv_bfloat16*)wB, acc32, acc32_elems, d_err,
                                    s));
            VIE_CUDA(cudaGetLastError());
            return VIE_OK;
        }
    }
    const int total = ly.co * ly.ci * KK;
    const long long work = (long long)B * V;
    int chunks = (int)std::min<long long>(work, std::max<long long>(1, (long long)(600000 + total - 1) / total));
    const int chunk = (int)((work + chunks - 1) / chunks);
    chunks = (int)((work + chunk - 1) / chunk);
    dim3 gg((total + 255) / 256, chunks);
    k_wgrad<S><<<gg, 256, 0, s>>>(g, gbs, x, ch_[src] * V, ly.gw, ly.gb, ly.ci, ly.co, Dl, ly.ks, B, chunk);
    count_launch();
    if (want_dx) {
        k_wflip<<<grid1(ly.nw), 256, 0, s>>>(ly.w, ly.wt, ly.ci, ly.co, KK);
        dim3 g2((unsigned)((V + CONV_T - 1) / CONV_T), (ly.ci + CONV_CO - 1) / CONV_CO, B);
        k_conv<S><<<g2, CONV_T, 0, s>>>(g, gbs, ly.wt, nullptr, (S*)grd[src] + (long long)src_c0 * V, ch_[src] * V,
                                       ly.co, ly.ci, Dl, ly.ks, 0);
        count_launch(2);
    }
    VIE_CUDA(cudaGetLastError());
    return VIE_OK;
}

template <typename S> int Net::backward_t(int B, cudaStream_t s) {
    const int c0 = c[0], c1 = c[1], c2 = c[2], c3 = c[3];
    const int D0 = D, D1 = D / 2, D2 = D / 4, D3 = D / 8;
    for (int l = 0; l < NL; ++l) {
        VIE_CUDA(cudaMemsetAsync(L[l].gw, 0, 4 * L[l].nw, s));
        VIE_CUDA(cudaMemsetAsync(L[l].gb, 0, 4 * L[l].co, s));
    }
    auto upb = [&](int gsrc, int gsrc_c0, int C, int Dl, int gdst) {  // Dl = fine edge; grd[gdst] = coarse
        const long long V = (long long)Dl * Dl * Dl;
        k_up_bwd<S><<<grid1((long long)B * C * V / 8), 256, 0, s>>>((const S*)grd[gsrc] + (long long)gsrc_c0 * V,
                                                                    ch_[gsrc] * V, (S*)grd[gdst], ch_[gdst] * V / 8,
                                                                    C, Dl, B);
        count_launch();
    };
    auto poolb = [&](int gsrc, int C, int Dl, int gdst, int gdst_c0) {  // coarse grad -> += fine skip grad
        const long long V = (long long)Dl * Dl * Dl;
        k_up<S><<<grid1((long long)B * C * V), 256, 0, s>>>((const S*)grd[gsrc], ch_[gsrc] * V / 8,
                                                            (S*)grd[gdst] + (long long)gdst_c0 * V, ch_[gdst] * V, C,
                                                            Dl, B, 0.125f, 1);
        count_launch();
    };
    // grd[OUT] holds dL/dy
    VIE_TRY(conv_bwd<S>(14, D0B, 0, OUT, 0, D0, B, 0, 1, s));
    VIE_TRY(conv_bwd<S>(13, D0A, 0, D0B, 0, D0, B, 1, 1, s));
    VIE_TRY(conv_bwd<S>(12, CAT0, 0, D0A, 0, D0, B, 1, 1, s));  // -> grd[CAT0] (both parts)
    upb(CAT0, 0, c1, D0, D1B);
    VIE_TRY(conv_bwd<S>(11, D1A, 0, D1B, 0, D1, B, 1, 1, s));
    VIE_TRY(conv_bwd<S>(10, CAT1, 0, D1A, 0, D1, B, 1, 1, s));
    upb(CAT1, 0, c2, D1, D2B);
    VIE_TRY(conv_bwd<S>(9, D2A, 0, D2B, 0, D2, B, 1, 1, s));
    VIE_TRY(conv_bwd<S>(8, CAT2, 0, D2A, 0, D2, B, 1, 1, s));
    upb(CAT2, 0, c3, D2, BB);
    VIE_TRY(conv_bwd<S>(7, BA, 0, BB, 0, D3, B, 1, 1, s));
    VIE_TRY(conv_bwd<S>(6, P2, 0, BA, 0, D3, B, 1, 1, s));
    poolb(P2, c2, D2, CAT2, c3);  // s2 grad += pool^T
    VIE_TRY(conv_bwd<S>(5, E2A, 0, CAT2, c3, D2, B, 1, 1, s));
    VIE_TRY(conv_bwd<S>(4, P1, 0, E2A, 0, D2, B, 1, 1, s));
    poolb(P1, c1, D1, CAT1, c2);
    VIE_TRY(conv_bwd<S>(3, E1A, 0, CAT1, c2, D1, B, 1, 1, s));
    VIE_TRY(conv_bwd<S>(2, P0, 0, E1A, 0, D1, B, 1, 1, s));
    poolb(P0, c0, D0, CAT0, c1);
    VIE_TRY(conv_bwd<S>(1, E0A, 0, CAT0, c1, D0, B, 1, 1, s));
    VIE_TRY(conv_bwd<S>(0, IN, 0, E0A, 0, D0, B, 1, 1, s));  // dL/dinput in grd[IN]
    VIE_CUDA(cudaGetLastError());
    return VIE_OK;
}

// a tensor-core wait that ran out (reported once, then cleared)
static int tc_status(int* d_err, cudaStream_t s) {
    int h = 0;
    VIE_CUDA(cudaMemcpyAsync(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    VIE_CUDA(cudaStreamSynchronize(s));
    if (h) {
        VIE_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), s));
        return fail(VIE_ETIMEOUT, "tensor-core convolution: a wait for the MMAs ran out");
    }
    return VIE_OK;
}

int Net::forward(int B, cudaStream_t s) {
    VIE_TRY(bf16 ? forward_t<__nv_bfloat16>(B, s) : forward_t<float>(B, s));
    return bf16 && tc ? tc_status(d_err, s) : VIE_OK;
}
int Net::backward(int B, cudaStream_t s) {
    VIE_TRY(bf16 ? backward_t<__nv_bfloat16>(B, s) : backward_t<float>(B, s));
    return bf16 && tc ? tc_status(d_err, s) : VIE_OK;
}

int Net::set_input(const float* x_dev, int B, cudaStream_t s) {
    const long long n = (long long)B * cin * D * D * D;
    if (bf16) k_to_s<__nv_bfloat16><<<grid1(n), 256, 0, s>>>(x_dev, (__nv_bfloat16*)act[IN], n);
    else VIE_CUDA(cudaMemcpyAsync(act[IN], x_dev, 4 * n, cudaMemcpyDeviceToDevice, s));
    count_launch();
    VIE_CUDA(cudaGetLastError());
    return VIE_OK;
}

int Net::get_output(float* y_dev, int B, cudaStream_t s) {
    const long long n = (long long)B * 6 * D * D * D;
    if (bf16) k_to_f<__nv_bfloat16><<<grid1(n), 256, 0, s>>>((const __nv_bfloat16*)act[OUT], y_dev, n);
    else VIE_CUDA(cudaMemcpyAsync(y_dev, act[OUT], 4 * n, cudaMemcpyDeviceToDevice, s));
    count_launch();
    VIE_CUDA(cudaGetLastError());
    return VIE_OK;
}

int Net::loss_grad(const float* t_dev, const float* m_dev, int B, cudaStream_t s, float* loss_host) {
    const long long V = (long long)D * D * D;
    // denominator: (sum of mask) * 6 channels, computed on the host side of the caller
    VIE_CUDA(cudaMemsetAsync(d_loss, 0, 4, s));
    const float inv_den = 1.f / std::max(1.f, mask_sum * 6.f);
    if (bf16)
        k_mse<__nv_bfloat16><<<grid1((long long)B * 6 * V), 256, 0, s>>>((const __nv_bfloat16*)act[OUT], t_dev, m_dev,
                                                                         (__nv_bfloat16*)grd[OUT], 6, (int)V, B,
                                                                         inv_den, d_loss);
    else
        k_mse<float><<<grid1((long long)B * 6 * V), 256, 0, s>>>((const float*)act[OUT], t_dev, m_dev,
                                                                (float*)grd[OUT], 6, (int)V, B, inv_den, d_loss);
    count_launch();
    VIE_CUDA(cudaGetLastError());
    if (loss_host) {
        VIE_CUDA(cudaMemcpyAsync(loss_host, d_loss, 4, cudaMemcpyDeviceToHost, s));
        VIE_CUDA(cudaStreamSynchronize(s));
    }
    return VIE_OK;
}

int Net::adam(float lr, cudaStream_t s) {
    ++t;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - std::pow(b1, (float)t), c2 = 1.f - std::pow(b2, (float)t);
    for (int l = 0; l < NL; ++l) {
        k_adam<<<grid1(L[l].nw), 256, 0, s>>>(L[l].w, L[l].gw, L[l].mw, L[l].vw, L[l].nw, lr, b1, b2, eps, c1, c2);
        k_adam<<<1, 256, 0, s>>>(L[l].b, L[l].gb, L[l].mb, L[l].vb, L[l].co, lr, b1, b2, eps, c1, c2);
        count_launch(2);
    }
    VIE_CUDA(cudaGetLastError());
    return VIE_OK;
}

}  // namespace vie

namespace vie {

// ---------------------------------------------------------------------------
// solver <-> network features on the coarse grid
// ---------------------------------------------------------------------------
__global__ void k_net_features(int n0, int n1, int n2, int f, int D, double h, double cx, double cy, double cz,
                               double k0, const double* __restrict__ chans, const int* __restrict__ idx_map,
                               const double* __restrict__ chi, const c64* __restrict__ w, long long wstride,
                               long long Nb, float* __restrict__ x, float* __restrict__ t, float* __restrict__ m) {
    const int r = blockIdx.y;
    const long long V = (long long)D * D * D;
    const long long cvox = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (cvox >= V) return;
    const int X = (int)(cvox / ((long long)D * D)), Y = (int)((cvox / D) % D), Z = (int)(cvox % D);
    const double* c = chans + 9 * r;
    double chisum = 0.0;
    int nbody = 0;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int q = 0; q < f * f * f; ++q) {
        const int i = X * f + q / (f * f), j = Y * f + (q / f) % f, k = Z * f + q % f;
        if (i >= n0 || j >= n1 || k >= n2) continue;
        const int vi = idx_map[((long long)i * n1 + j) * n2 + k];
        if (vi < 0) continue;
        const double ch = chi[vi];
        chisum += ch;
        ++nbody;
        if (w) {
            // (E_tot - E_inc) exp(-i k0 khat.r) = (w/chi) exp(-i phase) - pol
            const double ph = k0 * (c[0] * (cx + i * h) + c[1] * (cy + j * h) + c[2] * (cz + k * h));
            double sn, cs;
            sincos(ph, &sn, &cs);
            for (int a = 0; a < 3; ++a) {
                const c64 wv = w[r * wstride + a * Nb + vi];
                const double er = wv.x / ch, ei = wv.y / ch;
                acc[2 * a] += er * cs + ei * sn - c[3 + 2 * a];
                acc[2 * a + 1] += ei * cs - er * sn - c[4 + 2 * a];
            }
        }
    }
    float* xr = x + (long long)r * NET_IN * V;
    xr[cvox] = (float)(chisum / (f * f * f));
    for (int a = 0; a < 3; ++a) {
        xr[(1 + 2 * a) * V + cvox] = (float)c[3 + 2 * a];  // polarisation (constant channels)
        xr[(2 + 2 * a) * V + cvox] = (float)c[4 + 2 * a];
        xr[(7 + a) * V + cvox] = (float)c[a];              // propagation direction
    }
    if (t) {
        float* tr = t + (long long)r * 6 * V;
        for (int a = 0; a < 6; ++a) tr[a * V + cvox] = nbody ? (float)(acc[a] / nbody) : 0.f;
        m[(long long)r * V + cvox] = (float)nbody / (float)(f * f * f);
    }
}

__global__ void k_net_guess(int n1, int n2, int f, int D, double h, double cx, double cy, double cz, double k0,
                            const double* __restrict__ chans, const int* __restrict__ vox,
                            const double* __restrict__ chi, long long Nb, const float* __restrict__ y,
                            c64* __restrict__ x0, long long xstride) {
    const int r = blockIdx.y;
    const long long V = (long long)D * D * D;
    const double* c = chans + 9 * r;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < Nb;
         v += (long long)gridDim.x * blockDim.x) {
        const int lin = vox[v];
        const int k = lin % n2, j = (lin / n2) % n1, i = lin / (n1 * n2);
        const long long cv = ((long long)(i / f) * D + j / f) * D + k / f;
        const double ph = k0 * (c[0] * (cx + i * h) + c[1] * (cy + j * h) + c[2] * (cz + k * h));
        double sn, cs;
        sincos(ph, &sn, &cs);
        const double ch = chi[v];
        const float* yr = y + (long long)r * 6 * V;
        for (int a = 0; a < 3; ++a) {
            // E = (pol + d) exp(i k0 khat.r)
            const double ur = c[3 + 2 * a] + yr[(2 * a) * V + cv], ui = c[4 + 2 * a] + yr[(2 * a + 1) * V + cv];
            x0[r * xstride + a * Nb + v] = c64{ch * (ur * cs - ui * sn), ch * (ur * sn + ui * cs)};
        }
    }
}

static void grid_corner(const Operator& op, double* cx, double* cy, double* cz) {
    *cx = op.origin[0] - 0.5 * (op.n[0] - 1) * op.h;
    *cy = op.origin[1] - 0.5 * (op.n[1] - 1) * op.h;
    *cz = op.origin[2] - 0.5 * (op.n[2] - 1) * op.h;
}

int net_features(Operator& op, const double* chans_dev, int n_rhs, int f, float* x, const c64* w, long long wstride,
                 float* t, float* m, cudaStream_t s) {
    const int D = op.n[0] / f;
    const long long V = (long long)D * D * D;
    double cx, cy, cz;
    grid_corner(op, &cx, &cy, &cz);
    k_net_features<<<dim3((unsigned)((V + 127) / 128), n_rhs), 128, 0, s>>>(
        op.n[0], op.n[1], op.n[2], f, D, op.h, cx, cy, cz, op.k0, chans_dev, op.idx_map, op.chi64, w, wstride, op.Nb,
        x, t, m);
    count_launch();
    VIE_CUDA(cudaGetLastError());
    return VIE_OK;
}

int net_initial_guess(Operator& op, const double* chans_dev, int n_rhs, int f, const float* y, c64* x0,
                      long long xstride, cudaStream_t s) {
    const int D = op.n[0] / f;
    double cx, cy, cz;
    grid_corner(op, &cx, &cy, &cz);
    k_net_guess<<<dim3((unsigned)std::max(1LL, std::min(2048LL, (op.Nb + 255) / 256)), n_rhs), 256, 0, s>>>(
        op.n[1], op.n[2], f, D, op.h, cx, cy, cz, op.k0, chans_dev, op.vox, op.chi64, op.Nb, y, x0, xstride);
    count_launch();
    VIE_CUDA(cudaGetLastError());
    return VIE_OK;
}

// ---- learned right preconditioner (FGMRES) ---------------------------------
// Input of slot s (vector u of RHS r = list[s]): channel 0 the block-averaged
// chi, channels 1..6 Re/Im of sc[s] * (block average of u) per component, with
// sc[s] = sqrt(3 Nb) / ||u|| (unit RMS).  With a training partner v (A v = u)
// the target is sc[s] * block average of (v - u) and m the body fraction.
template <typename T>
__global__ void k_pre_features(int n0, int n1, int n2, int f, int D, const int* __restrict__ idx_map,
                               const double* __restrict__ chi, const cplx<T>* __restrict__ u, long long ustride,
                               const cplx<T>* __restrict__ v, long long vstride, const int* __restrict__ list,
                               const double* __restrict__ sc, double sc0, long long Nb, float* __restrict__ x,
                               float* __restrict__ t, float* __restrict__ m) {
    const int s = blockIdx.y;
    const int r = list ? list[s] : s;
    const long long V = (long long)D * D * D;
    const long long cvox = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (cvox >= V) return;
    const double scale = sc ? sc[s] : sc0;
    const int X = (int)(cvox / ((long long)D * D)), Y = (int)((cvox / D) % D), Z = (int)(cvox % D);
    double chisum = 0.0;
    int nbody = 0;
    double au[6] = {0, 0, 0, 0, 0, 0}, av[6] = {0, 0, 0, 0, 0, 0};
    for (int q = 0; q < f * f * f; ++q) {
        const int i = X * f + q / (f * f), j = Y * f + (q / f) % f, k = Z * f + q % f;
        if (i >= n0 || j >= n1 || k >= n2) continue;
        const int vi = idx_map[((long long)i * n1 + j) * n2 + k];
        if (vi < 0) continue;
        chisum += chi[vi];
        ++nbody;
        for (int a = 0; a < 3; ++a) {
            const cplx<T> uu = u[r * ustride + a * Nb + vi];
            au[2 * a] += (double)uu.x;
            au[2 * a + 1] += (double)uu.y;
            if (v) {
                const cplx<T> vv = v[r * vstride + a * Nb + vi];
                av[2 * a] += (double)vv.x;
                av[2 * a + 1] += (double)vv.y;
            }
        }
    }
    const double inv = nbody ? scale / nbody : 0.0;
    float* xr = x + (long long)s * PRE_IN * V;
    xr[cvox] = (float)(chisum / (f * f * f));
    for (int a = 0; a < 6; ++a) xr[(1 + a) * V + cvox] = (float)(au[a] * inv);
    if (t) {
        float* tr = t + (long long)s * 6 * V;
        for (int a = 0; a < 6; ++a) tr[a * V + cvox] = (float)((av[a] - au[a]) * inv);
        m[(long long)s * V + cvox] = (float)nbody / (float)(f * f * f);
    }
}

// z = v + coef * upsampled y on the body voxels (coef = 1 / sqrt(3 Nb) for unit-norm v)
template <typename T>
__global__ void k_pre_apply(int n1, int n2, int f, int D, const int* __restrict__ vox, long long Nb,
                            const cplx<T>* __restrict__ v, long long vrs, const int* __restrict__ list,
                            const float* __restrict__ y, double coef, cplx<T>* __restrict__ z, long long zrs) {
    const int s = blockIdx.y;
    const int r = list[s];
    const long long V = (long long)D * D * D;
    const float* ys = y + (long long)s * 6 * V;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < Nb;
         e += (long long)gridDim.x * blockDim.x) {
        const int lin = vox[e];
        const int k = lin % n2, j = (lin / n2) % n1, i = lin / (n1 * n2);
        const long long cv = ((long long)(i / f) * D + j / f) * D + k / f;
        for (int a = 0; a < 3; ++a) {
            const cplx<T> vv = v[r * vrs + a * Nb + e];
            z[r * zrs + a * Nb + e] = cplx<T>{(T)((double)vv.x + coef * ys[(2 * a) * V + cv]),
                                              (T)((double)vv.y + coef * ys[(2 * a + 1) * V + cv])};
        }
    }
}

PrecondCtx::~PrecondCtx() {
    cudaFree(x);
    cudaFree(y);
}

template <typename T>
int precond_apply(Operator& op, PrecondCtx& pc, const cplx<T>* v, long long vrs, cplx<T>* z, long long zrs,
                  const int* list, int n, cudaStream_t s) {
    Net& net = *pc.net;
    const int f = pc.f, D = op.n[0] / f;
    const long long V = (long long)D * D * D;
    const int B = std::min(n, 8);
    if (pc.bcap < n) {
        cudaFree(pc.x);
        cudaFree(pc.y);
        pc.x = pc.y = nullptr;
        pc.bcap = 0;
        VIE_CUDA(cudaMalloc(&pc.x, sizeof(float) * PRE_IN * V * n));
        VIE_CUDA(cudaMalloc(&pc.y, sizeof(float) * 6 * V * n));
        pc.bcap = n;
    }
    VIE_TRY(net.reserve(B, D));
    // Krylov vectors have unit norm: sc = sqrt(3 Nb)
    const double sc0 = std::sqrt(3.0 * (double)op.Nb);
    k_pre_features<T><<<dim3((unsigned)((V + 127) / 128), n), 128, 0, s>>>(
        op.n[0], op.n[1], op.n[2], f, D, op.idx_map, op.chi64, v, vrs, (const cplx<T>*)nullptr, 0, list, nullptr, sc0,
        op.Nb, pc.x, nullptr, nullptr);
    count_launch();
    VIE_CUDA(cudaGetLastError());
    for (int r0 = 0; r0 < n; r0 += B) {
        const int nb = std::min(B, n - r0);
        VIE_TRY(net.set_input(pc.x + (long long)r0 * PRE_IN * V, nb, s));
        VIE_TRY(net.forward(nb, s));
        VIE_TRY(net.get_output(pc.y + (long long)r0 * 6 * V, nb, s));
    }
    k_pre_apply<T><<<dim3((unsigned)std::max(1LL, std::min(2048LL, (op.Nb + 255) / 256)), n), 256, 0, s>>>(
        op.n[1], op.n[2], f, D, op.vox, op.Nb, v, vrs, list, pc.y, 1.0 / sc0, z, zrs);
    count_launch();
    VIE_CUDA(cudaGetLastError());
    return VIE_OK;
}
template int precond_apply<float>(Operator&, PrecondCtx&, const c32*, long long, c32*, long long, const int*, int,
                                  cudaStream_t);
template int precond_apply<double>(Operator&, PrecondCtx&, const c64*, long long, c64*, long long, const int*, int,
                                   cudaStream_t);

// sum of |u|^2 per slot (FP64 atomics; training-data path only)
__global__ void k_sq_norms(const c32* __restrict__ u, long long stride, long long n, double* __restrict__ out) {
    const int s = blockIdx.y;
    double acc = 0.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const c32 a = u[s * stride + e];
        acc += (double)a.x * a.x + (double)a.y * a.y;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out + s, acc);
}
__global__ void k_inv_scale(double* __restrict__ a, int n, double sq) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = a[i] > 0 ? sq / sqrt(a[i]) : 0.0;
}

int precond_pairs(Operator& op, int f, const c32* v, int n, const c32* u, float* x, float* t, float* m,
                  cudaStream_t s) {
    const int D = op.n[0] / f;
    const long long V = (long long)D * D * D, nv = 3 * op.Nb;
    double* sc = nullptr;
    VIE_CUDA(cudaMalloc(&sc, sizeof(double) * n));
    int st = VIE_OK;
    cudaMemsetAsync(sc, 0, sizeof(double) * n, s);
    k_sq_norms<<<dim3(256, n), 256, 0, s>>>(u, nv, nv, sc);
    k_inv_scale<<<(n + 127) / 128, 128, 0, s>>>(sc, n, std::sqrt((double)nv));
    k_pre_features<float><<<dim3((unsigned)((V + 127) / 128), n), 128, 0, s>>>(
        op.n[0], op.n[1], op.n[2], f, D, op.idx_map, op.chi64, u, nv, v, nv, nullptr, sc, 0.0, op.Nb, x, t, m);
    count_launch();
    count_launch();
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "preconditioner training pairs");
    cudaFree(sc);
    return st;
}

__global__ void k_sum(const float* __restrict__ a, long long n, float* __restrict__ out) {
    float s = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        s += a[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

int device_sum(const float* a, long long n, float* out_host, float* scratch, cudaStream_t s) {
    VIE_CUDA(cudaMemsetAsync(scratch, 0, 4, s));
    k_sum<<<grid1(n), 256, 0, s>>>(a, n, scratch);
    count_launch();
    VIE_CUDA(cudaMemcpyAsync(out_host, scratch, 4, cudaMemcpyDeviceToHost, s));
    VIE_CUDA(cudaStreamSynchronize(s));
    return VIE_OK;
}

}  // namespace vie
