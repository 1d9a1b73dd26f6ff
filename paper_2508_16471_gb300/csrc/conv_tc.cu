// 3-D convolutions of the U-Net (net.cu) on the tensor cores: implicit GEMM
// with tcgen05.mma kind::f16 (BF16 operands, FP32 accumulator in tensor
// memory).
//
// Forward (and data gradient, which is a convolution with the transposed,
// offset-reversed weights):
//   y[b][co][v] = bias[co] + sum_{tap, ci} w[co][ci][tap] x[b][ci][v + off(tap)]
// is the product D[m][n] = sum_k A[m][k] B[k][n] with m = a voxel of a tile of
// 128 consecutive voxels, n = the output channel and k = (tap, ci) in chunks of
// 16 channels of one tap.  The CTA stages A (the shifted input, zero outside
// the grid and beyond Ci) and B (the weights, pre-arranged once per call by
// k_conv_tc_weights) in shared memory in the canonical no-swizzle K-major
// layout (core matrices of 8 rows x 16 bytes), one elected thread issues the
// MMAs, completion is signalled through an mbarrier by tcgen05.commit, and the
// epilogue reads the accumulator with tcgen05.ld, adds the bias, applies the
// ReLU and rounds to BF16.  Four stage buffers rotate: the threads stage chunk
// c + 3 while the tensor cores work on chunk c.
//
// Weight gradient:
//   gw[co][ci][tap] += sum_{b, v} gy[b][co][v] x[b][ci][v + off(tap)]
// is, per tap, the product D[m][n] = sum_k A[m][k] B[k][n] with m = co, n = ci
// and k = the (batch, voxel) pairs, split into ranges of kper (a multiple of
// 16, chosen for about eight CTAs per SM) per CTA (split K; the CTA adds its
// FP32 partial product to gw with atomics).
//
// Every wait is bounded; on timeout the kernel records an error flag, frees
// its tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cstdint>

#include "net.cuh"

namespace vie {

namespace {

constexpr int CT_M = 128;         // voxels (rows) per CTA
constexpr int CT_K = 16;          // K per MMA and per chunk (16 BF16 = 32 bytes)
constexpr int CT_THREADS = 128;   // one accumulator lane per thread
constexpr int CT_STAGES = 4;
constexpr int CT_NMAX = 256;      // largest N (output channels, padded to 16)
constexpr long long CT_WAIT_LIMIT = 1LL << 24;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (row, k) of a rows x 16 BF16 tile in the canonical
// K-major no-swizzle layout: core matrix = 8 rows x 8 elements (16 bytes);
// the two K-adjacent core matrices 128 bytes apart (LBO), 8-row groups 256
// bytes apart (SBO)
__host__ __device__ __forceinline__ uint32_t ct_off(int row, int k) {
    return (uint32_t)(((row >> 3) * 2 + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}
constexpr uint32_t CT_LBO = 128;
constexpr uint32_t CT_SBO = 256;

__device__ __forceinline__ uint64_t ct_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((CT_LBO >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((CT_SBO >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
    return d;                // base offset 0, no swizzle
}

// instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major, M = 128
__host__ __device__ constexpr uint32_t ct_idesc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(CT_M >> 4) << 24);
}

__device__ __forceinline__ void ct_mma(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, int acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ bool ct_wait(uint32_t bar, uint32_t phase) {
    for (long long it = 0; it < CT_WAIT_LIMIT; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(phase)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__host__ __device__ constexpr uint32_t tmem_cols(int n) {
    return n <= 32 ? 32u : n <= 64 ? 64u : n <= 128 ? 128u : 256u;
}

// offsets (-1, 0, 1 per axis) of tap 0..26 of a 3x3x3 kernel; 0 for a 1x1x1 one
__device__ __forceinline__ void tap_off(int tap, int ks, int& ox, int& oy, int& oz) {
    if (ks == 1) {
        ox = oy = oz = 0;
        return;
    }
    ox = tap / 9 - 1;
    oy = (tap / 3) % 3 - 1;
    oz = tap % 3 - 1;
}

// Allocate / free tensor memory (warp 0) and set up the mbarriers (thread 0).
__device__ __forceinline__ void ct_begin(uint32_t* tmem_slot, uint32_t cols, uint64_t* bar, int nbar) {
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                     "r"(cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < nbar; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar[i])));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
}

__device__ __forceinline__ void ct_end(uint32_t tmem, uint32_t cols) {
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols));
}

// MMAs of one staged chunk (thread 0) and the commit that frees its stage.
__device__ __forceinline__ void ct_issue(uint32_t tmem, const uint8_t* sa, const uint8_t* sb, uint32_t idesc, int acc,
                                         uint64_t* bar) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    ct_mma(tmem, ct_desc(smem_addr(sa)), ct_desc(smem_addr(sb)), idesc, acc);
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar)));
}

// Completion parity of chunk c on its stage's mbarrier (the (c / CT_STAGES)-th
// use of that stage).
__device__ __forceinline__ uint32_t ct_parity(int c) { return (uint32_t)((c / CT_STAGES) & 1); }

// The chunk loop shared by both kernels: stage(c, s) fills stage buffer s with
// chunk c (all threads); thread 0 issues each chunk's MMA and commits it to
// the stage's mbarrier; a stage is refilled once the MMA that last read it has
// completed.  On return the accumulator is complete, or *failed is set (a wait
// ran out), in which case the MMAs already issued have been waited for (again
// bounded) so that the tensor memory can be freed.
template <typename F>
__device__ __forceinline__ void ct_pipeline(int nch, F&& stage, uint32_t tmem, uint32_t idesc, uint32_t stage_bytes,
                                            uint32_t sa_bytes, uint64_t* bar, int* failed, int* err) {
    extern __shared__ __align__(1024) uint8_t ct_smem[];
    const int tid = threadIdx.x;
    for (int c = 0; c < CT_STAGES - 1 && c < nch; ++c) stage(c, c);
    __syncthreads();
    int last = -1;  // last chunk whose MMA was issued
    for (int c = 0; c < nch; ++c) {
        const int s = c % CT_STAGES;
        if (tid == 0) {
            uint8_t* sa = ct_smem + (size_t)s * stage_bytes;
            ct_issue(tmem, sa, sa + sa_bytes, idesc, c > 0 ? 1 : 0, &bar[s]);
        }
        last = c;
        const int cn = c + CT_STAGES - 1;  // next chunk to stage
        if (cn < nch) {
            const int sn = cn % CT_STAGES;
            // stage sn was last read by the MMA of chunk cn - CT_STAGES
            if (cn >= CT_STAGES && !ct_wait(smem_addr(&bar[sn]), ct_parity(cn - CT_STAGES)) && tid == 0) {
                *failed = 1;
                atomicOr(err, 1);
            }
            __syncthreads();
            if (*failed) break;
            stage(cn, sn);
        }
        __syncthreads();
    }
    // a commit completes after every MMA before it: wait for the last one
    if (last >= 0 && !ct_wait(smem_addr(&bar[last % CT_STAGES]), ct_parity(last)) && tid == 0) {
        *failed = 1;
        atomicOr(err, 1);
    }
    __syncthreads();
}

}  // namespace

// wB[chunk][n][16] in the canonical layout of one chunk's B tile (N rows of 16
// K values): chunk = tap * CIC + cc, K value kk = input channel cc * 16 + kk;
// n >= Co and channels >= Ci are zero.  flip: the data-gradient weights
// (w[ci][co][KK - 1 - tap] read as w'[co' = ci][ci' = co][tap]).
__global__ void k_conv_tc_weights(const float* __restrict__ w, int Ci, int Co, int KK, int Npad, int flip,
                                  __nv_bfloat16* __restrict__ wB) {
    const int CIC = (Ci + CT_K - 1) / CT_K;
    const long long total = (long long)KK * CIC * Npad * CT_K;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int kk = (int)(i % CT_K);
        const int n = (int)((i / CT_K) % Npad);
        const long long ch = i / ((long long)CT_K * Npad);
        const int tap = (int)(ch / CIC), cc = (int)(ch % CIC);
        const int ci = cc * CT_K + kk;
        float v = 0.f;
        if (n < Co && ci < Ci) {
            // forward: w[co = n][ci][tap] with w laid out [Co][Ci][KK];
            // flip: the stored tensor is the forward one of the transposed layer, [Ci][Co][KK]
            v = flip ? w[((long long)ci * Co + n) * KK + (KK - 1 - tap)] : w[((long long)n * Ci + ci) * KK + tap];
        }
        uint8_t* tile = reinterpret_cast<uint8_t*>(wB) + (size_t)ch * Npad * CT_K * 2;
        *reinterpret_cast<__nv_bfloat16*>(tile + ct_off(n, kk)) = __float2bfloat16(v);
    }
}

// grid: (ceil(V / 128), B, nsplit); dynamic shared memory CT_STAGES stages.
// nsplit > 1 (small grids, where the (tile, batch) CTAs alone would leave most
// SMs idle): CTA z takes the chunks [z nch / nsplit, (z + 1) nch / nsplit) and
// adds its partial sums to the FP32 array acc [B][Co][V] (zeroed by the host);
// k_conv_tc_finish then applies bias, ReLU and the BF16 rounding.
__global__ void __launch_bounds__(CT_THREADS) k_conv_tc(const __nv_bfloat16* __restrict__ x, long long xbs,
                                                       const __nv_bfloat16* __restrict__ wB,
                                                       const float* __restrict__ bias, __nv_bfloat16* __restrict__ y,
                                                       long long ybs, int Ci, int Co, int Npad, int D, int ks,
                                                       int relu, float* __restrict__ acc, int* __restrict__ err) {
    extern __shared__ __align__(1024) uint8_t ct_smem[];
    __shared__ __align__(8) uint64_t bar[CT_STAGES];
    __shared__ uint32_t tmem_base;
    __shared__ int failed;
    const uint32_t sa_bytes = CT_M * CT_K * 2;
    const uint32_t sb_bytes = (uint32_t)Npad * CT_K * 2;
    const uint32_t stage_bytes = sa_bytes + sb_bytes;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int V = D * D * D;
    const int KK = ks * ks * ks;
    const int CIC = (Ci + CT_K - 1) / CT_K;
    const int nall = KK * CIC;
    const int cbeg = (int)((long long)blockIdx.z * nall / gridDim.z);
    const int nch = (int)((long long)(blockIdx.z + 1) * nall / gridDim.z) - cbeg;
    const uint32_t cols = tmem_cols(Npad);
    if (tid == 0) failed = 0;
    ct_begin(&tmem_base, cols, bar, CT_STAGES);
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = ct_idesc(Npad);
    const int v = blockIdx.x * CT_M + tid;  // this thread's voxel (A row)
    const int vx = v / (D * D), vy = (v / D) % D, vz = v % D;
    const __nv_bfloat16* xb = x + blockIdx.y * xbs;

    auto stage = [&](int cl, int s) {
        const int c = cbeg + cl;
        uint8_t* sa = ct_smem + (size_t)s * stage_bytes;
        uint8_t* sb = sa + sa_bytes;
        const int tap = c / CIC, cc = c % CIC;
        int ox, oy, oz;
        tap_off(tap, ks, ox, oy, oz);
        const int X = vx + ox, Y = vy + oy, Z = vz + oz;
        const bool in = v < V && X >= 0 && X < D && Y >= 0 && Y < D && Z >= 0 && Z < D;
        const long long src = ((long long)X * D + Y) * D + Z;
        __align__(16) __nv_bfloat16 r[CT_K];
#pragma unroll
        for (int k = 0; k < CT_K; ++k) {
            const int ci = cc * CT_K + k;
            r[k] = (in && ci < Ci) ? xb[(long long)ci * V + src] : __float2bfloat16(0.f);
        }
        *reinterpret_cast<uint4*>(sa + ct_off(tid, 0)) = *reinterpret_cast<const uint4*>(&r[0]);
        *reinterpret_cast<uint4*>(sa + ct_off(tid, 8)) = *reinterpret_cast<const uint4*>(&r[8]);
        // B tile: a straight copy of the pre-arranged chunk
        const uint4* g = reinterpret_cast<const uint4*>(reinterpret_cast<const uint8_t*>(wB) + (size_t)c * sb_bytes);
        uint4* d = reinterpret_cast<uint4*>(sb);
        for (uint32_t i = tid; i < sb_bytes / 16; i += CT_THREADS) d[i] = g[i];
        asm volatile("fence.proxy.async.shared::cta;");
    };

    ct_pipeline(nch, stage, tmem, idesc, stage_bytes, sa_bytes, bar, &failed, err);
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (!failed) {
        const int row = warp * 32 + (tid & 31);
        const int vv = blockIdx.x * CT_M + row;
        __nv_bfloat16* yb = y + blockIdx.y * ybs;
        for (int c0 = 0; c0 < Npad; c0 += 8) {
            uint32_t r[8];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7])
                         : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            if (vv < V) {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int co = c0 + q;
                    if (co < Co) {
                        if (acc) {
                            atomicAdd(acc + ((long long)blockIdx.y * Co + co) * V + vv, __uint_as_float(r[q]));
                        } else {
                            float a = __uint_as_float(r[q]) + (bias ? bias[co] : 0.f);
                            if (relu) a = fmaxf(a, 0.f);
                            yb[(long long)co * V + vv] = __float2bfloat16(a);
                        }
                    }
                }
            }
        }
    }
    ct_end(tmem, cols);
}

// y[b][co][v] = bf16(relu(acc[b][co][v] + bias[co])) after a split-K convolution
__global__ void k_conv_tc_finish(const float* __restrict__ acc, const float* __restrict__ bias,
                                 __nv_bfloat16* __restrict__ y, long long ybs, int Co, int V, int B, int relu) {
    const long long n = (long long)B * Co * V;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(i / ((long long)Co * V));
        const long long r = i - (long long)b * Co * V;
        const int co = (int)(r / V);
        float a = acc[i] + (bias ? bias[co] : 0.f);
        if (relu) a = fmaxf(a, 0.f);
        y[b * ybs + r] = __float2bfloat16(a);
    }
}

// grid: (ceil(B V / kper), KK); M = Co (<= 128 rows of A, zero-padded),
// N = Ci padded to 16 (<= 256), K = (batch, voxel) pairs
__global__ void __launch_bounds__(CT_THREADS) k_wgrad_tc(const __nv_bfloat16* __restrict__ gy, long long gbs,
                                                        const __nv_bfloat16* __restrict__ x, long long xbs,
                                                        float* __restrict__ gw, int Ci, int Co, int Npad, int D,
                                                        int ks, int B, int kper, int* __restrict__ err) {
    extern __shared__ __align__(1024) uint8_t ct_smem[];
    __shared__ __align__(8) uint64_t bar[CT_STAGES];
    __shared__ uint32_t tmem_base;
    __shared__ int failed;
    const uint32_t sa_bytes = CT_M * CT_K * 2;
    const uint32_t sb_bytes = (uint32_t)Npad * CT_K * 2;
    const uint32_t stage_bytes = sa_bytes + sb_bytes;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int V = D * D * D;
    const int KK = ks * ks * ks;
    const int tap = blockIdx.y;
    int ox, oy, oz;
    tap_off(tap, ks, ox, oy, oz);
    const long long t0 = (long long)blockIdx.x * kper;
    const long long tot = (long long)B * V;
    const int nch = kper / CT_K;
    const uint32_t cols = tmem_cols(Npad);
    if (tid == 0) failed = 0;
    ct_begin(&tmem_base, cols, bar, CT_STAGES);
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = ct_idesc(Npad);

    // chunk c: K values t0 + 16 c .. + 15 (batch b, voxel v)
    auto stage = [&](int c, int s) {
        uint8_t* sa = ct_smem + (size_t)s * stage_bytes;
        uint8_t* sb = sa + sa_bytes;
        // A: rows co (128, zero beyond Co), 16 K values of gy; thread = row
        {
            const int co = tid;
            __align__(16) __nv_bfloat16 r[CT_K];
#pragma unroll
            for (int k = 0; k < CT_K; ++k) {
                const long long t = t0 + c * CT_K + k;
                __nv_bfloat16 val = __float2bfloat16(0.f);
                if (co < Co && t < tot) {
                    const int b = (int)(t / V), vv = (int)(t - (long long)b * V);
                    val = gy[b * gbs + (long long)co * V + vv];
                }
                r[k] = val;
            }
            *reinterpret_cast<uint4*>(sa + ct_off(co, 0)) = *reinterpret_cast<const uint4*>(&r[0]);
            *reinterpret_cast<uint4*>(sa + ct_off(co, 8)) = *reinterpret_cast<const uint4*>(&r[8]);
        }
        // B: rows ci (Npad), the 16 K values of the shifted input (zero outside the grid)
        for (int e = tid; e < Npad * CT_K; e += CT_THREADS) {
            const int ci = e / CT_K, k = e % CT_K;
            const long long t = t0 + c * CT_K + k;
            __nv_bfloat16 val = __float2bfloat16(0.f);
            if (ci < Ci && t < tot) {
                const int b = (int)(t / V), vv = (int)(t - (long long)b * V);
                const int X = vv / (D * D) + ox, Y = (vv / D) % D + oy, Z = vv % D + oz;
                if (X >= 0 && X < D && Y >= 0 && Y < D && Z >= 0 && Z < D)
                    val = x[b * xbs + (long long)ci * V + ((long long)X * D + Y) * D + Z];
            }
            *reinterpret_cast<__nv_bfloat16*>(sb + ct_off(ci, k)) = val;
        }
        asm volatile("fence.proxy.async.shared::cta;");
    };

    ct_pipeline(nch, stage, tmem, idesc, stage_bytes, sa_bytes, bar, &failed, err);
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (!failed) {
        const int co = warp * 32 + (tid & 31);
        for (int c0 = 0; c0 < Npad; c0 += 8) {
            uint32_t r[8];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7])
                         : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            if (co < Co) {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int ci = c0 + q;
                    if (ci < Ci) atomicAdd(gw + ((long long)co * Ci + ci) * KK + tap, __uint_as_float(r[q]));
                }
            }
        }
    }
    ct_end(tmem, cols);
}

namespace {
size_t conv_tc_smem(int Npad) { return (size_t)CT_STAGES * (CT_M * CT_K * 2 + (size_t)Npad * CT_K * 2); }

// the dynamic shared memory of the largest tile, set once per kernel
int set_attr(const void* f, std::atomic<unsigned long long>& done) {
    if (first_on_device(done))
        VIE_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)conv_tc_smem(CT_NMAX)));
    return VIE_OK;
}
}  // namespace

int conv_tc_npad(int n) { return ((n + CT_K - 1) / CT_K) * CT_K; }

// the shapes the kernels take: N (output channels, or input channels of the
// weight gradient) padded to 16 up to 256, M of the weight gradient up to 128
bool conv_tc_fits(int Ci, int Co) {
    return Ci >= 1 && Co >= 1 && conv_tc_npad(Co) <= CT_NMAX && conv_tc_npad(Ci) <= CT_NMAX && Co <= CT_M;
}

long long conv_tc_weight_elems(int Ci, int Co, int ks) {
    const int KK = ks * ks * ks;
    return (long long)KK * ((Ci + CT_K - 1) / CT_K) * conv_tc_npad(Co) * CT_K;
}

int conv_tc_fwd(const __nv_bfloat16* x, long long xbs, const float* w, int flip, const float* bias,
                __nv_bfloat16* y, long long ybs, int Ci, int Co, int D, int ks, int relu, int B,
                __nv_bfloat16* wB, float* acc, long long acc_elems, int* err, cudaStream_t s) {
    const int Npad = conv_tc_npad(Co);
    if (Npad > CT_NMAX || Ci < 1 || B < 1 || B > 65535) return fail(VIE_EINVAL, "tensor-core convolution: bad sizes");
    const int KK = ks * ks * ks;
    const long long nw = conv_tc_weight_elems(Ci, Co, ks);
    k_conv_tc_weights<<<(unsigned)std::min<long long>(4096, (nw + 255) / 256), 256, 0, s>>>(w, Ci, Co, KK, Npad, flip,
                                                                                          wB);
    count_launch();
    VIE_CUDA(cudaGetLastError());
    static std::atomic<unsigned long long> attr{0};
    VIE_TRY(set_attr((const void*)k_conv_tc, attr));
    const long long V = (long long)D * D * D;
    const long long base = ((V + CT_M - 1) / CT_M) * B;  // (tile, batch) CTAs
    const int nall = KK * ((Ci + CT_K - 1) / CT_K);
    // split K where the CTAs would not fill the GPU twice over, keeping >= 8
    // chunks per CTA, when the FP32 accumulation array is large enough
    int nsplit = 1;
    if (acc && base < 2 * 152 && (long long)B * Co * V <= acc_elems)
        nsplit = (int)std::max<long long>(1, std::min<long long>((2 * 152 + base - 1) / base, nall / 8));
    if (nsplit > 1) VIE_CUDA(cudaMemsetAsync(acc, 0, sizeof(float) * B * Co * V, s));
    dim3 g((unsigned)((V + CT_M - 1) / CT_M), (unsigned)B, (unsigned)nsplit);
    k_conv_tc<<<g, CT_THREADS, conv_tc_smem(Npad), s>>>(x, xbs, wB, bias, y, ybs, Ci, Co, Npad, D, ks, relu,
                                                        nsplit > 1 ? acc : nullptr, err);
    count_launch();
    VIE_CUDA(cudaGetLastError());
    if (nsplit > 1) {
        const long long n = (long long)B * Co * V;
        k_conv_tc_finish<<<(unsigned)std::min<long long>(4096, (n + 255) / 256), 256, 0, s>>>(acc, bias, y, ybs, Co,
                                                                                             (int)V, B, relu);
        count_launch();
        VIE_CUDA(cudaGetLastError());
    }
    return VIE_OK;
}

int conv_tc_wgrad(const __nv_bfloat16* gy, long long gbs, const __nv_bfloat16* x, long long xbs, float* gw, int Ci,
                  int Co, int D, int ks, int B, int* err, cudaStream_t s) {
    const int Npad = conv_tc_npad(Ci);
    if (Npad > CT_NMAX || Co > CT_M || Co < 1 || B < 1) return fail(VIE_EINVAL, "tensor-core weight gradient: bad sizes");
    static std::atomic<unsigned long long> attr{0};
    VIE_TRY(set_attr((const void*)k_wgrad_tc, attr));
    const long long tot = (long long)B * D * D * D;
    const int KK = ks * ks * ks;
    // K per CTA: about eight CTAs per SM over all taps, at least 256
    long long kper = (tot * KK + 8 * 152 - 1) / (8 * 152);
    kper = std::max<long long>(256, ((kper + CT_K - 1) / CT_K) * CT_K);
    kper = std::min<long long>(kper, ((tot + CT_K - 1) / CT_K) * CT_K);
    dim3 g((unsigned)((tot + kper - 1) / kper), (unsigned)KK);
    k_wgrad_tc<<<g, CT_THREADS, conv_tc_smem(Npad), s>>>(gy, gbs, x, xbs, gw, Ci, Co, Npad, D, ks, B, (int)kper, err);
    count_launch();
    VIE_CUDA(cudaGetLastError());
    return VIE_OK;
}

}  // namespace vie
