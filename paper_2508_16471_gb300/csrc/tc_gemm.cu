// Tensor-core (tcgen05) batched complex GEMM with a 3xTF32 split, used by the
// far-field contraction (Eq. 25 on a (theta, phi) product grid factorises
// into short dense contractions over z, y and x).
//
// C[b](m, n) = sum_k A[b](m, k) B[b](k, n), complex64 operands with arbitrary
// strides.  The complex product is embedded in a real one with interleaved
// (re, im) columns:
//   Ar[m][2k+p]  = (re, im) of A(m, k)
//   Bs[2k+p][2n+q] = [[ re B, im B ], [ -im B, re B ]](p, q) of B(k, n)
//   C[m][2n+q]   = (re, im) of C(m, n)
// and each real operand x is split x = hi + lo with hi = tf32(x),
// lo = tf32(x - hi); the accumulator (FP32, in tensor memory) receives
// hi*hi + hi*lo + lo*hi, which keeps ~FP32 accuracy (Ootomo & Yokota's split).
//
// One CTA computes a 128 x BN real tile.  Per K chunk the CTA stages A and B
// (hi and lo) in shared memory in the canonical no-swizzle K-major layout
// (8-row x 16-byte core matrices), one elected thread issues tcgen05.mma with
// shared-memory descriptors, completion is signalled through an mbarrier by
// tcgen05.commit, and the epilogue reads the accumulator with tcgen05.ld.
// Two stage buffers alternate: while the tensor cores work on chunk c, the
// threads convert and stage chunk c + 1 into the other buffer, waiting only
// for the MMAs of chunk c - 1 that last read it.  Every wait is bounded; on
// timeout the kernel records an error flag, frees its tensor memory and
// returns.
#include <atomic>
#include <cstdint>

#include "vie_internal.cuh"

namespace vie {

namespace {

constexpr int TC_BM = 128;  // rows per CTA (one accumulator lane per row)
constexpr int TC_BN = 256;  // real columns per CTA (128 complex outputs): A is staged once per 128 outputs
constexpr int TC_BK = 16;   // real K per chunk (8 complex; two MMAs of K = 8)
constexpr int TC_THREADS = 128;
constexpr uint32_t TC_TMEM_COLS = 256;  // two CTAs per SM fill the 512 columns
constexpr long long TC_WAIT_LIMIT = 1LL << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm volatile("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// byte offset of element (row, k) of a rows x TC_BK tile in the K-major,
// no-swizzle canonical layout: core matrix = 8 rows x 4 fp32 (16 B per row);
// K-adjacent core matrices 128 B apart (LBO), 8-row groups 1024 B apart (SBO)
__device__ __forceinline__ uint32_t core_off(int row, int k) {
    return (uint32_t)(((row >> 3) * (TC_BK / 4) + (k >> 2)) * 128 + (row & 7) * 16 + (k & 3) * 4);
}
constexpr uint32_t TC_LBO = 128;
constexpr uint32_t TC_SBO = (TC_BK / 4) * 128;

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((TC_LBO >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((TC_SBO >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
    // base offset 0, absolute LBO mode 0, layout type 0 (no swizzle)
    return d;
}

// instruction descriptor: D f32, A/B tf32, both K-major, M = 128, N = TC_BN
__host__ __device__ constexpr uint32_t tc_idesc() {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_BN >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, int acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase) {
    for (long long it = 0; it < TC_WAIT_LIMIT; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(phase));
        if (ok) return true;
    }
    return false;
}

}  // namespace

// stage chunk kr0 of A (128 rows x TC_BK real) and of Bs^T (TC_BN real output
// columns x TC_BK real) as tf32 hi / lo into one stage buffer
__device__ __forceinline__ void tc_stage(uint8_t* sA_hi, uint8_t* sA_lo, uint8_t* sB_hi, uint8_t* sB_lo, int M, int N,
                                         int K, const c32* __restrict__ A, long long sAm, long long sAk,
                                         const c32* __restrict__ B, long long sBk, long long sBn, int m0, int nr0,
                                         int kr0) {
    const int tid = threadIdx.x;
    for (int e = tid; e < TC_BM * (TC_BK / 2); e += TC_THREADS) {
        const int row = e / (TC_BK / 2), kc = e % (TC_BK / 2);
        const int m = m0 + row, k = kr0 / 2 + kc;
        c32 v = {0.f, 0.f};
        if (m < M && k < K) v = A[m * sAm + k * sAk];
        const uint32_t hr = to_tf32(v.x), hi_ = to_tf32(v.y);
        const uint32_t lr = to_tf32(v.x - __uint_as_float(hr)), li = to_tf32(v.y - __uint_as_float(hi_));
        const uint32_t o0 = core_off(row, 2 * kc), o1 = core_off(row, 2 * kc + 1);
        *reinterpret_cast<uint32_t*>(sA_hi + o0) = hr;
        *reinterpret_cast<uint32_t*>(sA_hi + o1) = hi_;
        *reinterpret_cast<uint32_t*>(sA_lo + o0) = lr;
        *reinterpret_cast<uint32_t*>(sA_lo + o1) = li;
    }
    // Bs^T: row = real output column nr, K contiguous
    for (int e = tid; e < (TC_BN / 2) * (TC_BK / 2); e += TC_THREADS) {
        const int nc = e / (TC_BK / 2), kc = e % (TC_BK / 2);
        const int n = nr0 / 2 + nc, k = kr0 / 2 + kc;
        c32 v = {0.f, 0.f};
        if (n < N && k < K) v = B[k * sBk + n * sBn];
        // rows 2nc (re output) and 2nc+1 (im output); columns 2kc (A re) and 2kc+1 (A im)
        const float vals[4] = {v.x, -v.y, v.y, v.x};
        const int rr[4] = {2 * nc, 2 * nc, 2 * nc + 1, 2 * nc + 1};
        const int kk[4] = {2 * kc, 2 * kc + 1, 2 * kc, 2 * kc + 1};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t h = to_tf32(vals[q]);
            const uint32_t l = to_tf32(vals[q] - __uint_as_float(h));
            const uint32_t o = core_off(rr[q], kk[q]);
            *reinterpret_cast<uint32_t*>(sB_hi + o) = h;
            *reinterpret_cast<uint32_t*>(sB_lo + o) = l;
        }
    }
}

constexpr uint32_t TC_STAGE_BYTES = (uint32_t)(2 * TC_BM + 2 * TC_BN) * TC_BK * 4;

// grid: (ceil(2N / TC_BN), ceil(M / TC_BM), batch)
__global__ void __launch_bounds__(TC_THREADS) k_tc_cgemm(int M, int N, int K, const c32* __restrict__ A, long long sAb,
                                                        long long sAm, long long sAk, const c32* __restrict__ B,
                                                        long long sBb, long long sBk, long long sBn,
                                                        c32* __restrict__ C, long long sCb, long long sCm,
                                                        long long sCn, int* __restrict__ err) {
    extern __shared__ __align__(1024) uint8_t tc_smem[];
    uint8_t* stage[2] = {tc_smem, tc_smem + TC_STAGE_BYTES};
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ uint32_t tmem_base;
    __shared__ int failed;

    const int tid = threadIdx.x, warp = tid >> 5;
    const int bz = blockIdx.z;
    const int m0 = blockIdx.y * TC_BM;
    const int nr0 = blockIdx.x * TC_BN;  // first real output column
    A += bz * sAb;
    B += bz * sBb;
    C += bz * sCb;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;");
        failed = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = tc_idesc();
    const int KR = 2 * K;  // real K
    const int nch = (KR + TC_BK - 1) / TC_BK;
    uint32_t phase[2] = {0, 0};
    auto bufs = [&](int b, uint8_t** ah, uint8_t** al, uint8_t** bh, uint8_t** bl) {
        *ah = stage[b];
        *al = *ah + TC_BM * TC_BK * 4;
        *bh = *al + TC_BM * TC_BK * 4;
        *bl = *bh + TC_BN * TC_BK * 4;
    };
    {
        uint8_t *ah, *al, *bh, *bl;
        bufs(0, &ah, &al, &bh, &bl);
        tc_stage(ah, al, bh, bl, M, N, K, A, sAm, sAk, B, sBk, sBn, m0, nr0, 0);
    }
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    for (int c = 0; c < nch; ++c) {
        const int b = c & 1;
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            uint8_t *ah, *al, *bh, *bl;
            bufs(b, &ah, &al, &bh, &bl);
            const uint32_t aH = smem_u32(ah), aL = smem_u32(al), bH = smem_u32(bh), bL = smem_u32(bl);
#pragma unroll
            for (int kk = 0; kk < TC_BK / 8; ++kk) {
                const uint32_t off = (uint32_t)kk * 2 * 128;  // two K core matrices per MMA (K = 8)
                const int acc0 = (c > 0 || kk > 0) ? 1 : 0;
                mma_tf32(tmem, smem_desc(aH + off), smem_desc(bH + off), idesc, acc0);
                mma_tf32(tmem, smem_desc(aH + off), smem_desc(bL + off), idesc, 1);
                mma_tf32(tmem, smem_desc(aL + off), smem_desc(bH + off), idesc, 1);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&bar[b])));
        }
        if (c + 1 < nch) {
            // the other buffer was last read by the MMAs of chunk c - 1
            const int nb = b ^ 1;
            if (c >= 1) {
                if (!mbar_wait(smem_u32(&bar[nb]), phase[nb]) && tid == 0) {
                    failed = 1;
                    atomicOr(err, 1);
                }
                phase[nb] ^= 1;
            }
            __syncthreads();
            if (failed) break;
            uint8_t *ah, *al, *bh, *bl;
            bufs(nb, &ah, &al, &bh, &bl);
            tc_stage(ah, al, bh, bl, M, N, K, A, sAm, sAk, B, sBk, sBn, m0, nr0, (c + 1) * TC_BK);
            asm volatile("fence.proxy.async.shared::cta;");
        }
        __syncthreads();
    }
    // the last commit completes after every MMA before it
    if (!failed && nch > 0) {
        const int lb = (nch - 1) & 1;
        if (!mbar_wait(smem_u32(&bar[lb]), phase[lb]) && tid == 0) {
            failed = 1;
            atomicOr(err, 1);
        }
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (!failed) {
        // epilogue: warp w owns accumulator lanes (rows) 32w .. 32w+31
        const int row = m0 + warp * 32 + (tid & 31);
#pragma unroll
        for (int c0 = 0; c0 < TC_BN; c0 += 8) {
            uint32_t r[8];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7])
                         : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            if (row < M) {
#pragma unroll
                for (int q = 0; q < 8; q += 2) {
                    const int n = (nr0 + c0 + q) / 2;
                    if (n < N) C[row * sCm + n * sCn] = c32{__uint_as_float(r[q]), __uint_as_float(r[q + 1])};
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
    }
}

int tc_cgemm(int M, int N, int K, int batch, const c32* A, long long sAb, long long sAm, long long sAk, const c32* B,
             long long sBb, long long sBk, long long sBn, c32* C, long long sCb, long long sCm, long long sCn,
             int* d_err, cudaStream_t s) {
    if (M <= 0 || N <= 0 || K <= 0 || batch <= 0) return VIE_OK;
    dim3 g((2 * N + TC_BN - 1) / TC_BN, (M + TC_BM - 1) / TC_BM, batch);
    if (g.y > 65535 || g.z > 65535) return fail(VIE_EINVAL, "tensor-core GEMM grid too large");
    const size_t sm = 2 * (size_t)TC_STAGE_BYTES;  // two stage buffers
    static std::atomic<unsigned long long> init{0};  // repeated attribute calls from racing threads are harmless
    if (first_on_device(init))
        VIE_CUDA(cudaFuncSetAttribute(k_tc_cgemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_tc_cgemm<<<g, TC_THREADS, sm, s>>>(M, N, K, A, sAb, sAm, sAk, B, sBb, sBk, sBn, C, sCb, sCm, sCn, d_err);
    count_launch();
    VIE_CUDA(cudaGetLastError());
    return VIE_OK;
}

}  // namespace vie
