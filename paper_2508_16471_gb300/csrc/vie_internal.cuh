// Internal declarations shared by the library's translation units.
#pragma once

#include <vector>

#include "common.cuh"
#include "dfloat.cuh"
#include "fft.cuh"

namespace vie {

// device twiddle tables of one axis, in both precisions
struct AxisFFT {
    FFTPlan plan;
    c32* tw32 = nullptr;
    c64* tw64 = nullptr;
    c32* roots32 = nullptr;  // fast path: w_P^{k1 n2} as [k1][n2] then [n2][k1] (2P entries)
    cdf* twdf = nullptr;     // generic-plan twiddles in double-float (the F32X2 operator)
};

// matvec workspace of one precision
struct MatvecWork {
    void* A = nullptr;  // [cap][3][n0][n1][P2]   after the z pass
    void* B = nullptr;  // [cap][3][n0][P1][P2]   after the y pass (x pass in place)
    int cap = 0;        // RHS slots
};

// The discrete operator A w = w - chi (K * w) on one grid.
struct Operator {
    int n[3] = {0, 0, 0};
    int P[3] = {0, 0, 0};
    int H[3] = {0, 0, 0};  // octant extents P/2 + 1
    long long N = 0, Nb = 0;
    double h = 0, k0 = 0, origin[3] = {0, 0, 0};
    AxisFFT ax[3];
    c32* khat32 = nullptr;  // [6][H0][H1][H2] (D1) or [1][H0][H1][H2] (D2 scalar), scaled by 1/(P0 P1 P2)
    c64* khat64 = nullptr;
    cdf* khatdf = nullptr;   // khat64 in double-float (the F32X2 operator)
    int* idx_map = nullptr;  // [N] compact index or -1
    int* vox = nullptr;      // [Nb] linear voxel index of body voxel
    float* chi32 = nullptr;  // [Nb]
    double* chi64 = nullptr; // [Nb]
    dfl* chidf = nullptr;    // chi64 in double-float
    MatvecWork work[2];      // 0: FP32, 1: FP64
    int* d_list = nullptr;   // RHS index list for batched launches
    int list_cap = 0;
    cudaStream_t stream = nullptr;
    double bytes = 0;        // device bytes held
    double line_frac = 1.0;  // fraction of z lines holding a body voxel (algorithmic bytes of the z-inverse pass)
    int fft_path = 0;        // 0: register four-step where the length allows, 1: generic only
    int P_fixed[3] = {0, 0, 0};  // padded lengths chosen by the autotuner (0: padded_size)
    // discretisation: 0 = D1 (voxel-centred unknowns, dyadic kernel), 1 = D2
    // (rooftop unknowns on the +a faces, scalar kernel with discrete grad-div)
    int disc = 0;
    long long chi_cs = 0;    // component stride of chi32/chi64: 0 (D1) or Nb (D2, per-face contrast)
    c32* dtab32 = nullptr;   // D2 difference symbols [3 axes][2 (+,-)][dstride]
    c64* dtab64 = nullptr;
    cdf* dtabdf = nullptr;
    int dstride = 0;
    int ff_engine = 0;       // far-field contractions: 0 tcgen05 3xTF32, 1 CUDA-core FP32
    void* ff_ws = nullptr;   // far-field workspace (grows to the largest grid of directions asked for)
    size_t ff_ws_bytes = 0;
    // voxel maps per batch slot: slot list[s] reads idx_map + list[s] * idx_stride (0: one map for all slots;
    // the block operator of the block-Jacobi preconditioner keeps one map per block)
    long long idx_stride = 0;
    // component stride of the compact vectors this operator reads and writes (0: Nb).  A multi-body batch
    // (batch.cu) stores every body's vectors with the batch's largest body size as the stride.
    long long cstride = 0;
    // the RHS list last uploaded by op_set_list (host copy)
    std::vector<int> h_list;
    // non-null: this operator is the solver's view of a multi-body batch, and op_apply dispatches to it
    struct BatchOps* batch = nullptr;
};

inline long long comp_stride(const Operator& op) { return op.cstride ? op.cstride : op.Nb; }

// device allocation helpers (track bytes)
int dev_alloc(Operator& op, void** p, size_t bytes);
void dev_free(Operator& op, void* p, size_t bytes);

// smooth padded size >= m (factors 2, 3, 5, 7)
int smooth_size(int m);
// padded FFT length used for a grid axis of n voxels
int padded_size(int n);
// padded length >= m: power of two within 15 % of the smooth length, else smooth
int padded_len(int m);

// ---- operator (matvec.cu) ---------------------------------------------------
int op_init_axes(Operator& op);
int op_build_kernel(Operator& op);                 // K-hat octants (FP64 build)
// new padded lengths: frees the twiddles, the kernel spectrum and the matvec
// workspace, then rebuilds the axes and the spectrum (body data unchanged)
int op_replan(Operator& op, const int P[3]);
int op_set_body_device(Operator& op, const double* eps_dev);  // chi, idx_map, vox
int op_reserve(Operator& op, int prec, int nrhs);  // matvec workspace
int op_set_list(Operator& op, const int* host_list, int nr);  // uploads d_list
// y[list[s]] = A w[list[s]] for s < nr.  w, y on the compact layout with RHS
// stride `rstride` elements; prec 0 = float, 1 = double, 2 = double-float
// arithmetic on double inputs and outputs.
int op_apply(Operator& op, int prec, const void* w, long long w_rstride, void* y, long long y_rstride,
             const int* d_list, int nr);
// the same for a multi-body batch (batch.cu); d_list must be op.d_list as set by op_set_list
int batch_apply(Operator& op, int prec, const void* w, long long w_rstride, void* y, long long y_rstride, int nr);
void op_free(Operator& op);

// FP32 fast passes (matvec_fast.cu), power-of-two lengths 16..512
bool fast_length(int L);
void fast_factors(int L, int* R1, int* R2);
int fast_axis(const c32* in, c32* out, long long outer, int n_in, int n_out, long long inner, int L,
              const c32* roots, bool inv, cudaStream_t s);
// D2 spectral multiply: U_a = G (k^2 W_a + d+_a sum_b d-_b W_b), d tables [3][2][dstride]
struct D2Spec {
    const c32* dtab = nullptr;
    int dstride = 0;
    float k2 = 0.f;
};
int fast_xfused(c32* B, int n0, long long inner, int L, int P1, int P2, const c32* kh, const int* H,
                const c32* roots, int ns, cudaStream_t s, const D2Spec* d2 = nullptr);
// idx_stride: voxel maps per slot (slot list[s] uses idx + list[s] * idx_stride); 0 = one shared map
int fast_zfwd(const c32* w, long long wr, const int* list, const int* idx, c32* A, int n0, int n1, int n2,
              long long Nb, long long nlines, int L, const c32* roots, cudaStream_t s, long long idx_stride = 0);
int fast_zinv(const c32* A, const c32* w, long long wr, c32* y, long long yr, const int* list, const int* idx,
              const float* chi, int n0, int n1, int n2, long long Nb, long long nlines, int L, const c32* roots,
              cudaStream_t s, long long chi_cs = 0, long long idx_stride = 0);

// one slot (one RHS of one body) of a multi-body launch (batch.cu, matvec_fast.cu)
struct MSlot {
    const c32* w;            // input row of the RHS (components cst apart)
    c32* y;                  // output row
    const int* idx;          // the body's voxel map [n0][n1][n2]
    const float* chi;        // the body's contrast [Nb]
    const c32* khat;         // the body's kernel octant [6][H0][H1][H2]
    long long a_off, b_off;  // offsets of the slot's work areas in A ([3][n0][n1][P2]) and B ([3][n0][P1][P2])
    long long zb0, yb0;      // first CTA of the slot in the z and y passes
    int n0, n1, n2, pad;
};
int multi_lines_per_cta(int L);
// the five FP32 passes over ns slots of equal cubic padded size L, in one launch each
int fast_multi_apply(const MSlot* d_slots, int ns, long long zblocks, long long yblocks, c32* A, c32* B,
                     long long cst, int L, const int* H, const c32* tw0, const c32* tw1, const c32* tw2,
                     cudaStream_t s);

// tensor-core batched complex GEMM (tc_gemm.cu): C = A B, complex64, strided
int tc_cgemm(int M, int N, int K, int batch, const c32* A, long long sAb, long long sAm, long long sAk, const c32* B,
             long long sBb, long long sBk, long long sBn, c32* C, long long sCb, long long sCm, long long sCn,
             int* d_err, cudaStream_t s);
// CUDA-core FP32 batched complex GEMM (farfield.cu), same contract
int cc_cgemm(int M, int N, int K, int batch, const c32* A, long long sAb, long long sAm, long long sAk, const c32* B,
             long long sBb, long long sBk, long long sBn, c32* C, long long sCb, long long sCm, long long sCn,
             cudaStream_t s);

// standalone batched line FFT (vie_fft_lines)
int fft_lines_device(const void* in, void* out, int L, int count, int inverse, int prec, cudaStream_t s);

}  // namespace vie
