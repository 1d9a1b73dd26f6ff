// Learned initial guess network (see net.cu).
#pragma once

#include <cuda_bf16.h>

#include <vector>

#include "krylov.cuh"

namespace vie {

constexpr int NET_IN = 10;  // input channels: chi, pol (Re/Im x3), khat (3)
constexpr int PRE_IN = 7;   // preconditioner input channels: chi, Re/Im of the vector (x3)

struct Net {
    static constexpr int NL = 15;  // layers
    enum Buf { IN = 0, E0A, CAT0, P0, E1A, CAT1, P1, E2A, CAT2, P2, BA, BB, D2A, D2B, D1A, D1B, D0A, D0B, OUT, NBUF };
    struct Layer {
        int ci = 0, co = 0, ks = 3;
        long long nw = 0;
        float *w = nullptr, *b = nullptr, *wt = nullptr, *gw = nullptr, *gb = nullptr;
        float *mw = nullptr, *vw = nullptr, *mb = nullptr, *vb = nullptr;
    };
    int c[4] = {16, 32, 64, 128};
    int bf16 = 1;
    int cin = NET_IN;  // input channels
    Layer L[NL];
    long long nparams = 0;
    int t = 0;  // Adam step
    int D = 0, Bcap = 0;
    void* act[NBUF] = {};
    void* grd[NBUF] = {};
    int ch_[NBUF] = {};
    long long vox_[NBUF] = {};
    float* d_loss = nullptr;
    float mask_sum = 1.f;
    std::vector<void*> owned;
    // BF16 storage: convolutions on the tensor cores (conv_tc.cu) unless switched off
    int tc = 1;
    void* wB = nullptr;       // BF16 weights of one layer in the tensor-core chunk layout
    int* d_err = nullptr;     // set by a tensor-core kernel whose wait ran out
    float* acc32 = nullptr;   // FP32 split-K accumulation of the small-grid convolutions
    long long acc32_elems = 0;

    ~Net();
    int alloc(void** p, size_t bytes);
    int init(const int* ch, unsigned long long seed, int store_bf16, int cin = NET_IN);
    int reserve(int B, int D);
    int set_input(const float* x_dev, int B, cudaStream_t s);
    int get_output(float* y_dev, int B, cudaStream_t s);
    int forward(int B, cudaStream_t s);
    int backward(int B, cudaStream_t s);
    int loss_grad(const float* t_dev, const float* m_dev, int B, cudaStream_t s, float* loss_host);
    int adam(float lr, cudaStream_t s);
    const float* bly_w(int l) const;

    template <typename S> int forward_t(int B, cudaStream_t s);
    template <typename S> int backward_t(int B, cudaStream_t s);
    template <typename S> int conv_fwd(int l, int src, int src_c0, int dst, int dst_c0, int Dl, int B, int relu,
                                       cudaStream_t s);
    template <typename S> int conv_bwd(int l, int src, int src_c0, int dst, int dst_c0, int Dl, int B, int relu,
                                       int want_dx, cudaStream_t s);
};

// Tensor-core (tcgen05, BF16 operands, FP32 accumulation) convolutions of the
// network; see conv_tc.cu.  wB holds conv_tc_weight_elems(Ci, Co, ks) BF16.
int conv_tc_npad(int n);
long long conv_tc_weight_elems(int Ci, int Co, int ks);
// acc: FP32 scratch of acc_elems floats for the split-K path on small grids
// (needs B Co D^3; NULL: never split)
int conv_tc_fwd(const __nv_bfloat16* x, long long xbs, const float* w, int flip, const float* bias,
                __nv_bfloat16* y, long long ybs, int Ci, int Co, int D, int ks, int relu, int B,
                __nv_bfloat16* wB, float* acc, long long acc_elems, int* err, cudaStream_t s);
int conv_tc_wgrad(const __nv_bfloat16* gy, long long gbs, const __nv_bfloat16* x, long long xbs, float* gw, int Ci,
                  int Co, int D, int ks, int B, int* err, cudaStream_t s);
bool conv_tc_fits(int Ci, int Co);

// features of the solver's RHS on the coarse grid (edge n/f per axis):
// x [rhs][10][D^3] = (chi averaged over each f^3 block, Re/Im of the
// polarisation, khat); when `w` is given also the training target
// t [rhs][6][D^3] (block average over body voxels of
// (E_tot - E_inc) exp(-i k0 khat.r), E_tot = w/chi) and the mask m [rhs][D^3]
// (fraction of body voxels in the block)
int net_features(Operator& op, const double* chans_dev, int n_rhs, int f, float* x, const c64* w, long long wstride,
                 float* t, float* m, cudaStream_t s);
// x0 on the fine body voxels: chi (E_inc + upsampled prediction y [rhs][6][D^3])
int device_sum(const float* a, long long n, float* out_host, float* scratch, cudaStream_t s);
int net_initial_guess(Operator& op, const double* chans_dev, int n_rhs, int f, const float* y, c64* x0,
                      long long xstride, cudaStream_t s);

// preconditioner training pairs: for n FP32 vectors v [n][3 Nb] and u = A v,
// x [n][7][D^3] from u and targets t [n][6][D^3] = block average of (v - u),
// both scaled by sqrt(3 Nb)/||u||; m [n][D^3] the body fraction
int precond_pairs(Operator& op, int f, const c32* v, int n, const c32* u, float* x, float* t, float* m,
                  cudaStream_t s);

}  // namespace vie
