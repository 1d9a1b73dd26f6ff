// Batched GMRES state and driver (see krylov.cu).
#pragma once

#include <vector>

#include "vie_internal.cuh"

namespace vie {

constexpr int MAX_RESTART = 512;

struct Net;
// Learned right preconditioner of FGMRES: z = v + (||v|| / sqrt(3 Nb)) up(Net(x)),
// x = [block-averaged chi, sqrt(3 Nb)/||v|| block-averaged Re/Im v] on the D^3
// coarse grid (D = n / f); see net.cu.
struct PrecondCtx {
    Net* net = nullptr;
    int f = 4;
    float* x = nullptr;  // [bcap][7][D^3] network input
    float* y = nullptr;  // [bcap][6][D^3] network output
    int bcap = 0;
    ~PrecondCtx();
};
template <typename T>
int precond_apply(Operator& op, PrecondCtx& pc, const cplx<T>* v, long long vrs, cplx<T>* z, long long zrs,
                  const int* list, int n, cudaStream_t s);

// Block-Jacobi right preconditioner of FGMRES (the block preconditioner of
// Sec. III-B): z approximately solves A_bd z = v, where A_bd keeps only the
// interactions inside each block.  Blocks are the cells of a tiling of the
// grid (cut positions per axis), each cropped to the bounding box of its body
// voxels; A_bd is one batched FFT operator on the largest such box (`bop`),
// one batch slot per block with its own voxel map into the global compact
// vector.  The inner solve is a fixed number of COCR steps from z = 0 (A_bd is
// symmetric in the same chi-weighted bilinear form as A).
struct BlockPrecond {
    Operator bop;             // block-grid operator; chi borrowed from the main operator
    int T = 0;                // non-empty blocks
    int* tiles = nullptr;     // [T] slot list 0..T-1 (device)
    int iters = 8;            // inner COCR steps
    int box[3] = {0, 0, 0};   // block grid
    void* V = nullptr;        // [rcap][5][n3] FP32 inner vectors
    c64* coef = nullptr;      // [rcap][8] inner scalars
    c64* partial = nullptr;   // [rcap][2][nblk]
    int* flag = nullptr;      // [rcap] breakdown flags (inner steps continue with zeroed scalars)
    int rcap = 0;
    long long n3 = 0;
    void release(Operator& op);
};
// Host part: blocks of the tiling given by `cuts` (ncuts[a] interior cuts on axis a), each cropped to the box
// of its body voxels (vox: increasing linear indices); box = the largest extent per axis; T = non-empty
// blocks; map (optional) [T][box voxels] = compact index or -1.
int block_layout(const int n[3], const int* vox, long long Nb, const int* cuts, const int ncuts[3], int box[3],
                 int* T, std::vector<int>* map);
int block_precond_setup(Operator& op, BlockPrecond& bp, const int* cuts, const int ncuts[3], int iters);
// y = A_bd w for one FP32 compact vector
int block_apply(Operator& op, BlockPrecond& bp, const c32* w, c32* y);
// z[r] = M(v[r]) for the RHS in d_list / hlist (n of them), FP32 basis
int block_precond_apply(Operator& op, BlockPrecond& bp, const c32* v, long long vrs, c32* z, long long zrs,
                        const int* d_list, const int* hlist, int n, int R);

struct Solver {
    int R = 0, m = 0, prec = 0, nblk = 0;
    long long n3 = 0;          // vector length 3 * Nb
    c64* x = nullptr;          // [R][n3] solution (FP64)
    c64* b = nullptr;          // [R][n3] right-hand sides
    c64* res = nullptr;        // [R][n3] residual / A x scratch
    void* V = nullptr;         // [R][m+1][n3] Krylov basis (float2 or double2)
    c64* H = nullptr;          // [R][m][m+1] Hessenberg, column-major
    double* cs = nullptr;      // [R][m] Givens cosines
    c64* sn = nullptr;         // [R][m] Givens sines
    c64* g = nullptr;          // [R][m+1] rotated residual vector
    c64* y = nullptr;          // [R][m] least-squares solution
    c64* coef = nullptr;       // [R][m+2] projection coefficients (+ ||w||^2 before projection)
    c64* partial = nullptr;    // [R][m+2][nblk] block partial dot products
    double* normpart = nullptr;  // [R][nblk]
    double* inv = nullptr;     // [R] 1 / h_{j+1,j}
    double* target = nullptr;  // [R] inner-cycle stopping threshold
    double* bnorm = nullptr;   // [R]
    double* rnorm = nullptr;   // [R]
    int* kcount = nullptr;     // [R] steps taken in the current cycle
    int* flag = nullptr;       // [R] 1 = stop the current cycle
    int* reorth = nullptr;     // [R] 1 = second Gram-Schmidt pass needed this step
    double* chans = nullptr;   // [R][9] channels of the current right-hand sides
    void* Z = nullptr;         // [R][m][n3] preconditioned basis (FGMRES; allocated on first use)
    // one-sweep Arnoldi (opts.arnoldi = 1; allocated on first use)
    void* Wz = nullptr;        // [R][n3] operator image of the not yet orthogonalised vector
    c64* Hu = nullptr;         // [R][m][m+1] Hessenberg before the Givens rotations, column-major
    c64* lag = nullptr;        // [R][m+1] coefficients that turn the pending vector into the next basis vector
    c64* cvec = nullptr;       // [R][m+2] H_unrotated * lag
    double* beta2 = nullptr;   // [R] squared norm of the pending vector's orthogonal part
    int* kerr = nullptr;       // [1] set by the sweep kernel when a bulk copy did not arrive in time
    // incremental refinement residual (mixed precision; allocated on first use)
    void* dz = nullptr;        // [R][n3] the last cycle's correction, working precision
    int* keep = nullptr;       // [R] 1 = dz holds this RHS's correction
    PrecondCtx* pc = nullptr;  // learned right preconditioner for the next solve (not owned), or null
    BlockPrecond* bpc = nullptr;  // block-Jacobi right preconditioner for the next solve (not owned), or null

    int alloc(Operator& op, int R, int m, int prec);
    void release(Operator& op);
};

struct SolveResult {
    std::vector<int> iters;
    std::vector<double> relres;
    int converged = 0, iters_max = 0, outer_max = 0;
    long long matvecs32 = 0, matvecs64 = 0;
    double relres_max = 0;
    int guesses_rejected = 0;  // initial guesses replaced by zero (worse than x0 = 0)
};

int solver_run(Operator& op, Solver& S, const vie_solve_opts& o, SolveResult& out);

// right-hand sides b[r][c][v] = chi_v pol_rc exp(i k0 khat_r . r_v) (FP64)
int build_rhs(Operator& op, Solver& S, const vie_channel* ch, int n_rhs);

}  // namespace vie
