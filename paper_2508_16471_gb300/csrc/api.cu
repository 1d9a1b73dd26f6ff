// C ABI of libvie.so (declarations and contracts in include/vie.h).
#include <array>
#include <algorithm>
#include <thread>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "farfield.cuh"
#include "net.cuh"

struct vie_net {
    vie::Net net;
};

struct vie_handle {
    vie::Operator op;
    vie::Solver S;
    int device = 0;
    int n_rhs = 0;
    bool have_solution = false;
    std::vector<int> vox_host;  // body voxel list (for host-side scatter/gather)
    vie_net* net = nullptr;     // attached initial-guess network (not owned)
    int net_factor = 4;         // coarsening of the network grid
    int guesses_rejected = 0;
    vie::PrecondCtx pctx;       // attached preconditioner network (pctx.net not owned)
    vie::BlockPrecond bpc;      // block-Jacobi preconditioner (vie_set_block_precond)
};

namespace vie {

static thread_local std::string g_err;
static std::atomic<long long> g_launches{0};

void set_error(const std::string& msg) { g_err = msg; }
int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}
int cuda_fail(cudaError_t e, const char* where) {
    g_err = std::string(where) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? VIE_ENOMEM : VIE_EDEVICE;
}
void count_launch(long long n) { g_launches += n; }

int dev_alloc(Operator& op, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(VIE_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    op.bytes += (double)bytes;
    return VIE_OK;
}
void dev_free(Operator& op, void* p, size_t bytes) {
    if (!p) return;
    cudaFree(p);
    op.bytes -= (double)bytes;
}

Operator* handle_operator(vie_handle* hd) { return &hd->op; }
int handle_device(const vie_handle* hd) { return hd->device; }

}  // namespace vie

using namespace vie;

static int check_grid(const vie_grid* g) {
    if (!g) return fail(VIE_EINVAL, "grid is NULL");
    long long N = 1;
    for (int a = 0; a < 3; ++a) {
        if (g->n[a] < 1 || g->n[a] > 4096) return fail(VIE_EINVAL, "grid size per axis must be in 1..4096");
        N *= g->n[a];
    }
    if (N > (1LL << 28)) return fail(VIE_EINVAL, "grid has more than 2^28 voxels");
    if (!(g->h > 0) || !std::isfinite(g->h)) return fail(VIE_EINVAL, "voxel size h must be positive and finite");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(g->origin[a])) return fail(VIE_EINVAL, "origin must be finite");
    return VIE_OK;
}

static int check_eps_host(const double* eps, long long N) {
    if (!eps) return fail(VIE_EINVAL, "eps_r is NULL");
    long long nb = 0;
    for (long long i = 0; i < N; ++i) {
        const double e = eps[i];
        if (!std::isfinite(e) || e < 1.0) return fail(VIE_EINVAL, "eps_r must be finite and >= 1 (lossless dielectric)");
        nb += e > 1.0;
    }
    if (nb == 0) return fail(VIE_EINVAL, "the body is empty (no voxel with eps_r > 1)");
    return VIE_OK;
}

static int refresh_vox_host(vie_handle* hd) {
    hd->vox_host.resize(hd->op.Nb);
    VIE_CUDA(cudaMemcpy(hd->vox_host.data(), hd->op.vox, sizeof(int) * hd->op.Nb, cudaMemcpyDeviceToHost));
    return VIE_OK;
}

static int set_eps_dev(vie_handle* hd, const double* eps_dev) {
    hd->S.release(hd->op);
    hd->bpc.release(hd->op);  // its blocks follow the body
    hd->have_solution = false;
    hd->n_rhs = 0;
    VIE_TRY(op_set_body_device(hd->op, eps_dev));
    return refresh_vox_host(hd);
}

// initial currents of every RHS from the attached network (use_x0 = 2)
static int net_guess(vie_handle* hd, int n_rhs) {
    Operator& op = hd->op;
    const int f = hd->net_factor;
    if (op.n[0] != op.n[1] || op.n[0] != op.n[2] || op.n[0] % (8 * f) != 0)
        return fail(VIE_EINVAL, "the network needs a cubic grid with n divisible by 8 x coarsening factor");
    const int D = op.n[0] / f;
    const long long V = (long long)D * D * D;
    Net& net = hd->net->net;
    const int Bb = std::min(n_rhs, 8);
    VIE_TRY(net.reserve(Bb, D));
    float *x = nullptr, *y = nullptr;
    cudaError_t e = cudaMalloc(&x, sizeof(float) * NET_IN * V * n_rhs);
    if (e == cudaSuccess) e = cudaMalloc(&y, sizeof(float) * 6 * V * n_rhs);
    int st = e == cudaSuccess ? VIE_OK : cuda_fail(e, "network buffers");
    if (st == VIE_OK) st = net_features(op, hd->S.chans, n_rhs, f, x, nullptr, 0, nullptr, nullptr, op.stream);
    for (int r0 = 0; st == VIE_OK && r0 < n_rhs; r0 += Bb) {
        const int nb = std::min(Bb, n_rhs - r0);
        st = net.set_input(x + (long long)r0 * NET_IN * V, nb, op.stream);
        if (st == VIE_OK) st = net.forward(nb, op.stream);
        if (st == VIE_OK) st = net.get_output(y + (long long)r0 * 6 * V, nb, op.stream);
    }
    if (st == VIE_OK) st = net_initial_guess(op, hd->S.chans, n_rhs, f, y, hd->S.x, hd->S.n3, op.stream);
    if (st == VIE_OK) {
        e = cudaStreamSynchronize(op.stream);
        if (e != cudaSuccess) st = cuda_fail(e, "network initial guess");
    }
    cudaFree(x);
    cudaFree(y);
    return st;
}

extern "C" {

void vie_default_opts(vie_solve_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->tol = 1e-6;
    o->restart = 30;
    o->max_iter = 5000;
    o->precision = VIE_PREC_MIXED;
    o->inner_tol = 1e-6;
    o->use_x0 = 0;
    o->precond = 0;
    o->solver = VIE_SOLVER_GMRES;
    o->resid_fp64 = 0;
    o->reorth_eta = 0.1;
    o->inner_floor = 0.7;
    o->arnoldi = 1;
}

const char* vie_last_error(void) { return g_err.c_str(); }

long long vie_kernel_launches(void) { return g_launches.load(); }

int vie_setup(const vie_grid* g, const double* eps_r, double k0, vie_handle** out) {
    return vie_setup_disc(g, eps_r, k0, VIE_DISC_D1, out);
}

int vie_setup_disc(const vie_grid* g, const double* eps_r, double k0, int disc, vie_handle** out) {
    if (!out) return fail(VIE_EINVAL, "out is NULL");
    if (disc != VIE_DISC_D1 && disc != VIE_DISC_D2) return fail(VIE_EINVAL, "disc must be VIE_DISC_D1 or VIE_DISC_D2");
    *out = nullptr;
    VIE_TRY(check_grid(g));
    if (!(k0 > 0) || !std::isfinite(k0)) return fail(VIE_EINVAL, "k0 must be positive and finite");
    const long long N = (long long)g->n[0] * g->n[1] * g->n[2];
    VIE_TRY(check_eps_host(eps_r, N));
    vie_handle* hd = new vie_handle();
    int st = VIE_OK;
    cudaError_t e = cudaGetDevice(&hd->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&hd->op.stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) st = cuda_fail(e, "device / stream setup");
    Operator& op = hd->op;
    for (int a = 0; a < 3; ++a) {
        op.n[a] = g->n[a];
        op.origin[a] = g->origin[a];
    }
    op.N = N;
    op.h = g->h;
    op.k0 = k0;
    op.disc = disc;
    if (st == VIE_OK) st = op_init_axes(op);
    if (st == VIE_OK) st = op_build_kernel(op);
    double* deps = nullptr;
    if (st == VIE_OK) {
        e = cudaMalloc(&deps, sizeof(double) * N);
        if (e == cudaSuccess) e = cudaMemcpy(deps, eps_r, sizeof(double) * N, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) st = cuda_fail(e, "eps upload");
    }
    if (st == VIE_OK) st = set_eps_dev(hd, deps);
    cudaFree(deps);
    if (st != VIE_OK) {
        vie_destroy(hd);
        return st;
    }
    *out = hd;
    return VIE_OK;
}

int vie_set_eps(vie_handle* hd, const double* eps_r) {
    if (!hd) return fail(VIE_EINVAL, "handle is NULL");
    VIE_TRY(check_eps_host(eps_r, hd->op.N));
    VIE_CUDA(cudaSetDevice(hd->device));
    double* deps = nullptr;
    VIE_CUDA(cudaMalloc(&deps, sizeof(double) * hd->op.N));
    cudaError_t e = cudaMemcpy(deps, eps_r, sizeof(double) * hd->op.N, cudaMemcpyHostToDevice);
    int st = e == cudaSuccess ? set_eps_dev(hd, deps) : cuda_fail(e, "eps upload");
    cudaFree(deps);
    return st;
}

int vie_set_eps_device(vie_handle* hd, const double* eps_dev) {
    if (!hd || !eps_dev) return fail(VIE_EINVAL, "NULL argument");
    VIE_CUDA(cudaSetDevice(hd->device));
    return set_eps_dev(hd, eps_dev);
}

int vie_solve(vie_handle* hd, const vie_channel* ch, int n_rhs, const vie_solve_opts* opts, vie_solve_stats* stats) {
    if (!hd || !ch) return fail(VIE_EINVAL, "NULL argument");
    if (n_rhs < 1 || n_rhs > 65535) return fail(VIE_EINVAL, "n_rhs must be in 1..65535");
    vie_solve_opts o;
    if (opts) o = *opts;
    else vie_default_opts(&o);
    if (!(o.tol > 0) || o.restart < 1 || o.restart > MAX_RESTART || o.max_iter < 1 ||
        (o.precision != VIE_PREC_MIXED && o.precision != VIE_PREC_FP64) || !(o.inner_tol > 0))
        return fail(VIE_EINVAL, "invalid solve options (tol > 0, restart 1..512, max_iter >= 1, precision 0/1)");
    for (int r = 0; r < n_rhs; ++r) {
        const double* k = ch[r].khat;
        const double* p = ch[r].pol;
        double kn = 0, pn = 0;
        bool fin = true;
        for (int q = 0; q < 3; ++q) {
            kn += k[q] * k[q];
            fin = fin && std::isfinite(k[q]);
        }
        for (int q = 0; q < 6; ++q) {
            pn += p[q] * p[q];
            fin = fin && std::isfinite(p[q]);
        }
        if (!fin || std::fabs(kn - 1.0) > 1e-9) return fail(VIE_EINVAL, "khat must be a finite unit vector");
        if (!(pn > 0)) return fail(VIE_EINVAL, "polarisation must be nonzero");
        const double dr = p[0] * k[0] + p[2] * k[1] + p[4] * k[2];
        const double di = p[1] * k[0] + p[3] * k[1] + p[5] * k[2];
        if (std::sqrt(dr * dr + di * di) > 1e-10 * std::sqrt(pn))
            return fail(VIE_EINVAL, "polarisation must be transverse to khat");
    }
    if (o.use_x0 == 1 &&
        (!hd->have_solution || hd->n_rhs != n_rhs || hd->S.m != o.restart || hd->S.prec != o.precision))
        return fail(VIE_ESTATE, "use_x0 needs a stored solution with the same n_rhs, restart and precision");
    if (o.use_x0 == 2 && !hd->net) return fail(VIE_ESTATE, "use_x0 = 2 needs a network attached with vie_attach_net");
    if (o.use_x0 < 0 || o.use_x0 > 2) return fail(VIE_EINVAL, "use_x0 must be 0, 1 or 2");
    if (o.precond < 0 || o.precond > 2) return fail(VIE_EINVAL, "precond must be 0, 1 or 2");
    if (o.precond == 2 && (!hd->bpc.T || o.precision != VIE_PREC_MIXED || o.solver != VIE_SOLVER_GMRES ||
                           o.use_x0 == 2))
        return fail(VIE_ESTATE, "precond = 2 needs vie_set_block_precond, mixed precision, GMRES and use_x0 0 or 1");
    if (!(o.reorth_eta >= 0) || !std::isfinite(o.reorth_eta)) return fail(VIE_EINVAL, "reorth_eta must be >= 0");
    if (!(o.inner_floor > 0) || !(o.inner_floor <= 1)) return fail(VIE_EINVAL, "inner_floor must be in (0, 1]");
    if (o.arnoldi != 0 && o.arnoldi != 1) return fail(VIE_EINVAL, "arnoldi must be 0 or 1");
    if (o.solver != VIE_SOLVER_GMRES && o.solver != VIE_SOLVER_BICGSTAB && o.solver != VIE_SOLVER_COCR)
        return fail(VIE_EINVAL, "solver must be VIE_SOLVER_GMRES, VIE_SOLVER_BICGSTAB or VIE_SOLVER_COCR");
    if (o.solver == VIE_SOLVER_BICGSTAB && (o.restart < 8 || o.precond || o.use_x0 == 2))
        return fail(VIE_EINVAL, "BiCGStab needs restart >= 8, precond 0 and use_x0 0 or 1");
    if (o.solver == VIE_SOLVER_COCR && (o.restart < 4 || o.precond || o.use_x0 == 2))
        return fail(VIE_EINVAL, "COCR needs restart >= 4, precond 0 and use_x0 0 or 1");
    if (o.precond == 1 && !hd->pctx.net)
        return fail(VIE_ESTATE, "precond = 1 needs a network attached with vie_attach_precond");
    VIE_CUDA(cudaSetDevice(hd->device));
    auto t0 = std::chrono::steady_clock::now();
    VIE_TRY(hd->S.alloc(hd->op, n_rhs, o.restart, o.precision));
    hd->have_solution = false;
    VIE_TRY(build_rhs(hd->op, hd->S, ch, n_rhs));
    if (o.use_x0 == 2) VIE_TRY(net_guess(hd, n_rhs));
    SolveResult res;
    hd->S.pc = o.precond == 1 ? &hd->pctx : nullptr;
    hd->S.bpc = o.precond == 2 ? &hd->bpc : nullptr;
    int st = solver_run(hd->op, hd->S, o, res);
    hd->S.pc = nullptr;
    hd->S.bpc = nullptr;
    VIE_CUDA(cudaStreamSynchronize(hd->op.stream));
    auto t1 = std::chrono::steady_clock::now();
    if (st != VIE_OK) return st;
    hd->n_rhs = n_rhs;
    hd->have_solution = true;
    hd->guesses_rejected = res.guesses_rejected;
    if (stats) {
        stats->n_rhs = n_rhs;
        stats->converged = res.converged;
        stats->iters_max = res.iters_max;
        stats->outer_max = res.outer_max;
        stats->matvecs32 = res.matvecs32;
        stats->matvecs64 = res.matvecs64;
        stats->relres_max = res.relres_max;
        stats->seconds = std::chrono::duration<double>(t1 - t0).count();
        if (stats->iters)
            for (int r = 0; r < n_rhs; ++r) stats->iters[r] = res.iters[r];
        if (stats->relres)
            for (int r = 0; r < n_rhs; ++r) stats->relres[r] = res.relres[r];
    }
    if (res.converged < n_rhs)
        return fail(VIE_ENOCONV, "solve stopped before reaching tol; largest FP64 residual " +
                                     std::to_string(res.relres_max));
    return VIE_OK;
}

int vie_farfield_dirs_device(vie_handle* hd, const double* dirs_dev, int D, int basis, double* out_dev) {
    if (!hd || !dirs_dev || !out_dev || D < 1) return fail(VIE_EINVAL, "bad arguments");
    if (basis < 0 || basis > 2) return fail(VIE_EINVAL, "basis must be 0, 1 or 2");
    if (!hd->have_solution) return fail(VIE_ESTATE, "no solution stored: call vie_solve first");
    VIE_CUDA(cudaSetDevice(hd->device));
    return farfield_dirs(hd->op, hd->S.x, hd->S.n3, hd->n_rhs, dirs_dev, D, basis, (c64*)out_dev);
}

}  // extern "C"

namespace {
// Gauss-Legendre nodes and weights on [-1, 1] (Newton on P_n from the
// Chebyshev-like initial guesses cos(pi (i + 3/4) / (n + 1/2)))
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            const double pn = n == 0 ? 1.0 : (n == 1 ? z : p1), pm = n == 1 ? 1.0 : p0;
            dp = n * (z * pn - pm) / (z * z - 1.0);
            const double dz = pn / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}
}  // namespace

extern "C" {

int vie_farfield_na(vie_handle* hd, const double* centers, const double* pols, int D, double theta_na, double sigma,
                    int nt, int nphi, double* out) {
    if (!hd || !centers || !pols || !out || D < 1 || nt < 1 || nt > 64 || nphi < 1 || nphi > 256)
        return fail(VIE_EINVAL, "bad arguments (nt in 1..64, nphi in 1..256)");
    if (!(theta_na > 0) || !(theta_na <= M_PI / 2) || !(sigma > 0))
        return fail(VIE_EINVAL, "aperture half-angle in (0, pi/2] and sigma > 0 required");
    if (!hd->have_solution) return fail(VIE_ESTATE, "no solution stored: call vie_solve first");
    const int Q = nt * nphi;
    std::vector<double> gx, gw, dirs(3 * (size_t)D * Q), wts((size_t)D * Q);
    gauss_legendre(nt, gx, gw);
    for (int d = 0; d < D; ++d) {
        double c[3] = {centers[3 * d], centers[3 * d + 1], centers[3 * d + 2]};
        const double cn = std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        if (!(cn > 0)) return fail(VIE_EINVAL, "detector axis is zero");
        for (double& v : c) v /= cn;
        // frame: u = (a x c)/|a x c|, a = z (x when |c_z| >= 0.9); v = c x u
        const double a[3] = {std::fabs(c[2]) < 0.9 ? 0.0 : 1.0, 0.0, std::fabs(c[2]) < 0.9 ? 1.0 : 0.0};
        double u[3] = {a[1] * c[2] - a[2] * c[1], a[2] * c[0] - a[0] * c[2], a[0] * c[1] - a[1] * c[0]};
        const double un = std::sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        for (double& v : u) v /= un;
        const double v[3] = {c[1] * u[2] - c[2] * u[1], c[2] * u[0] - c[0] * u[2], c[0] * u[1] - c[1] * u[0]};
        double tot = 0.0;
        for (int i = 0; i < nt; ++i) {
            const double t = 0.5 * theta_na * (gx[i] + 1.0);
            const double wt = 0.5 * theta_na * gw[i] * std::exp(-t * t / (2.0 * sigma * sigma)) * std::sin(t) *
                              (2.0 * M_PI / nphi);
            for (int j = 0; j < nphi; ++j) {
                const double p = 2.0 * M_PI * j / nphi;
                const size_t q = (size_t)d * Q + (size_t)i * nphi + j;
                for (int k = 0; k < 3; ++k)
                    dirs[3 * q + k] = std::cos(t) * c[k] + std::sin(t) * (std::cos(p) * u[k] + std::sin(p) * v[k]);
                wts[q] = wt;
                tot += wt;
            }
        }
        for (int q = 0; q < Q; ++q) wts[(size_t)d * Q + q] /= tot;
    }
    VIE_CUDA(cudaSetDevice(hd->device));
    const int R = hd->n_rhs;
    double *dd = nullptr, *dw = nullptr, *dp = nullptr, *dout = nullptr;
    cudaError_t e = cudaMalloc(&dd, sizeof(double) * dirs.size());
    if (e == cudaSuccess) e = cudaMalloc(&dw, sizeof(double) * wts.size());
    if (e == cudaSuccess) e = cudaMalloc(&dp, sizeof(double) * 6 * D);
    if (e == cudaSuccess) e = cudaMalloc(&dout, sizeof(double) * 2 * (size_t)D * R);
    if (e == cudaSuccess) e = cudaMemcpy(dd, dirs.data(), sizeof(double) * dirs.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dw, wts.data(), sizeof(double) * wts.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dp, pols, sizeof(double) * 6 * D, cudaMemcpyHostToDevice);
    int st = e == cudaSuccess ? VIE_OK : cuda_fail(e, "aperture buffers");
    if (st == VIE_OK) st = farfield_na(hd->op, hd->S.x, hd->S.n3, R, dd, dw, (const c64*)dp, D, Q, (c64*)dout);
    if (st == VIE_OK) {
        e = cudaMemcpy(out, dout, sizeof(double) * 2 * (size_t)D * R, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) st = cuda_fail(e, "aperture copy");
    }
    cudaFree(dd);
    cudaFree(dw);
    cudaFree(dp);
    cudaFree(dout);
    return st;
}

int vie_farfield_dirs(vie_handle* hd, const double* dirs, int D, int basis, double* out) {
    if (!hd || !dirs || !out || D < 1) return fail(VIE_EINVAL, "bad arguments");
    for (int d = 0; d < D; ++d) {
        const double n2 = dirs[3 * d] * dirs[3 * d] + dirs[3 * d + 1] * dirs[3 * d + 1] + dirs[3 * d + 2] * dirs[3 * d + 2];
        if (!(std::fabs(n2 - 1.0) < 1e-9)) return fail(VIE_EINVAL, "directions must be unit vectors");
    }
    if (!hd->have_solution) return fail(VIE_ESTATE, "no solution stored: call vie_solve first");
    VIE_CUDA(cudaSetDevice(hd->device));
    double* dd = nullptr;
    double* dout = nullptr;
    const size_t ob = sizeof(double) * 6 * (size_t)D * hd->n_rhs;
    VIE_CUDA(cudaMalloc(&dd, sizeof(double) * 3 * D));
    cudaError_t e = cudaMalloc(&dout, ob);
    int st = VIE_OK;
    if (e == cudaSuccess) e = cudaMemcpy(dd, dirs, sizeof(double) * 3 * D, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) st = cuda_fail(e, "far-field buffers");
    if (st == VIE_OK) st = farfield_dirs(hd->op, hd->S.x, hd->S.n3, hd->n_rhs, dd, D, basis, (c64*)dout);
    if (st == VIE_OK) {
        e = cudaMemcpy(out, dout, ob, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) st = cuda_fail(e, "far-field copy");
    }
    cudaFree(dd);
    cudaFree(dout);
    return st;
}

int vie_farfield(vie_handle* hd, const double* theta, int nt, const double* phi, int np, int basis, double* out) {
    if (!hd || !theta || !phi || !out || nt < 1 || np < 1) return fail(VIE_EINVAL, "bad arguments");
    if (basis < 0 || basis > 2) return fail(VIE_EINVAL, "basis must be 0, 1 or 2");
    for (int i = 0; i < nt; ++i)
        if (!std::isfinite(theta[i])) return fail(VIE_EINVAL, "theta must be finite");
    for (int i = 0; i < np; ++i)
        if (!std::isfinite(phi[i])) return fail(VIE_EINVAL, "phi must be finite");
    if (!hd->have_solution) return fail(VIE_ESTATE, "no solution stored: call vie_solve first");
    VIE_CUDA(cudaSetDevice(hd->device));
    double *dth = nullptr, *dph = nullptr, *dout = nullptr;
    const size_t ob = sizeof(double) * 6 * (size_t)nt * np * hd->n_rhs;
    int st = VIE_OK;
    cudaError_t e = cudaMalloc(&dth, sizeof(double) * nt);
    if (e == cudaSuccess) e = cudaMalloc(&dph, sizeof(double) * np);
    if (e == cudaSuccess) e = cudaMalloc(&dout, ob);
    if (e == cudaSuccess) e = cudaMemcpy(dth, theta, sizeof(double) * nt, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dph, phi, sizeof(double) * np, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) st = cuda_fail(e, "far-field buffers");
    if (st == VIE_OK) st = farfield_grid(hd->op, hd->S.x, hd->S.n3, hd->n_rhs, dth, nt, dph, np, basis, (c64*)dout);
    if (st == VIE_OK) {
        e = cudaMemcpy(out, dout, ob, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) st = cuda_fail(e, "far-field copy");
    }
    cudaFree(dth);
    cudaFree(dph);
    cudaFree(dout);
    return st;
}

int hom_transfer(const double E[8], const double omega[2], double sigma, const double* dtau, int n_tau, double* g2,
                 double* Nc, double* visibility) {
    if (!E || (n_tau > 0 && (!dtau || !Nc)) || n_tau < 0) return fail(VIE_EINVAL, "bad arguments");
    for (int i = 0; i < 8; ++i)
        if (!std::isfinite(E[i])) return fail(VIE_EINVAL, "amplitudes must be finite");
    const double w1 = omega ? omega[0] : 1.0, w2 = omega ? omega[1] : 1.0;
    if (!(w1 > 0) || !(w2 > 0)) return fail(VIE_EINVAL, "omega must be positive");
    if (n_tau > 0 && !(sigma > 0)) return fail(VIE_EINVAL, "sigma must be positive");
    const HomScalars s = hom_scalars(E, w1, w2);
    if (g2) *g2 = s.g2;
    for (int i = 0; i < n_tau; ++i) Nc[i] = hom_nc(s, dtau[i], sigma);
    if (visibility) *visibility = s.undefined_nc ? NAN : 1.0 - s.nc0;
    if (s.undefined_g2 || (s.undefined_nc && (n_tau > 0 || visibility)))
        return fail(VIE_EUNDEF, "g2 or N~c undefined: a channel is absent at the detectors (0/0)");
    return VIE_OK;
}

int vie_hom_map(const double* Ea, int nA, const double* Eb, int nB, double sigma, double* g2, double* vis,
                double* p2) {
    (void)sigma;
    if (!Ea || !Eb || nA < 1 || nB < 1) return fail(VIE_EINVAL, "bad arguments");
    const long long n = (long long)nA * nB;
    void *dA = nullptr, *dB = nullptr, *dg = nullptr, *dv = nullptr, *dp = nullptr;
    int st = VIE_OK;
    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&dA, sizeof(c64) * 2 * nA);
    if (e == cudaSuccess) e = cudaMalloc(&dB, sizeof(c64) * 2 * nB);
    if (e == cudaSuccess && g2) e = cudaMalloc(&dg, sizeof(double) * n);
    if (e == cudaSuccess && vis) e = cudaMalloc(&dv, sizeof(double) * n);
    if (e == cudaSuccess && p2) e = cudaMalloc(&dp, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMemcpy(dA, Ea, sizeof(c64) * 2 * nA, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dB, Eb, sizeof(c64) * 2 * nB, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) st = cuda_fail(e, "hom map buffers");
    if (st == VIE_OK) st = hom_map_device((const c64*)dA, nA, (const c64*)dB, nB, (double*)dg, (double*)dv,
                                          (double*)dp, s);
    if (st == VIE_OK) {
        e = cudaStreamSynchronize(s);
        if (e == cudaSuccess && g2) e = cudaMemcpy(g2, dg, sizeof(double) * n, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && vis) e = cudaMemcpy(vis, dv, sizeof(double) * n, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && p2) e = cudaMemcpy(p2, dp, sizeof(double) * n, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) st = cuda_fail(e, "hom map copy");
    }
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dg);
    cudaFree(dv);
    cudaFree(dp);
    if (s) cudaStreamDestroy(s);
    return st;
}

int vie_get_current(vie_handle* hd, int rhs, double* out) {
    if (!hd || !out) return fail(VIE_EINVAL, "NULL argument");
    if (!hd->have_solution) return fail(VIE_ESTATE, "no solution stored");
    if (rhs < 0 || rhs >= hd->n_rhs) return fail(VIE_EINVAL, "rhs index out of range");
    const long long Nb = hd->op.Nb, N = hd->op.N;
    std::vector<double> buf(6 * Nb);
    VIE_CUDA(cudaMemcpy(buf.data(), hd->S.x + rhs * hd->S.n3, sizeof(c64) * 3 * Nb, cudaMemcpyDeviceToHost));
    std::memset(out, 0, sizeof(double) * 6 * N);
    for (int c = 0; c < 3; ++c)
        for (long long v = 0; v < Nb; ++v) {
            const long long o = (c * N + hd->vox_host[v]) * 2;
            out[o] = buf[(c * Nb + v) * 2];
            out[o + 1] = buf[(c * Nb + v) * 2 + 1];
        }
    return VIE_OK;
}

int vie_apply_device(vie_handle* hd, const void* w_dev, void* y_dev, int n_rhs, int precision) {
    if (!hd || !w_dev || !y_dev || n_rhs < 1) return fail(VIE_EINVAL, "bad arguments");
    if (precision != VIE_PREC_MIXED && precision != VIE_PREC_FP64 && precision != VIE_PREC_F32X2)
        return fail(VIE_EINVAL, "bad precision");
    VIE_CUDA(cudaSetDevice(hd->device));
    std::vector<int> list(n_rhs);
    for (int r = 0; r < n_rhs; ++r) list[r] = r;
    VIE_TRY(op_set_list(hd->op, list.data(), n_rhs));
    const long long n3 = 3 * hd->op.Nb;
    return op_apply(hd->op, precision, w_dev, n3, y_dev, n3, hd->op.d_list, n_rhs);
}

int vie_apply(vie_handle* hd, const double* w, double* y, int n_rhs, int precision) {
    if (!hd || !w || !y || n_rhs < 1) return fail(VIE_EINVAL, "bad arguments");
    if (precision != VIE_PREC_MIXED && precision != VIE_PREC_FP64 && precision != VIE_PREC_F32X2)
        return fail(VIE_EINVAL, "bad precision");
    VIE_CUDA(cudaSetDevice(hd->device));
    const long long Nb = hd->op.Nb, N = hd->op.N, n3 = 3 * Nb;
    const bool io64 = precision != VIE_PREC_MIXED;  // FP64 and F32X2 take double vectors
    const size_t esz = io64 ? sizeof(c64) : sizeof(c32);
    std::vector<unsigned char> hbuf(esz * n3 * n_rhs);
    for (int r = 0; r < n_rhs; ++r)
        for (int c = 0; c < 3; ++c)
            for (long long v = 0; v < Nb; ++v) {
                const long long i = ((long long)r * 3 * N + c * N + hd->vox_host[v]) * 2;
                const long long o = (long long)r * n3 + c * Nb + v;
                if (io64) reinterpret_cast<c64*>(hbuf.data())[o] = c64{w[i], w[i + 1]};
                else reinterpret_cast<c32*>(hbuf.data())[o] = c32{(float)w[i], (float)w[i + 1]};
            }
    void *dw = nullptr, *dy = nullptr;
    VIE_CUDA(cudaMalloc(&dw, hbuf.size()));
    cudaError_t e = cudaMalloc(&dy, hbuf.size());
    int st = VIE_OK;
    if (e == cudaSuccess) e = cudaMemcpy(dw, hbuf.data(), hbuf.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) st = cuda_fail(e, "apply buffers");
    if (st == VIE_OK) st = vie_apply_device(hd, dw, dy, n_rhs, precision);
    if (st == VIE_OK) {
        e = cudaStreamSynchronize(hd->op.stream);
        if (e == cudaSuccess) e = cudaMemcpy(hbuf.data(), dy, hbuf.size(), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) st = cuda_fail(e, "apply");
    }
    cudaFree(dw);
    cudaFree(dy);
    if (st != VIE_OK) return st;
    std::memcpy(y, w, sizeof(double) * 2 * 3 * N * n_rhs);  // y = w outside the body
    for (int r = 0; r < n_rhs; ++r)
        for (int c = 0; c < 3; ++c)
            for (long long v = 0; v < Nb; ++v) {
                const long long i = ((long long)r * 3 * N + c * N + hd->vox_host[v]) * 2;
                const long long o = (long long)r * n3 + c * Nb + v;
                if (io64) {
                    const c64 a = reinterpret_cast<c64*>(hbuf.data())[o];
                    y[i] = a.x;
                    y[i + 1] = a.y;
                } else {
                    const c32 a = reinterpret_cast<c32*>(hbuf.data())[o];
                    y[i] = a.x;
                    y[i + 1] = a.y;
                }
            }
    return VIE_OK;
}

int vie_fft_lines(const double* in, double* out, int L, int count, int inverse, int precision) {
    if (!in || !out || L < 1 || count < 1) return fail(VIE_EINVAL, "bad arguments");
    const size_t n = (size_t)L * count;
    const size_t esz = precision == VIE_PREC_FP64 ? sizeof(c64) : sizeof(c32);
    std::vector<unsigned char> h(esz * n);
    for (size_t i = 0; i < n; ++i) {
        if (precision == VIE_PREC_FP64) reinterpret_cast<c64*>(h.data())[i] = c64{in[2 * i], in[2 * i + 1]};
        else reinterpret_cast<c32*>(h.data())[i] = c32{(float)in[2 * i], (float)in[2 * i + 1]};
    }
    void *di = nullptr, *dout = nullptr;
    VIE_CUDA(cudaMalloc(&di, h.size()));
    cudaError_t e = cudaMalloc(&dout, h.size());
    int st = VIE_OK;
    if (e == cudaSuccess) e = cudaMemcpy(di, h.data(), h.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) st = cuda_fail(e, "fft buffers");
    if (st == VIE_OK) st = fft_lines_device(di, dout, L, count, inverse, precision, 0);
    if (st == VIE_OK) {
        e = cudaMemcpy(h.data(), dout, h.size(), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) st = cuda_fail(e, "fft copy");
    }
    cudaFree(di);
    cudaFree(dout);
    if (st != VIE_OK) return st;
    for (size_t i = 0; i < n; ++i) {
        if (precision == VIE_PREC_FP64) {
            const c64 a = reinterpret_cast<c64*>(h.data())[i];
            out[2 * i] = a.x;
            out[2 * i + 1] = a.y;
        } else {
            const c32 a = reinterpret_cast<c32*>(h.data())[i];
            out[2 * i] = a.x;
            out[2 * i + 1] = a.y;
        }
    }
    return VIE_OK;
}

int vie_get_info(const vie_handle* hd, vie_info* info) {
    if (!hd || !info) return fail(VIE_EINVAL, "NULL argument");
    for (int a = 0; a < 3; ++a) {
        info->n[a] = hd->op.n[a];
        info->P[a] = hd->op.P[a];
    }
    info->n_body = hd->op.Nb;
    info->n_rhs = hd->n_rhs;
    info->device = hd->device;
    info->device_bytes = hd->op.bytes;
    return VIE_OK;
}

int vie_set_farfield_engine(vie_handle* hd, int engine) {
    if (!hd || (engine != 0 && engine != 1)) return fail(VIE_EINVAL, "far-field engine must be 0 or 1");
    hd->op.ff_engine = engine;
    return VIE_OK;
}

int vie_cgemm(int M, int N, int K, const double* A, const double* B, double* C, int engine) {
    if (!A || !B || !C || M < 1 || N < 1 || K < 1 || (engine != 0 && engine != 1))
        return fail(VIE_EINVAL, "bad arguments");
    std::vector<c32> a((size_t)M * K), b((size_t)K * N), c((size_t)M * N);
    for (size_t i = 0; i < a.size(); ++i) a[i] = c32{(float)A[2 * i], (float)A[2 * i + 1]};
    for (size_t i = 0; i < b.size(); ++i) b[i] = c32{(float)B[2 * i], (float)B[2 * i + 1]};
    c32 *da = nullptr, *db = nullptr, *dc = nullptr;
    int* derr = nullptr;
    int st = VIE_OK;
    cudaError_t e = cudaMalloc(&da, sizeof(c32) * a.size());
    if (e == cudaSuccess) e = cudaMalloc(&db, sizeof(c32) * b.size());
    if (e == cudaSuccess) e = cudaMalloc(&dc, sizeof(c32) * c.size());
    if (e == cudaSuccess) e = cudaMalloc(&derr, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(da, a.data(), sizeof(c32) * a.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(db, b.data(), sizeof(c32) * b.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(derr, 0, sizeof(int));
    if (e != cudaSuccess) st = cuda_fail(e, "gemm buffers");
    if (st == VIE_OK)
        st = engine == 0 ? tc_cgemm(M, N, K, 1, da, 0, K, 1, db, 0, N, 1, dc, 0, N, 1, derr, 0)
                         : cc_cgemm(M, N, K, 1, da, 0, K, 1, db, 0, N, 1, dc, 0, N, 1, 0);
    int herr = 0;
    if (st == VIE_OK) {
        e = cudaDeviceSynchronize();
        if (e == cudaSuccess) e = cudaMemcpy(c.data(), dc, sizeof(c32) * c.size(), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) st = cuda_fail(e, "gemm");
    }
    cudaFree(da);
    cudaFree(db);
    cudaFree(dc);
    cudaFree(derr);
    if (st != VIE_OK) return st;
    if (herr) return fail(VIE_ETIMEOUT, "tensor-core GEMM: a bounded wait on the MMA barrier gave up");
    for (size_t i = 0; i < c.size(); ++i) {
        C[2 * i] = c[i].x;
        C[2 * i + 1] = c[i].y;
    }
    return VIE_OK;
}

}  // extern "C"

namespace {
// deterministic test vectors for the autotuner's timed applications
__global__ void k_fill_test(vie::c32* w, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        unsigned long long z = (unsigned long long)i * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        w[i] = vie::c32{(float)((z & 0xFFFF) / 65536.0 - 0.5), (float)(((z >> 16) & 0xFFFF) / 65536.0 - 0.5)};
    }
}

// candidate padded lengths of an axis of n voxels: the default choice and the
// other of (next power of two >= 2n-1, smallest 2,3,5,7-smooth length)
std::vector<int> pad_candidates(int n, int disc) {
    const int need = disc ? 2 * n : 2 * n - 1;
    std::vector<int> c{vie::padded_len(need)};
    const int sm = vie::smooth_size(need);
    int p2 = 1;
    while (p2 < need) p2 *= 2;
    for (int v : {sm, p2})
        if (v != c[0] && v <= 1024 && v * 2 <= 5 * sm) c.push_back(v);
    return c;
}
}  // namespace

extern "C" {

int vie_autotune(vie_handle* hd, int n_rhs, int reps, int P_out[3], double* ms_per_apply) {
    if (!hd || n_rhs < 1 || reps < 1) return fail(VIE_EINVAL, "NULL handle, n_rhs < 1 or reps < 1");
    VIE_CUDA(cudaSetDevice(hd->device));
    Operator& op = hd->op;
    std::vector<int> cand[3];
    for (int a = 0; a < 3; ++a) cand[a] = pad_candidates(op.n[a], op.disc);
    std::vector<std::array<int, 4>> cands;  // P0, P1, P2, fft path
    const bool cubic = op.n[0] == op.n[1] && op.n[1] == op.n[2];
    for (int i0 = 0; i0 < (int)cand[0].size(); ++i0)
        for (int i1 = 0; i1 < (int)cand[1].size(); ++i1)
            for (int i2 = 0; i2 < (int)cand[2].size(); ++i2) {
                if (cubic && (i0 != i1 || i1 != i2)) continue;
                const int P[3] = {cand[0][i0], cand[1][i1], cand[2][i2]};
                const bool any_fast = fast_length(P[0]) || fast_length(P[1]) || fast_length(P[2]);
                for (int path = 0; path < (any_fast ? 2 : 1); ++path) cands.push_back({P[0], P[1], P[2], path});
            }
    const int P0[3] = {op.P[0], op.P[1], op.P[2]};
    const int path0 = op.fft_path;
    const long long nv = 3 * op.Nb;
    c32 *w = nullptr, *y = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int st = VIE_OK;
    cudaError_t ce = cudaMalloc(&w, sizeof(c32) * nv * n_rhs);
    if (ce == cudaSuccess) ce = cudaMalloc(&y, sizeof(c32) * nv * n_rhs);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) st = cuda_fail(ce, "autotune buffers");
    if (st == VIE_OK) {
        k_fill_test<<<1024, 256, 0, op.stream>>>(w, nv * n_rhs);
        count_launch();
        std::vector<int> lst(n_rhs);
        for (int i = 0; i < n_rhs; ++i) lst[i] = i;
        st = op_set_list(op, lst.data(), n_rhs);
    }
    double best = 1e300;
    int bi = -1;
    for (int c = 0; st == VIE_OK && c < (int)cands.size(); ++c) {
        const int P[3] = {cands[c][0], cands[c][1], cands[c][2]};
        if (P[0] != op.P[0] || P[1] != op.P[1] || P[2] != op.P[2]) st = op_replan(op, P);
        op.fft_path = cands[c][3];
        if (st == VIE_OK) st = op_apply(op, VIE_PREC_MIXED, w, nv, y, nv, op.d_list, n_rhs);  // warm-up
        if (st != VIE_OK) break;
        cudaEventRecord(e0, op.stream);
        for (int r = 0; st == VIE_OK && r < reps; ++r) st = op_apply(op, VIE_PREC_MIXED, w, nv, y, nv, op.d_list, n_rhs);
        cudaEventRecord(e1, op.stream);
        ce = cudaEventSynchronize(e1);
        if (ce != cudaSuccess) st = cuda_fail(ce, "autotune timing");
        float ms = 0.f;
        if (st == VIE_OK) cudaEventElapsedTime(&ms, e0, e1);
        if (st == VIE_OK && ms / reps < best) {
            best = ms / reps;
            bi = c;
        }
    }
    // keep the fastest configuration (or restore the original one on error)
    const int keep[3] = {bi >= 0 && st == VIE_OK ? cands[bi][0] : P0[0], bi >= 0 && st == VIE_OK ? cands[bi][1] : P0[1],
                         bi >= 0 && st == VIE_OK ? cands[bi][2] : P0[2]};
    const int st2 = (keep[0] != op.P[0] || keep[1] != op.P[1] || keep[2] != op.P[2]) ? op_replan(op, keep) : VIE_OK;
    op.fft_path = bi >= 0 && st == VIE_OK ? cands[bi][3] : path0;
    cudaFree(w);
    cudaFree(y);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st != VIE_OK) return st;
    if (st2 != VIE_OK) return st2;
    if (P_out)
        for (int a = 0; a < 3; ++a) P_out[a] = op.P[a];
    if (ms_per_apply) *ms_per_apply = best;
    return VIE_OK;
}

int vie_set_fft_path(vie_handle* hd, int path) {
    if (!hd || (path != 0 && path != 1)) return fail(VIE_EINVAL, "fft path must be 0 or 1");
    hd->op.fft_path = path;
    return VIE_OK;
}

void* vie_stream(vie_handle* hd) { return hd ? (void*)hd->op.stream : nullptr; }

void vie_destroy(vie_handle* hd) {
    if (!hd) return;
    cudaSetDevice(hd->device);
    if (hd->op.stream) cudaStreamSynchronize(hd->op.stream);
    hd->S.release(hd->op);
    hd->bpc.release(hd->op);
    op_free(hd->op);
    if (hd->op.stream) cudaStreamDestroy(hd->op.stream);
    delete hd;
}

// ---- block-Jacobi preconditioner -------------------------------------------
int vie_set_block_precond(vie_handle* hd, const int* cuts, const int ncuts[3], int inner_iters) {
    if (!hd || !ncuts || (!cuts && ncuts[0] + ncuts[1] + ncuts[2] > 0)) return fail(VIE_EINVAL, "NULL argument");
    VIE_CUDA(cudaSetDevice(hd->device));
    VIE_CUDA(cudaStreamSynchronize(hd->op.stream));
    static const int none = 0;
    return block_precond_setup(hd->op, hd->bpc, cuts ? cuts : &none, ncuts, inner_iters);
}

int vie_block_layout(const int n[3], const int* vox, long long n_body, const int* cuts, const int ncuts[3],
                     int box_out[3], int* blocks_out, int* map_out) {
    if (!n || !ncuts || !box_out || !blocks_out || (n_body > 0 && !vox) || n_body < 0 ||
        (!cuts && ncuts[0] + ncuts[1] + ncuts[2] > 0))
        return fail(VIE_EINVAL, "NULL or negative argument");
    static const int none = 0;
    std::vector<int> map;
    VIE_TRY(block_layout(n, vox, n_body, cuts ? cuts : &none, ncuts, box_out, blocks_out, map_out ? &map : nullptr));
    if (map_out) std::copy(map.begin(), map.end(), map_out);
    return VIE_OK;
}

int vie_block_apply_device(vie_handle* hd, const void* w_dev, void* y_dev) {
    if (!hd || !w_dev || !y_dev) return fail(VIE_EINVAL, "NULL argument");
    VIE_CUDA(cudaSetDevice(hd->device));
    return block_apply(hd->op, hd->bpc, (const c32*)w_dev, (c32*)y_dev);
}

// ---- learned initial guess ------------------------------------------------
int vie_net_create(const int channels[4], unsigned long long seed, int bf16, vie_net** out) {
    return vie_net_create_io(channels, NET_IN, seed, bf16, out);
}

int vie_net_create_io(const int channels[4], int cin, unsigned long long seed, int bf16, vie_net** out) {
    if (!out || !channels) return fail(VIE_EINVAL, "NULL argument");
    for (int i = 0; i < 4; ++i)
        if (channels[i] < 1 || channels[i] > 256) return fail(VIE_EINVAL, "channels must be in 1..256");
    if (cin < 1 || cin > 64) return fail(VIE_EINVAL, "input channels must be in 1..64");
    vie_net* n = new vie_net();
    int st = n->net.init(channels, seed, bf16 ? 1 : 0, cin);
    if (st != VIE_OK) {
        delete n;
        return st;
    }
    *out = n;
    return VIE_OK;
}

void vie_net_destroy(vie_net* n) { delete n; }

long long vie_net_num_params(const vie_net* n) { return n ? n->net.nparams : 0; }

int vie_net_set_tensor_cores(vie_net* n, int on) {
    if (!n) return fail(VIE_EINVAL, "NULL network");
    n->net.tc = on ? 1 : 0;
    return VIE_OK;
}

int vie_net_get_params(const vie_net* n, float* host) {
    if (!n || !host) return fail(VIE_EINVAL, "NULL argument");
    long long o = 0;
    for (int l = 0; l < Net::NL; ++l) {
        VIE_CUDA(cudaMemcpy(host + o, n->net.L[l].w, 4 * n->net.L[l].nw, cudaMemcpyDeviceToHost));
        o += n->net.L[l].nw;
        VIE_CUDA(cudaMemcpy(host + o, n->net.L[l].b, 4 * n->net.L[l].co, cudaMemcpyDeviceToHost));
        o += n->net.L[l].co;
    }
    return VIE_OK;
}

int vie_net_set_params(vie_net* n, const float* host) {
    if (!n || !host) return fail(VIE_EINVAL, "NULL argument");
    long long o = 0;
    for (int l = 0; l < Net::NL; ++l) {
        VIE_CUDA(cudaMemcpy(n->net.L[l].w, host + o, 4 * n->net.L[l].nw, cudaMemcpyHostToDevice));
        o += n->net.L[l].nw;
        VIE_CUDA(cudaMemcpy(n->net.L[l].b, host + o, 4 * n->net.L[l].co, cudaMemcpyHostToDevice));
        o += n->net.L[l].co;
    }
    return VIE_OK;
}

static int net_check(vie_net* n, int B, int D) {
    if (!n || B < 1 || D < 8 || D % 8 != 0 || D > 256) return fail(VIE_EINVAL, "bad network arguments (D % 8 == 0)");
    return VIE_OK;
}

int vie_net_forward(vie_net* n, const float* x_dev, float* y_dev, int B, int D) {
    VIE_TRY(net_check(n, B, D));
    if (!x_dev || !y_dev) return fail(VIE_EINVAL, "NULL argument");
    Net& net = n->net;
    VIE_TRY(net.reserve(B, D));
    VIE_TRY(net.set_input(x_dev, B, 0));
    VIE_TRY(net.forward(B, 0));
    VIE_TRY(net.get_output(y_dev, B, 0));
    VIE_CUDA(cudaStreamSynchronize(0));
    return VIE_OK;
}

static int net_fwd_bwd(vie_net* n, const float* x, const float* t, const float* m, int B, int D, float* loss) {
    VIE_TRY(net_check(n, B, D));
    if (!x || !t || !m) return fail(VIE_EINVAL, "NULL argument");
    Net& net = n->net;
    VIE_TRY(net.reserve(B, D));
    VIE_TRY(device_sum(m, (long long)B * D * D * D, &net.mask_sum, net.d_loss, 0));
    VIE_TRY(net.set_input(x, B, 0));
    VIE_TRY(net.forward(B, 0));
    VIE_TRY(net.loss_grad(t, m, B, 0, loss));
    VIE_TRY(net.backward(B, 0));
    return VIE_OK;
}

int vie_net_gradients(vie_net* n, const float* x_dev, const float* t_dev, const float* m_dev, int B, int D, float* loss,
                      float* grads_host) {
    VIE_TRY(net_fwd_bwd(n, x_dev, t_dev, m_dev, B, D, loss));
    VIE_CUDA(cudaStreamSynchronize(0));
    if (grads_host) {
        long long o = 0;
        for (int l = 0; l < Net::NL; ++l) {
            VIE_CUDA(cudaMemcpy(grads_host + o, n->net.L[l].gw, 4 * n->net.L[l].nw, cudaMemcpyDeviceToHost));
            o += n->net.L[l].nw;
            VIE_CUDA(cudaMemcpy(grads_host + o, n->net.L[l].gb, 4 * n->net.L[l].co, cudaMemcpyDeviceToHost));
            o += n->net.L[l].co;
        }
    }
    return VIE_OK;
}

int vie_net_train_step(vie_net* n, const float* x_dev, const float* t_dev, const float* m_dev, int B, int D, float lr,
                       float* loss) {
    if (!(lr > 0)) return fail(VIE_EINVAL, "learning rate must be positive");
    VIE_TRY(net_fwd_bwd(n, x_dev, t_dev, m_dev, B, D, loss));
    VIE_TRY(n->net.adam(lr, 0));
    VIE_CUDA(cudaStreamSynchronize(0));
    return VIE_OK;
}

int vie_net_features(vie_handle* hd, int factor, float* x_dev, float* t_dev, float* m_dev) {
    if (!hd || !x_dev) return fail(VIE_EINVAL, "NULL argument");
    if (hd->op.disc) return fail(VIE_EINVAL, "the learned parts are built for the D1 discretisation");
    if (!hd->have_solution && t_dev) return fail(VIE_ESTATE, "training targets need a solve first");
    const Operator& op = hd->op;
    if (factor < 1 || op.n[0] != op.n[1] || op.n[0] != op.n[2] || op.n[0] % factor != 0)
        return fail(VIE_EINVAL, "features need a cubic grid with n divisible by the factor");
    if (!hd->S.chans) return fail(VIE_ESTATE, "no right-hand sides yet: call vie_solve first");
    VIE_CUDA(cudaSetDevice(hd->device));
    VIE_TRY(net_features(hd->op, hd->S.chans, hd->S.R, factor, x_dev, t_dev ? hd->S.x : nullptr, hd->S.n3, t_dev,
                         m_dev, hd->op.stream));
    VIE_CUDA(cudaStreamSynchronize(hd->op.stream));
    return VIE_OK;
}

int vie_attach_net(vie_handle* hd, vie_net* n, int factor) {
    if (!hd) return fail(VIE_EINVAL, "NULL handle");
    if (n && hd->op.disc) return fail(VIE_EINVAL, "the learned parts are built for the D1 discretisation");
    if (n && factor < 1) return fail(VIE_EINVAL, "factor must be >= 1");
    if (n && n->net.cin != NET_IN) return fail(VIE_EINVAL, "the initial-guess network takes 10 input channels");
    hd->net = n;
    hd->net_factor = factor;
    return VIE_OK;
}

int vie_guesses_rejected(const vie_handle* hd) { return hd ? hd->guesses_rejected : 0; }

int vie_solve_many(vie_handle* const* hds, const vie_channel* const* ch, const int* n_rhs, int n_bodies,
                   const vie_solve_opts* opts, vie_solve_stats* stats, int max_threads) {
    if (!hds || !ch || !n_rhs || n_bodies < 1) return fail(VIE_EINVAL, "NULL argument or n_bodies < 1");
    if (tmr_enabled()) return fail(VIE_EINVAL, "disable the kernel timer for concurrent solves");
    for (int i = 0; i < n_bodies; ++i) {
        if (!hds[i] || !ch[i]) return fail(VIE_EINVAL, "NULL handle or channel list");
        for (int j = 0; j < i; ++j)
            if (hds[j] == hds[i]) return fail(VIE_EINVAL, "a handle appears twice (handles are not thread-safe)");
    }
    const int nt = std::max(1, std::min(max_threads > 0 ? max_threads : 8, n_bodies));
    std::vector<int> codes(n_bodies, VIE_OK);
    std::vector<std::string> msgs(n_bodies);
    std::atomic<int> next{0};
    auto worker = [&]() {
        for (int i = next++; i < n_bodies; i = next++) {
            codes[i] = vie_solve(hds[i], ch[i], n_rhs[i], opts, stats ? &stats[i] : nullptr);
            if (codes[i] != VIE_OK) msgs[i] = vie_last_error();
        }
    };
    std::vector<std::thread> pool;
    for (int t = 0; t < nt; ++t) pool.emplace_back(worker);
    for (std::thread& t : pool) t.join();
    // first hard error, else the first non-convergence
    int first = -1;
    for (int i = 0; i < n_bodies && first < 0; ++i)
        if (codes[i] != VIE_OK && codes[i] != VIE_ENOCONV) first = i;
    for (int i = 0; i < n_bodies && first < 0; ++i)
        if (codes[i] != VIE_OK) first = i;
    if (first < 0) return VIE_OK;
    return fail(codes[first], "body " + std::to_string(first) + ": " + msgs[first]);
}

int vie_attach_precond(vie_handle* hd, vie_net* n, int factor) {
    if (!hd) return fail(VIE_EINVAL, "NULL handle");
    if (n && hd->op.disc) return fail(VIE_EINVAL, "the learned parts are built for the D1 discretisation");
    if (n) {
        const Operator& op = hd->op;
        if (factor < 1 || op.n[0] != op.n[1] || op.n[0] != op.n[2] || op.n[0] % (8 * factor) != 0)
            return fail(VIE_EINVAL, "the preconditioner needs a cubic grid with n divisible by 8 x factor");
        if (n->net.cin != PRE_IN) return fail(VIE_EINVAL, "the preconditioner network takes 7 input channels");
    }
    hd->pctx.net = n ? &n->net : nullptr;
    hd->pctx.f = factor;
    return VIE_OK;
}

int vie_precond_pairs(vie_handle* hd, int factor, const void* v_dev, int n, float* x_dev, float* t_dev,
                      float* m_dev) {
    if (!hd || !v_dev || !x_dev || !t_dev || !m_dev || n < 1) return fail(VIE_EINVAL, "NULL argument or n < 1");
    if (hd->op.disc) return fail(VIE_EINVAL, "the learned parts are built for the D1 discretisation");
    Operator& op = hd->op;
    if (factor < 1 || op.n[0] != op.n[1] || op.n[0] != op.n[2] || op.n[0] % factor != 0)
        return fail(VIE_EINVAL, "pairs need a cubic grid with n divisible by the factor");
    VIE_CUDA(cudaSetDevice(hd->device));
    const long long nv = 3 * op.Nb;
    c32* u = nullptr;
    VIE_CUDA(cudaMalloc(&u, sizeof(c32) * nv * n));
    std::vector<int> lst(n);
    for (int i = 0; i < n; ++i) lst[i] = i;
    int st = op_set_list(op, lst.data(), n);
    if (st == VIE_OK) st = op_apply(op, VIE_PREC_MIXED, v_dev, nv, u, nv, op.d_list, n);
    if (st == VIE_OK) st = precond_pairs(op, factor, (const c32*)v_dev, n, u, x_dev, t_dev, m_dev, op.stream);
    cudaFree(u);
    return st;
}

}  // extern "C"
