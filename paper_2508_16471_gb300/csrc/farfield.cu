// Right-hand sides, far-field projection (Eq. 25), detector components
// (Eq. Eproj, Eq. 30) and the two-photon observables (Eq. 10, Eqs. 18-22, 27).
//
// Far field F(rhat) = C (I - rhat rhat) S(rhat),  S = sum_v w_v e^{-i k0 rhat.r_v},
// C = kappa k0^2 h^3 / (4 pi).  The phase factorises over the grid axes,
// e^{-i k0 rhat.r} = ex(i) ey(j) ez(k), so
//   * an arbitrary direction list is summed directly in FP64 with per-block
//     1-D phase tables (two complex multiplies per voxel and direction);
//   * a (theta, phi) product grid is contracted axis by axis:
//       A[rc][x][y][t]   = sum_z W[rc][x][y][z] ez(t, z)          (depends on theta)
//       B[t][rc][x][p]   = sum_y A[rc][x][y][t] ey(t, p, y)
//       S[rc][t][p]      = sum_x B[t][rc][x][p] ex(t, p, x)
//     in FP32 with short (<= n) accumulations and FP64-computed phase tables.
#include <algorithm>
#include <cmath>
#include <vector>

#include "farfield.cuh"

namespace vie {

// ---------------------------------------------------------------------------
// right-hand sides (Eq. 24's right side in the w unknown: chi E_inc)
// ---------------------------------------------------------------------------
// D2 (chi_cs = Nb): component q sits at the +q face, h/2 beyond the cell centre,
// with its own face contrast chi[q Nb + v]
__global__ void k_rhs(c64* __restrict__ b, long long n3, const int* __restrict__ vox, const double* __restrict__ chi,
                      long long Nb, int n1, int n2, double h, double cx, double cy, double cz, double k0,
                      const double* __restrict__ ch, long long chi_cs, long long cst) {
    const int r = blockIdx.y;
    const double* c = ch + 9 * r;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < Nb;
         v += (long long)gridDim.x * blockDim.x) {
        const int lin = vox[v];
        const int k = lin % n2;
        const int j = (lin / n2) % n1;
        const int i = lin / (n1 * n2);
        const double px = cx + i * h, py = cy + j * h, pz = cz + k * h;
        const double ph0 = k0 * (c[0] * px + c[1] * py + c[2] * pz);
        for (int q = 0; q < 3; ++q) {
            const double ph = chi_cs ? ph0 + 0.5 * k0 * h * c[q] : ph0;
            double s, co;
            sincos(ph, &s, &co);
            const double x = chi[q * chi_cs + v];
            const double pr = c[3 + 2 * q], pi = c[4 + 2 * q];
            b[r * n3 + q * cst + v] = c64{x * (pr * co - pi * s), x * (pr * s + pi * co)};
        }
    }
}

int build_rhs_rows(Operator& op, c64* b, long long n3, double* chans_dev, const vie_channel* chs, int n_rhs) {
    std::vector<double> hc(9 * n_rhs);
    for (int r = 0; r < n_rhs; ++r) {
        for (int q = 0; q < 3; ++q) hc[9 * r + q] = chs[r].khat[q];
        for (int q = 0; q < 6; ++q) hc[9 * r + 3 + q] = chs[r].pol[q];
    }
    cudaError_t e = cudaMemcpyAsync(chans_dev, hc.data(), sizeof(double) * hc.size(), cudaMemcpyHostToDevice,
                                    op.stream);
    if (e == cudaSuccess) {
        const double cx = op.origin[0] - 0.5 * (op.n[0] - 1) * op.h;
        const double cy = op.origin[1] - 0.5 * (op.n[1] - 1) * op.h;
        const double cz = op.origin[2] - 0.5 * (op.n[2] - 1) * op.h;
        k_rhs<<<dim3(std::max(1, std::min(1024, ceil_div(op.Nb, 256))), n_rhs), 256, 0, op.stream>>>(
            b, n3, op.vox, op.chi64, op.Nb, op.n[1], op.n[2], op.h, cx, cy, cz, op.k0, chans_dev, op.chi_cs,
            comp_stride(op));
        count_launch();
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(op.stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "rhs build");
    return VIE_OK;
}

int build_rhs(Operator& op, Solver& S, const vie_channel* chs, int n_rhs) {
    std::vector<double> hc(9 * n_rhs);
    for (int r = 0; r < n_rhs; ++r) {
        for (int q = 0; q < 3; ++q) hc[9 * r + q] = chs[r].khat[q];
        for (int q = 0; q < 6; ++q) hc[9 * r + 3 + q] = chs[r].pol[q];
    }
    double* d = S.chans;
    cudaError_t e = cudaMemcpyAsync(d, hc.data(), sizeof(double) * hc.size(), cudaMemcpyHostToDevice, op.stream);
    if (e == cudaSuccess) {
        const double cx = op.origin[0] - 0.5 * (op.n[0] - 1) * op.h;
        const double cy = op.origin[1] - 0.5 * (op.n[1] - 1) * op.h;
        const double cz = op.origin[2] - 0.5 * (op.n[2] - 1) * op.h;
        k_rhs<<<dim3(std::max(1, std::min(1024, ceil_div(op.Nb, 256))), n_rhs), 256, 0, op.stream>>>(
            S.b, S.n3, op.vox, op.chi64, op.Nb, op.n[1], op.n[2], op.h, cx, cy, cz, op.k0, d, op.chi_cs,
            comp_stride(op));
        count_launch();
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(op.stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "rhs build");
    return VIE_OK;
}

// ---------------------------------------------------------------------------
// finite numerical aperture (Eq. NAfield): weighted sums of projected far fields
// ---------------------------------------------------------------------------
__global__ void k_na_reduce(const c64* __restrict__ F, const double* __restrict__ w, const c64* __restrict__ pol,
                            int D, int Q, c64* __restrict__ out) {
    // one warp per (detector, RHS)
    const int d = blockIdx.x, r = blockIdx.y;
    const c64 p0 = pol[3 * d], p1 = pol[3 * d + 1], p2 = pol[3 * d + 2];
    double ar = 0.0, ai = 0.0;
    for (int q = threadIdx.x; q < Q; q += 32) {
        const c64* f = F + ((long long)r * D * Q + (long long)d * Q + q) * 3;
        const c64 e = p0 * f[0] + p1 * f[1] + p2 * f[2];
        const double ww = w[(long long)d * Q + q];
        ar += ww * e.x;
        ai += ww * e.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        ar += __shfl_xor_sync(0xffffffffu, ar, o);
        ai += __shfl_xor_sync(0xffffffffu, ai, o);
    }
    if (threadIdx.x == 0) out[(long long)r * D + d] = c64{ar, ai};
}

int farfield_na(Operator& op, const c64* x, long long n3, int R, const double* ddirs, const double* dw,
                const c64* dpol, int D, int Q, c64* dout) {
    c64* F = nullptr;
    VIE_CUDA(cudaMalloc(&F, sizeof(c64) * 3 * (size_t)D * Q * R));
    int st = farfield_dirs(op, x, n3, R, ddirs, D * Q, VIE_BASIS_CART, F);
    if (st == VIE_OK) {
        k_na_reduce<<<dim3(D, R), 32, 0, op.stream>>>(F, dw, dpol, D, Q, dout);
        count_launch();
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(op.stream);
        if (e != cudaSuccess) st = cuda_fail(e, "finite-aperture reduction");
    }
    cudaFree(F);
    return st;
}

// ---------------------------------------------------------------------------
// far field on a direction list (FP64)
// ---------------------------------------------------------------------------
constexpr int FF_DB = 2;  // directions per block

// Sraw[r][d][3] = sum_v w[r][c][v] e^{-i k0 d.r_v}
__global__ void k_ff_dirs(const c64* __restrict__ x, long long n3, const int* __restrict__ vox, long long Nb, int n0,
                          int n1, int n2, double h, double cx, double cy, double cz, double k0,
                          const double* __restrict__ dirs, int D, c64* __restrict__ Sraw, long long cst) {
    extern __shared__ __align__(16) unsigned char smraw[];
    c64* tab = reinterpret_cast<c64*>(smraw);  // [FF_DB][n0 + n1 + n2]
    const int nt = n0 + n1 + n2;
    const int r = blockIdx.y;
    const int d0 = blockIdx.x * FF_DB;
    for (int e = threadIdx.x; e < FF_DB * nt; e += blockDim.x) {
        const int q = e / nt, a = e - q * nt;
        const int d = min(d0 + q, D - 1);
        double coord, dc;
        if (a < n0) {
            coord = cx + a * h;
            dc = dirs[3 * d + 0];
        } else if (a < n0 + n1) {
            coord = cy + (a - n0) * h;
            dc = dirs[3 * d + 1];
        } else {
            coord = cz + (a - n0 - n1) * h;
            dc = dirs[3 * d + 2];
        }
        double s, c;
        sincos(-k0 * dc * coord, &s, &c);
        tab[e] = c64{c, s};
    }
    __syncthreads();
    double acc[FF_DB][3][2];
#pragma unroll
    for (int q = 0; q < FF_DB; ++q)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[q][c][0] = acc[q][c][1] = 0.0;
    const c64* xr = x + r * n3;
    for (long long v = threadIdx.x; v < Nb; v += blockDim.x) {
        const int lin = vox[v];
        const int k = lin % n2;
        const int j = (lin / n2) % n1;
        const int i = lin / (n1 * n2);
        const c64 w0 = xr[v], w1 = xr[cst + v], w2 = xr[2 * cst + v];
#pragma unroll
        for (int q = 0; q < FF_DB; ++q) {
            const c64* t = tab + q * nt;
            const c64 ph = t[i] * t[n0 + j] * t[n0 + n1 + k];
            const c64 p0 = ph * w0, p1 = ph * w1, p2 = ph * w2;
            acc[q][0][0] += p0.x;
            acc[q][0][1] += p0.y;
            acc[q][1][0] += p1.x;
            acc[q][1][1] += p1.y;
            acc[q][2][0] += p2.x;
            acc[q][2][1] += p2.y;
        }
    }
    __shared__ double red[32][FF_DB * 6];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < FF_DB; ++q)
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                double v = acc[q][c][u];
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) red[wid][q * 6 + c * 2 + u] = v;
            }
    __syncthreads();
    if (threadIdx.x < FF_DB * 6) {
        double t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w][threadIdx.x];
        const int q = threadIdx.x / 6, c = (threadIdx.x / 2) % 3, u = threadIdx.x & 1;
        const int d = d0 + q;
        if (d < D) reinterpret_cast<double*>(Sraw)[((long long)r * D + d) * 6 + c * 2 + u] = t;
    }
}

// out[r][d][3] = basis components of C (I - dd) S
// half_kh = k0 h / 2 for D2: component c of the sums sits at the +c faces and
// takes the extra phase e^{-i k0 rhat_c h/2}; 0 for D1
__global__ void k_ff_project(const c64* __restrict__ Sraw, const double* __restrict__ dirs, int D, int R,
                             double C, int basis, c64* __restrict__ out, double half_kh) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)D * R) return;
    const int d = (int)(i % D);
    const double dx = dirs[3 * d], dy = dirs[3 * d + 1], dz = dirs[3 * d + 2];
    c64 s[3] = {Sraw[i * 3], Sraw[i * 3 + 1], Sraw[i * 3 + 2]};
    if (half_kh != 0.0) {
        const double dd[3] = {dx, dy, dz};
        for (int q = 0; q < 3; ++q) {
            double sn, cs;
            sincos(-half_kh * dd[q], &sn, &cs);
            s[q] = c64{s[q].x * cs - s[q].y * sn, s[q].x * sn + s[q].y * cs};
        }
    }
    const c64 ds = {dx * s[0].x + dy * s[1].x + dz * s[2].x, dx * s[0].y + dy * s[1].y + dz * s[2].y};
    c64 F[3] = {{C * (s[0].x - dx * ds.x), C * (s[0].y - dx * ds.y)},
                {C * (s[1].x - dy * ds.x), C * (s[1].y - dy * ds.y)},
                {C * (s[2].x - dz * ds.x), C * (s[2].y - dz * ds.y)}};
    c64* o = out + i * 3;
    if (basis == VIE_BASIS_CART) {
        o[0] = F[0];
        o[1] = F[1];
        o[2] = F[2];
        return;
    }
    const double th = acos(fmin(1.0, fmax(-1.0, dz)));
    const double ph = atan2(dy, dx);
    double st, ct, sp, cp;
    sincos(th, &st, &ct);
    sincos(ph, &sp, &cp);
    const double et[3] = {ct * cp, ct * sp, -st}, ep[3] = {-sp, cp, 0.0};
    const c64 Ft = {et[0] * F[0].x + et[1] * F[1].x + et[2] * F[2].x, et[0] * F[0].y + et[1] * F[1].y + et[2] * F[2].y};
    const c64 Fp = {ep[0] * F[0].x + ep[1] * F[1].x, ep[0] * F[0].y + ep[1] * F[1].y};
    const c64 Fr = {dx * F[0].x + dy * F[1].x + dz * F[2].x, dx * F[0].y + dy * F[1].y + dz * F[2].y};
    if (basis == VIE_BASIS_SPH) {
        o[0] = Ft;
        o[1] = Fp;
        o[2] = Fr;
    } else {
        const double s2 = 0.70710678118654752440;
        o[0] = c64{s2 * (Ft.x - Fp.y), s2 * (Ft.y + Fp.x)};  // (Ft + i Fp)/sqrt2
        o[1] = c64{s2 * (Ft.x + Fp.y), s2 * (Ft.y - Fp.x)};  // (Ft - i Fp)/sqrt2
        o[2] = Fr;
    }
}

static double ff_constant(const Operator& op) {
    const double a = op.h * std::cbrt(3.0 / (4.0 * M_PI));
    const double ka = op.k0 * a;
    double kap;
    if (ka < 1e-3) kap = 1.0 - ka * ka / 10.0 + ka * ka * ka * ka / 280.0;
    else kap = 3.0 * (std::sin(ka) - ka * std::cos(ka)) / (ka * ka * ka);
    return kap * op.k0 * op.k0 * op.h * op.h * op.h / (4.0 * M_PI);
}

int farfield_dirs(Operator& op, const c64* x, long long n3, int R, const double* ddirs, int D, int basis,
                  c64* dout) {
    c64* Sraw = nullptr;
    VIE_CUDA(cudaMalloc(&Sraw, sizeof(c64) * 3 * (size_t)D * R));
    const double cx = op.origin[0] - 0.5 * (op.n[0] - 1) * op.h;
    const double cy = op.origin[1] - 0.5 * (op.n[1] - 1) * op.h;
    const double cz = op.origin[2] - 0.5 * (op.n[2] - 1) * op.h;
    const size_t sm = sizeof(c64) * FF_DB * (op.n[0] + op.n[1] + op.n[2]);
    cudaFuncSetAttribute(k_ff_dirs, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    k_ff_dirs<<<dim3(ceil_div(D, FF_DB), R), 256, sm, op.stream>>>(x, n3, op.vox, op.Nb, op.n[0], op.n[1], op.n[2],
                                                                   op.h, cx, cy, cz, op.k0, ddirs, D, Sraw,
                                                                   comp_stride(op));
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        k_ff_project<<<ceil_div((long long)D * R, 256), 256, 0, op.stream>>>(Sraw, ddirs, D, R, ff_constant(op), basis,
                                                                             dout, op.disc ? 0.5 * op.k0 * op.h : 0.0);
        count_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(op.stream);
    cudaFree(Sraw);
    if (e != cudaSuccess) return cuda_fail(e, "far field (directions)");
    return VIE_OK;
}

// ---------------------------------------------------------------------------
// far field on a (theta, phi) product grid: separable contraction (FP32)
// ---------------------------------------------------------------------------
// full-grid FP32 copy of the currents: W[r][c][x][y][z]
__global__ void k_scatter_full(const c64* __restrict__ x, long long n3, const int* __restrict__ vox, long long Nb,
                               long long N, c32* __restrict__ W, long long cst) {
    const int rc = blockIdx.y;  // r*3 + c
    const int r = rc / 3, c = rc % 3;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < Nb;
         v += (long long)gridDim.x * blockDim.x) {
        const c64 a = x[r * n3 + c * cst + v];
        W[(long long)rc * N + vox[v]] = c32{(float)a.x, (float)a.y};
    }
}

// Batched complex GEMM C[b](m,n) = sum_k A[b](m,k) B[b](k,n), FP32, generic strides.
constexpr int GT = 32;  // tile
__global__ void k_cgemm(int M, int N, int K, const c32* __restrict__ A, long long sAb, long long sAm, long long sAk,
                        const c32* __restrict__ B, long long sBb, long long sBk, long long sBn, c32* __restrict__ C,
                        long long sCb, long long sCm, long long sCn) {
    __shared__ c32 As[GT][GT + 1];
    __shared__ c32 Bs[GT][GT + 1];
    const int bz = blockIdx.z;
    const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 16 x 16 threads, 2x2 outputs each
    A += bz * sAb;
    B += bz * sBb;
    C += bz * sCb;
    float acc[2][2][2] = {};
    for (int k0 = 0; k0 < K; k0 += GT) {
        for (int e = threadIdx.x; e < GT * GT; e += 256) {
            const int i = e / GT, kk = e % GT;
            const int m = m0 + i, k = k0 + kk;
            As[i][kk] = (m < M && k < K) ? A[m * sAm + k * sAk] : c32{0.f, 0.f};
            const int k2 = k0 + i, n = n0 + kk;
            Bs[i][kk] = (k2 < K && n < N) ? B[k2 * sBk + n * sBn] : c32{0.f, 0.f};
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < GT; ++kk) {
            c32 a0 = As[ty * 2][kk], a1 = As[ty * 2 + 1][kk];
            c32 b0 = Bs[kk][tx * 2], b1 = Bs[kk][tx * 2 + 1];
            const c32 av[2] = {a0, a1}, bv[2] = {b0, b1};
#pragma unroll
            for (int p = 0; p < 2; ++p)
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    acc[p][q][0] += av[p].x * bv[q].x - av[p].y * bv[q].y;
                    acc[p][q][1] += av[p].x * bv[q].y + av[p].y * bv[q].x;
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int m = m0 + ty * 2 + p, n = n0 + tx * 2 + q;
            if (m < M && n < N) C[m * sCm + n * sCn] = c32{acc[p][q][0], acc[p][q][1]};
        }
}

int cc_cgemm(int M, int N, int K, int batch, const c32* A, long long sAb, long long sAm, long long sAk, const c32* B,
             long long sBb, long long sBk, long long sBn, c32* C, long long sCb, long long sCm, long long sCn,
             cudaStream_t s) {
    if (M <= 0 || N <= 0 || K <= 0 || batch <= 0) return VIE_OK;
    dim3 g(ceil_div(N, GT), ceil_div(M, GT), batch);
    k_cgemm<<<g, 256, 0, s>>>(M, N, K, A, sAb, sAm, sAk, B, sBb, sBk, sBn, C, sCb, sCm, sCn);
    count_launch();
    VIE_CUDA(cudaGetLastError());
    return VIE_OK;
}

// phase tables: ez[t][z] = e^{-i k0 cos(th_t) z}, ey[t][p][y] = e^{-i k0 sin th sin ph y},
// ex[t][p][x] = e^{-i k0 sin th cos ph x}
// Phase factors exp(-i k0 d_a (c_a + j h)) of the separable far-field sum, per
// (theta) for z and per (theta, phi) for y and x.  The phase is formed in FP64
// and reduced to [-pi, pi] in FP64 (so that its FP32 rounding costs at most
// 2e-7 rad whatever the box size); the factor is then taken in FP32, the
// precision of the tables.
// trig[0..nt) = cos theta, [nt..2nt) = sin theta, then sin phi and cos phi (np each)
__global__ void k_trig_tables(const double* __restrict__ th, int nt, const double* __restrict__ ph, int np,
                              double* __restrict__ trig) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nt) sincos(th[i], &trig[nt + i], &trig[i]);
    else if (i < nt + np) sincos(ph[i - nt], &trig[2 * nt + i - nt], &trig[2 * nt + np + i - nt]);
}

__global__ void k_phase_tables(const double* __restrict__ trig, int nt, int np, int n0, int n1, int n2, double h,
                               double cx, double cy, double cz, double k0, c32* ez, c32* ey, c32* ex) {
    const double* cth = trig;
    const double* sth = trig + nt;
    const double* sph = trig + 2 * nt;
    const double* cph = trig + 2 * nt + np;
    const long long totz = (long long)nt * n2, toty = (long long)nt * np * n1, totx = (long long)nt * np * n0;
    constexpr double TWO_PI = 6.283185307179586;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < totz + toty + totx;
         i += (long long)gridDim.x * blockDim.x) {
        double arg;
        c32* out;
        if (i < totz) {
            const int t = (int)(i / n2), z = (int)(i % n2);
            arg = -k0 * cth[t] * (cz + z * h);
            out = ez + i;
        } else if (i < totz + toty) {
            const long long q = i - totz;
            const int y = (int)(q % n1);
            const int p = (int)((q / n1) % np);
            const int t = (int)(q / ((long long)n1 * np));
            arg = -k0 * sth[t] * sph[p] * (cy + y * h);
            out = ey + q;
        } else {
            const long long q = i - totz - toty;
            const int x = (int)(q % n0);
            const int p = (int)((q / n0) % np);
            const int t = (int)(q / ((long long)n0 * np));
            arg = -k0 * sth[t] * cph[p] * (cx + x * h);
            out = ex + q;
        }
        const float r = (float)(arg - TWO_PI * rint(arg / TWO_PI));
        float sn, cs;
        sincosf(r, &sn, &cs);
        *out = c32{cs, sn};
    }
}

// S[rc][t][p] = sum_x Bt[t][p][rc*n0 + x] ex[t][p][x]; then projection.  One
// warp per output: its lanes read consecutive x (coalesced) and reduce.
__global__ void k_ff_xreduce(const c32* __restrict__ Bt, const c32* __restrict__ ex, int nt, int np, int n0, int RC,
                             c64* __restrict__ Sraw /* [R][nt*np][3] */) {
    const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const long long tot = (long long)nt * np * RC;
    if (w >= tot) return;
    const int rc = (int)(w % RC);
    const long long tp = w / RC;  // t * np + p
    const c32* e = ex + tp * n0;
    const c32* b = Bt + tp * RC * n0 + (long long)rc * n0;
    float ar = 0.f, ai = 0.f;
    for (int x = lane; x < n0; x += 32) {
        const c32 bv = b[x];
        const c32 ev = e[x];
        ar += bv.x * ev.x - bv.y * ev.y;
        ai += bv.x * ev.y + bv.y * ev.x;
    }
    for (int o = 16; o > 0; o >>= 1) {
        ar += __shfl_xor_sync(0xffffffffu, ar, o);
        ai += __shfl_xor_sync(0xffffffffu, ai, o);
    }
    if (lane == 0) {
        const int t = (int)(tp / np), p = (int)(tp % np);
        const int r = rc / 3, c = rc % 3;
        Sraw[(((long long)r * nt + t) * np + p) * 3 + c] = c64{ar, ai};
    }
}

__global__ void k_grid_dirs(const double* __restrict__ th, int nt, const double* __restrict__ ph, int np,
                            double* __restrict__ dirs) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt * np) return;
    const int t = i / np, p = i % np;
    double st, ct, sp, cp;
    sincos(th[t], &st, &ct);
    sincos(ph[p], &sp, &cp);
    dirs[3 * i] = st * cp;
    dirs[3 * i + 1] = st * sp;
    dirs[3 * i + 2] = ct;
}

int farfield_grid(Operator& op, const c64* x, long long n3, int R, const double* dth, int nt, const double* dph,
                  int np, int basis, c64* dout) {
    const int n0 = op.n[0], n1 = op.n[1], n2 = op.n[2];
    const long long N = op.N;
    const int RC = 3 * R;
    // one workspace per operator, grown to the largest request and kept
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return o;
    };
    const size_t oW = carve(sizeof(c32) * N * RC);
    const size_t oz = carve(sizeof(c32) * (size_t)nt * n2);
    const size_t oy = carve(sizeof(c32) * (size_t)nt * np * n1);
    const size_t ox = carve(sizeof(c32) * (size_t)nt * np * n0);
    const size_t oA = carve(sizeof(c32) * (size_t)RC * n0 * n1 * nt);
    const size_t oB = carve(sizeof(c32) * (size_t)nt * RC * n0 * np);
    const size_t oS = carve(sizeof(c64) * 3 * (size_t)R * nt * np);
    const size_t od = carve(sizeof(double) * 3 * (size_t)nt * np);
    const size_t ot = carve(sizeof(double) * 2 * (size_t)(nt + np));
    const size_t oe = carve(sizeof(int));
    if (op.ff_ws_bytes < off) {
        if (op.ff_ws) dev_free(op, op.ff_ws, op.ff_ws_bytes);
        op.ff_ws = nullptr;
        op.ff_ws_bytes = 0;
        VIE_TRY(dev_alloc(op, &op.ff_ws, off));
        op.ff_ws_bytes = off;
    }
    char* ws = (char*)op.ff_ws;
    c32* W = (c32*)(ws + oW);
    c32* ez = (c32*)(ws + oz);
    c32* ey = (c32*)(ws + oy);
    c32* ex = (c32*)(ws + ox);
    c32* A = (c32*)(ws + oA);
    c32* Bt = (c32*)(ws + oB);
    c64* Sraw = (c64*)(ws + oS);
    double* dirs = (double*)(ws + od);
    double* trig = (double*)(ws + ot);
    int* derr = (int*)(ws + oe);
    cudaStream_t s = op.stream;
    const double cx = op.origin[0] - 0.5 * (n0 - 1) * op.h;
    const double cy = op.origin[1] - 0.5 * (n1 - 1) * op.h;
    const double cz = op.origin[2] - 0.5 * (n2 - 1) * op.h;
    tmr_begin(TMR_FFOTHER, s);
    cudaMemsetAsync(W, 0, sizeof(c32) * N * RC, s);
    k_scatter_full<<<dim3(std::max(1, std::min(2048, ceil_div(op.Nb, 256))), RC), 256, 0, s>>>(x, n3, op.vox, op.Nb,
                                                                                               N, W, comp_stride(op));
    k_trig_tables<<<ceil_div(nt + np, 256), 256, 0, s>>>(dth, nt, dph, np, trig);
    k_phase_tables<<<1024, 256, 0, s>>>(trig, nt, np, n0, n1, n2, op.h, cx, cy, cz, op.k0, ez, ey, ex);
    cudaMemsetAsync(derr, 0, sizeof(int), s);
    tmr_end(TMR_FFOTHER, s, 0.0);
    int st = VIE_OK;
    tmr_begin(TMR_FFGEMM, s);
    // Intermediates are laid out with the row index m fastest, so that the
    // GEMM epilogues (one thread per row) store coalesced and the next
    // contraction reads its K index contiguously.
    // stage A: M = RC*n0*n1 rows (rc, x, y), K = n2, N = nt; A[t][m]
    const int MA = RC * n0 * n1;
    {
        st = op.ff_engine == 0 ? tc_cgemm(MA, nt, n2, 1, W, 0, n2, 1, ez, 0, 1, n2, A, 0, 1, MA, derr, s)
                               : cc_cgemm(MA, nt, n2, 1, W, 0, n2, 1, ez, 0, 1, n2, A, 0, 1, MA, s);
    }
    // stage B: per t: M = RC*n0 rows (rc, x), K = n1 (y, contiguous in A[t]), N = np; Bt[t][p][m]
    if (st == VIE_OK) {
        const int M = RC * n0;
        st = op.ff_engine == 0
                 ? tc_cgemm(M, np, n1, nt, A, MA, n1, 1, ey, (long long)np * n1, 1, n1, Bt, (long long)M * np, 1, M,
                            derr, s)
                 : cc_cgemm(M, np, n1, nt, A, MA, n1, 1, ey, (long long)np * n1, 1, n1, Bt, (long long)M * np, 1, M,
                            s);
    }
    tmr_end(TMR_FFGEMM, s, 0.0);
    if (st != VIE_OK) return st;
    tmr_begin(TMR_FFOTHER, s);
    k_ff_xreduce<<<ceil_div((long long)nt * np * RC * 32, 256), 256, 0, s>>>(Bt, ex, nt, np, n0, RC, Sraw);
    k_grid_dirs<<<ceil_div(nt * np, 256), 256, 0, s>>>(dth, nt, dph, np, dirs);
    k_ff_project<<<ceil_div((long long)nt * np * R, 256), 256, 0, s>>>(Sraw, dirs, nt * np, R, ff_constant(op), basis,
                                                                       dout, op.disc ? 0.5 * op.k0 * op.h : 0.0);
    tmr_end(TMR_FFOTHER, s, 0.0);
    count_launch(6);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "far field (grid)");
    if (herr) return fail(VIE_ETIMEOUT, "tensor-core GEMM: a bounded wait on the MMA barrier gave up");
    return VIE_OK;
}

// ---------------------------------------------------------------------------
// two-photon observables
// ---------------------------------------------------------------------------
__global__ void k_hom_map(const c64* __restrict__ Ea, int nA, const c64* __restrict__ Eb, int nB, double* g2,
                          double* vis, double* p2) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)nA * nB) return;
    const int ia = (int)(i / nB), ib = (int)(i % nB);
    double E[8];
    const c64 a1 = Ea[ia], a2 = Ea[nA + ia], b1 = Eb[ib], b2 = Eb[nB + ib];
    E[0] = a1.x;
    E[1] = a1.y;
    E[2] = a2.x;
    E[3] = a2.y;
    E[4] = b1.x;
    E[5] = b1.y;
    E[6] = b2.x;
    E[7] = b2.y;
    HomScalars s = hom_scalars(E, 1.0, 1.0);
    if (g2) g2[i] = s.g2;
    if (vis) vis[i] = s.undefined_nc ? nan("") : 1.0 - s.nc0;
    if (p2) {
        const double Ia = (a1.x + a2.x) * (a1.x + a2.x) + (a1.y + a2.y) * (a1.y + a2.y);
        const double Ib = (b1.x + b2.x) * (b1.x + b2.x) + (b1.y + b2.y) * (b1.y + b2.y);
        p2[i] = Ia * Ib;
    }
}

__global__ void k_max(const double* __restrict__ v, long long n, unsigned long long* __restrict__ out) {
    double m = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        m = fmax(m, v[i]);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

__global__ void k_scale_by(double* __restrict__ v, long long n, const unsigned long long* __restrict__ mx) {
    const double m = __longlong_as_double((long long)*mx);
    const double s = m > 0 ? 1.0 / m : 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        v[i] *= s;
}

int hom_map_device(const c64* Ea, int nA, const c64* Eb, int nB, double* g2, double* vis, double* p2,
                   cudaStream_t s) {
    const long long n = (long long)nA * nB;
    k_hom_map<<<ceil_div(n, 256), 256, 0, s>>>(Ea, nA, Eb, nB, g2, vis, p2);
    count_launch();
    VIE_CUDA(cudaGetLastError());
    if (p2) {
        unsigned long long* mx = nullptr;
        VIE_CUDA(cudaMalloc(&mx, sizeof(unsigned long long)));
        cudaMemsetAsync(mx, 0, sizeof(unsigned long long), s);
        k_max<<<std::max(1, std::min(1024, ceil_div(n, 256))), 256, 0, s>>>(p2, n, mx);
        k_scale_by<<<std::max(1, std::min(1024, ceil_div(n, 256))), 256, 0, s>>>(p2, n, mx);
        count_launch(2);
        cudaError_t e = cudaStreamSynchronize(s);
        cudaFree(mx);
        if (e != cudaSuccess) return cuda_fail(e, "hom map");
    }
    return VIE_OK;
}

}  // namespace vie
