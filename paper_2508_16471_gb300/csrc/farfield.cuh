// Far field and two-photon observables (see farfield.cu).
#pragma once

#include <math.h>

#include "krylov.cuh"

namespace vie {

// g2 (Eq. 10) and the N~c ingredients for one detector pair and channel pair.
// E[8] = complex [det][ch] interleaved: (a,1) (a,2) (b,1) (b,2).
struct HomScalars {
    double g2;        // Eq. 10 (NaN if a first-order correlation vanishes)
    double ad_re, ad_im, ae_re, ae_im;  // A_dir = T_a1 T_b2, A_ex = T_a2 T_b1
    double nc0;       // N~c(0)
    int undefined_g2; // G1_a G1_b = 0
    int undefined_nc; // |A_dir|^2 + |A_ex|^2 = 0
};

__host__ __device__ inline HomScalars hom_scalars(const double* E, double w1, double w2) {
    HomScalars s;
    const double q1 = sqrt(w1), q2 = sqrt(w2);
    // T_aj = sqrt(omega_j) E_aj
    const double a1r = q1 * E[0], a1i = q1 * E[1], a2r = q2 * E[2], a2i = q2 * E[3];
    const double b1r = q1 * E[4], b1i = q1 * E[5], b2r = q2 * E[6], b2i = q2 * E[7];
    s.ad_re = a1r * b2r - a1i * b2i;
    s.ad_im = a1r * b2i + a1i * b2r;
    s.ae_re = a2r * b1r - a2i * b1i;
    s.ae_im = a2r * b1i + a2i * b1r;
    const double sr = s.ad_re + s.ae_re, si = s.ad_im + s.ae_im;
    const double num = sr * sr + si * si;
    const double Ga = a1r * a1r + a1i * a1i + a2r * a2r + a2i * a2i;
    const double Gb = b1r * b1r + b1i * b1i + b2r * b2r + b2i * b2i;
    const double den = Ga * Gb;
    s.undefined_g2 = !(den > 0.0);
    s.g2 = s.undefined_g2 ? NAN : num / den;
    const double pd = s.ad_re * s.ad_re + s.ad_im * s.ad_im + s.ae_re * s.ae_re + s.ae_im * s.ae_im;
    s.undefined_nc = !(pd > 0.0);
    s.nc0 = s.undefined_nc ? NAN : num / pd;
    return s;
}

// N~c(dtau) = 1 + 2 Re(A_dir conj(A_ex)) exp(-dtau^2/sigma^2) / (|A_dir|^2 + |A_ex|^2)
__host__ __device__ inline double hom_nc(const HomScalars& s, double dtau, double sigma) {
    if (s.undefined_nc) return NAN;
    const double pd = s.ad_re * s.ad_re + s.ad_im * s.ad_im + s.ae_re * s.ae_re + s.ae_im * s.ae_im;
    const double cr = s.ad_re * s.ae_re + s.ad_im * s.ae_im;  // Re(A_dir conj(A_ex))
    return 1.0 + 2.0 * cr * exp(-dtau * dtau / (sigma * sigma)) / pd;
}

int farfield_dirs(Operator& op, const c64* x, long long n3, int R, const double* ddirs, int D, int basis, c64* dout);
// right-hand sides b[r] = chi E_inc(channel r) for r < n_rhs (rows n3 apart, components comp_stride(op) apart);
// chans_dev receives the 9 doubles of each channel
int build_rhs_rows(Operator& op, c64* b, long long n3, double* chans_dev, const vie_channel* chs, int n_rhs);
// finite aperture: out[r][d] = sum_q wq[d Q + q] pol_d . F_r(dirs[d Q + q]) (device arrays; F of D Q directions)
int farfield_na(Operator& op, const c64* x, long long n3, int R, const double* ddirs, const double* dw,
                const c64* dpol, int D, int Q, c64* dout);
int farfield_grid(Operator& op, const c64* x, long long n3, int R, const double* dth, int nt, const double* dph,
                  int np, int basis, c64* dout);
int hom_map_device(const c64* Ea, int nA, const c64* Eb, int nB, double* g2, double* vis, double* p2,
                   cudaStream_t s);

}  // namespace vie
