/*
 * vie.h -- C ABI of the GB300 FFT-VIE library (libvie.so).
 *
 * Computes, for a lossless dielectric body on a uniform voxel grid, the
 * contrast current of every incident plane-wave channel by solving the volume
 * integral equation (arXiv 2508.16471, Sec. II-C, Eq. 24) with FFT-accelerated
 * matrix-vector products, projects the currents onto far-field amplitudes
 * (Eq. 25, Eq. Eproj, Eq. 30) and forms the two-photon observables g2
 * (Eq. 10), N~c(dtau) and the HOM visibility (Eqs. 18-22).
 *
 * Discretisation.  The unknown is the contrast current w = chi E_tot with
 * chi = eps_r - 1 (Eq. Js_def: J = -i omega eps0 w).  On every body voxel n
 *     w_n - chi_n sum_m K(n - m) w_m = chi_n E_inc(r_n)
 * where each source voxel is the ball of volume h^3 (radius a), tested at
 * voxel centres:  K(m != 0) = kappa k0^2 h^3 G(m h) with the dyadic Green's
 * function G of Eq. dyadicG and kappa = 3 (sin ka - ka cos ka)/(ka)^3;
 * K(0) = [2/3((1 - i ka) e^{i ka} - 1) - 1/3] I.  The far field is
 *     F(rhat) = kappa k0^2 h^3/(4 pi) (I - rhat rhat) sum_n w_n e^{-i k0 rhat.r_n}
 * with E_sca ~ F e^{i k0 r}/r, time convention e^{-i omega t}.
 *
 * Conventions shared by every entry point:
 *   - Grid arrays are C-ordered [i][j][k] over (x, y, z), z fastest.  Voxel
 *     (i,j,k) is centred at origin + ((i,j,k) - (n-1)/2) h.
 *   - Complex numbers are interleaved (re, im) doubles unless stated.
 *   - Host pointers are owned by the caller; the library copies from/to them.
 *     Device pointers ("_device" entry points) must point to memory of the
 *     device that was current at vie_setup; they are never freed by the
 *     library.  All device memory of a handle is owned by the handle and
 *     released by vie_destroy.
 *   - A handle is not thread-safe; use one handle per host thread / stream.
 *   - Every int-returning function returns VIE_OK (0) or a negative status;
 *     vie_last_error() then describes the failure (thread-local string).
 */
#ifndef VIE_H
#define VIE_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define VIE_OK        0
#define VIE_EINVAL   -1  /* bad argument: NaN, eps_r < 1, k0 <= 0, |pol.khat| > 1e-12,
                            empty body, size out of range, NULL pointer          */
#define VIE_ENOMEM   -2  /* device allocation failed                            */
#define VIE_ENOCONV  -3  /* solve stopped at max_iter; stats hold the achieved
                            FP64 residual and the currents are kept              */
#define VIE_ETIMEOUT -4  /* a bounded device-side wait gave up                  */
#define VIE_EUNDEF   -5  /* g2 or N~c undefined (zero denominator); NaN written  */
#define VIE_EDEVICE  -6  /* CUDA runtime error                                  */
#define VIE_ESTATE   -7  /* call out of order (e.g. far field before a solve)   */

/* ---- precision modes --------------------------------------------------- */
#define VIE_PREC_MIXED 0 /* FP32 FFT matvec inside GMRES (FP64 Arnoldi and
                            Givens), iterative refinement on the FP64 residual  */
#define VIE_PREC_FP64  1 /* plain FP64 GMRES(m): FP64 matvec and basis          */
#define VIE_PREC_F32X2 2 /* operator only (vie_apply, vie_apply_device): FP64
                            inputs and outputs, the FFTs, spectral multiply and
                            contrast in double-float arithmetic (pairs of FP32
                            numbers, ~2^-47 rounding; Knuth TwoSum and the FMA
                            TwoProduct).  The mixed solver forms its residuals
                            with this operator unless opts.resid_fp64 is set.   */

/* ---- Krylov solvers (vie_solve_opts.solver) ----------------------------- */
#define VIE_SOLVER_GMRES    0 /* batched restarted GMRES(m), CGS + selective reorth.  */
#define VIE_SOLVER_BICGSTAB 1 /* batched BiCGStab (van der Vorst), the paper's solver */
#define VIE_SOLVER_COCR     2 /* batched COCR (conjugate orthogonal conjugate residual,
                                 Sogabe-Zhang): A = I - diag(chi) K is symmetric in
                                 the bilinear form sum x y / chi because K is
                                 (reciprocity), so a short recurrence with one
                                 operator application per step and no restart applies */

/* ---- far-field component bases (vie_farfield*) -------------------------- */
#define VIE_BASIS_CART 0 /* (F_x, F_y, F_z)                                      */
#define VIE_BASIS_SPH  1 /* (F_theta, F_phi, F_r)   (F_r = 0 up to rounding)     */
#define VIE_BASIS_CIRC 2 /* (F_L, F_R, F_r), F_L,R = (F_theta +/- i F_phi)/sqrt2
                            (Eq. 30)                                             */

typedef struct vie_handle vie_handle;

typedef struct vie_grid {
    int n[3];          /* voxels along x, y, z (each >= 1, product <= 2^28)     */
    double h;          /* voxel edge, same length unit as 1/k0 (> 0)            */
    double origin[3];  /* position of the grid centre (phase origin)            */
} vie_grid;

typedef struct vie_channel {
    double khat[3];    /* unit propagation direction                            */
    double pol[6];     /* complex polarisation (x re, x im, y re, y im, z re, z im),
                          transverse to khat; E_inc = pol e^{i k0 khat.r}         */
} vie_channel;

typedef struct vie_solve_opts {
    double tol;        /* target ||b - A64 x||_2 / ||b||_2 per RHS (default 1e-6) */
    int restart;       /* GMRES restart length m (default 30, 1..512)            */
    int max_iter;      /* cap on inner iterations per RHS (default 5000)         */
    int precision;     /* VIE_PREC_MIXED (default) or VIE_PREC_FP64              */
    double inner_tol;  /* mixed mode: relative reduction asked of each FP32 inner
                          solve, floored at inner_floor tol ||b|| (default 1e-6)  */
    int use_x0;        /* 0: x0 = 0; 1: start from the currents stored in the
                          handle (same n_rhs, restart and precision as the previous
                          solve); 2: initial currents from the network attached
                          with vie_attach_net: the prediction x0 = b + s (Born
                          term b plus the network's scattered-field correction s)
                          enters as beta b + alpha s with (beta, alpha) minimising
                          the residual norm (needs restart >= 3).  A supplied
                          guess whose FP64 residual is not below ||b|| is
                          replaced by zero.                                       */
    int precond;       /* 0: GMRES; 1: FGMRES with the learned right preconditioner
                          attached by vie_attach_precond (mixed or FP64 basis);
                          2: FGMRES with the block-Jacobi preconditioner set up by
                          vie_set_block_precond (mixed precision, GMRES)          */
    int solver;        /* VIE_SOLVER_GMRES (default), VIE_SOLVER_BICGSTAB (the
                          paper's solver, Sec. II-C) or VIE_SOLVER_COCR, inside
                          the same FP64 refinement.  BiCGStab needs restart >= 8
                          (its 7 vectors use the basis storage), COCR restart >= 4
                          (5 vectors; restart has no other meaning for either);
                          both need use_x0 0 or 1 and precond 0                */
    int resid_fp64;    /* mixed mode: 0 (default) forms the refinement residual
                          b - A x with the double-float operator (VIE_PREC_F32X2,
                          FP64 accuracy within a few 2^-47, several times faster
                          on GB300, whose FP64 rate is 1/64 of FP32); 1 with the
                          FP64 operator                                           */
    double reorth_eta; /* GMRES: a second classical Gram-Schmidt pass runs for an
                          RHS when the first left ||w'||^2 < reorth_eta ||w||^2
                          (Daniel-Gragg-Kaufman-Stewart test; default 0.1, i.e.
                          ||w'|| < 0.32 ||w||; 0 never, values >= 1 always)       */
    double inner_floor; /* mixed mode: an inner solve stops once its recurrence
                          residual is below max(inner_tol ||r||, inner_floor tol
                          ||b||) (default 0.7, in (0, 1])                         */
    int arnoldi;       /* orthogonalisation of GMRES without a preconditioner:
                          1 (default) one-sweep Arnoldi: the operator is applied
                          to the not yet orthogonalised vector and the Arnoldi
                          relation of the shifted operator A - I gives the next
                          Hessenberg column, so one pass over the basis per step
                          orthogonalises, normalises and takes the inner
                          products (Pythagorean norm; two explicit classical
                          passes where beta^2 < reorth_eta ||B v||^2); 0
                          classical Gram-Schmidt, inner products then update
                          (two passes per step, a second pair where the
                          reorth_eta test asks for it).  FGMRES (precond 1, 2),
                          BiCGStab and COCR ignore it                             */
} vie_solve_opts;

typedef struct vie_solve_stats {
    int n_rhs;         /* RHS solved                                             */
    int converged;     /* RHS that reached tol                                   */
    int iters_max;     /* largest inner-iteration count over the RHS             */
    int outer_max;     /* largest number of FP64 refinement steps                */
    long long matvecs32;   /* FP32 operator applications (per RHS, summed)       */
    long long matvecs64;   /* FP64 operator applications (per RHS, summed)       */
    double relres_max; /* largest final FP64 relative residual                   */
    double seconds;    /* wall time of the solve (device-synchronised)           */
    int* iters;        /* optional caller array [n_rhs]: inner iterations per RHS */
    double* relres;    /* optional caller array [n_rhs]: final FP64 residual      */
} vie_solve_stats;

typedef struct vie_info {
    int n[3];          /* grid                                                   */
    int P[3];          /* padded FFT sizes: next power of two >= 2n-1 if within
                          15 % of the smallest 2,3,5,7-smooth size, else that   */
    long long n_body;  /* voxels with eps_r > 1 (unknowns / 3)                   */
    int n_rhs;         /* RHS held by the handle (last solve)                    */
    int device;        /* CUDA device ordinal                                    */
    double device_bytes; /* device memory held by the handle                     */
} vie_info;

/* Default options: tol 1e-6, restart 30, max_iter 5000, mixed precision, inner_tol 1e-6,
 * reorth_eta 0.1, inner_floor 0.7, GMRES, no start guess, no preconditioner. */
void vie_default_opts(vie_solve_opts* opts);

/*
 * vie_setup -- build the operator for one grid and wavenumber.
 * Sec. II-C: eps_r defines chi = eps_r - 1 (Eq. Js_def); the Green's tensor of
 * Eq. dyadicG is sampled on every voxel offset (-(n-1)..n-1)^3, embedded in a
 * zero-padded periodic array of size P and Fourier transformed once on the
 * device (FP64), keeping one octant per tensor component (Eq. 24's convolution
 * via FFT, the paragraph after Eq. Js_expand).
 *   g      : grid (n, h, origin), copied.
 *   eps_r  : host [n0][n1][n2] real relative permittivity, >= 1, finite.
 *   k0     : free-space wavenumber > 0.
 *   out    : receives the new handle (device = the current CUDA device).
 * Size limits: at most 2^28 voxels; padded lengths up to 8192 per axis, the
 * first one up to 3200 (the fused x pass holds three components of a column
 * in shared memory) and the last up to 6400 (two FP64 line buffers): long
 * boxes go shortest axis first, longest last.  Device memory grows with the
 * padded grid: about 18 B (FP32 work) + 36 B (FP64 work) + 24 B x 6 / 8
 * (kernel octants) per padded point, plus the Krylov basis.
 * Errors: VIE_EINVAL (bad g, eps_r, k0; body empty; a padded length beyond
 * the limits), VIE_ENOMEM, VIE_EDEVICE.
 */
int vie_setup(const vie_grid* g, const double* eps_r, double k0, vie_handle** out);

/* ---- discretisations (vie_setup_disc) ------------------------------------ */
#define VIE_DISC_D1 0 /* voxel-centred unknown w = chi E, ball-averaged dyadic kernel
                         (the default of vie_setup)                                   */
#define VIE_DISC_D2 1 /* the paper's rooftop expansion with pulse testing (Sec. II-C),
                         read as: unknown w_a on the +a face of each cell (face contrast
                         (chi(c) + chi(c + e_a))/2), scalar ball-averaged kernel G_h and
                         the grad-div by differences on the staggered grid,
                         y_a = w_a - chi_a (k^2 A_a + d+_a sum_b d-_b A_b), A = G_h * w;
                         the unknown set is the body plus its -x/-y/-z neighbour cells;
                         bodies should leave the first cell layer of the grid empty  */
/* vie_setup with a discretisation; with VIE_DISC_D2 every entry point works on
 * the face unknowns (layouts unchanged: component a of cell c is the +a face of
 * c; far fields place it at the face centre).  The learned parts and
 * vie_apply_noalloc are D1 only.  Errors: as vie_setup, VIE_EINVAL for disc. */
int vie_setup_disc(const vie_grid* g, const double* eps_r, double k0, int disc, vie_handle** out);

/* Replace the body on the same grid (keeps the kernel spectrum).  Host
 * [n0][n1][n2] eps_r.  Discards stored currents.  Errors as vie_setup. */
int vie_set_eps(vie_handle* hd, const double* eps_r);
/* Same with a device pointer to [n0][n1][n2] doubles. */
int vie_set_eps_device(vie_handle* hd, const double* eps_r_dev);

/*
 * vie_solve -- contrast currents of n_rhs incident channels (Sec. II-C, Eq. 24;
 * the paper solves each channel separately, Sec. III).  The right-hand sides
 * b_j = chi pol_j e^{i k0 khat_j.r} are built on the device; the solver is
 * restarted GMRES (the paper uses BiCGStab; both converge to the same
 * solution) over all channels at once.  The currents stay in the handle for
 * vie_farfield / vie_get_current.
 *   ch     : host array [n_rhs] of channels (|khat| = 1, pol transverse).
 *   opts   : NULL for defaults.
 *   stats  : optional output.
 * Errors: VIE_EINVAL, VIE_ENOMEM, VIE_ENOCONV (currents kept), VIE_EDEVICE.
 */
int vie_solve(vie_handle* hd, const vie_channel* ch, int n_rhs, const vie_solve_opts* opts,
              vie_solve_stats* stats);
/* Solves of independent bodies (handles, each with its own grid and stream)
 * run concurrently: up to max_threads host threads (<= 0: 8) each drive one
 * handle's vie_solve, so the kernels of different bodies share the GPU --
 * bodies of uneven grid sizes whose single solves would leave most SMs idle.
 * ch[i] / n_rhs[i]: the channels of body i; opts shared (NULL: defaults);
 * stats: optional array [n_bodies].  Every handle must be distinct (a handle
 * is not thread-safe) and the kernel timer off.  Returns VIE_OK, or the code
 * of the first body that failed (hard errors before VIE_ENOCONV) with its
 * message prefixed by the body index; the other bodies' results stand.
 * Batching of independent problems is this library's addition; the paper
 * solves one scatterer at a time. */
int vie_solve_many(vie_handle* const* hds, const vie_channel* const* ch, const int* n_rhs, int n_bodies,
                   const vie_solve_opts* opts, vie_solve_stats* stats, int max_threads);


/*
 * vie_farfield -- far-field amplitudes of every stored current on a product
 * grid of directions (Eq. 25 with C_inf = kappa k0^2 h^3/(4 pi); components
 * per Eq. Eproj / Eq. 30).  The incident plane wave contributes only in its
 * own forward direction and is omitted (E_tot,inf = F off-forward).
 *   theta[nt], phi[np] : angles in radians (host).
 *   basis              : VIE_BASIS_*.
 *   out                : host [n_rhs][nt][np][3] complex (interleaved doubles).
 * Errors: VIE_EINVAL, VIE_ESTATE (no solve yet), VIE_ENOMEM, VIE_EDEVICE.
 */
int vie_farfield(vie_handle* hd, const double* theta, int nt, const double* phi, int np,
                 int basis, double* out);

/* Same for an arbitrary list of unit vectors dirs[D][3] (host); out as above
 * with D directions: [n_rhs][D][3] complex.  Evaluated in FP64. */
int vie_farfield_dirs(vie_handle* hd, const double* dirs, int D, int basis, double* out);

/* Finite numerical aperture (Eq. NAfield): each detector d collects its field
 * over a cone around the unit axis centers[d] with the angular weight
 * W(t) = exp(-t^2 / (2 sigma^2)), t the angle to the axis, t <= theta_na:
 *   out[r][d] = sum_q w_q pol_d . F_r(rhat_q)   (bilinear, as Eq. Eproj),
 * on a product rule -- nt Gauss-Legendre nodes in t on [0, theta_na], nphi
 * uniform azimuths about the axis (frame u = (a x c)/|a x c|, a = z, or x when
 * |c_z| >= 0.9, v = c x u) -- with weights W sin(t) dt dphi normalised to sum 1,
 * so a vanishing aperture gives the point detector of Eq. Eproj.  The
 * amplitudes enter hom_transfer / vie_hom_map like point-detector ones (the
 * collected field operator is linear in the input modes).
 *   centers [D][3], pols [D][3] complex (interleaved), out [n_rhs][D] complex.
 * Errors: VIE_EINVAL (nt 1..64, nphi 1..256, 0 < theta_na <= pi/2, sigma > 0),
 * VIE_ESTATE (no solution), VIE_ENOMEM. */
int vie_farfield_na(vie_handle* hd, const double* centers, const double* pols, int D, double theta_na, double sigma,
                    int nt, int nphi, double* out);

/* Device variant of vie_farfield_dirs: dirs_dev [D][3] doubles and out_dev
 * [n_rhs][D][3] complex doubles on the device; enqueued on the handle's stream
 * and synchronised before return. */
int vie_farfield_dirs_device(vie_handle* hd, const double* dirs_dev, int D, int basis,
                             double* out_dev);

/*
 * hom_transfer -- two-photon observables of one detector pair and channel pair
 * (Sec. II-A/B).  E[8] = complex far-field amplitudes [det][ch] (det 0 = a at
 * r1, det 1 = b at r2; ch 0 = k1, ch 1 = k2), interleaved.  omega[2]: channel
 * frequencies (NULL = equal).  Outputs (any may be NULL):
 *   g2[1]      : Eq. 10, omega1 omega2 |E_a1 E_b2 + E_a2 E_b1|^2 /
 *                (sum_l omega_l |E_al|^2 sum_l omega_l |E_bl|^2)
 *   Nc[n_tau]  : N~c(dtau) = 1 + 2 Re(A_dir A_ex*) e^{-dtau^2/sigma^2} /
 *                (|A_dir|^2 + |A_ex|^2), A_dir = T_a1 T_b2, A_ex = T_a2 T_b1,
 *                T_aj = sqrt(omega_j) E_aj (Eqs. 18-22 with a Gaussian
 *                envelope, Eq. HOM_envelope)
 *   visibility : 1 - N~c(0)
 * Host-side scalar arithmetic (the same function the device map kernel runs).
 * Returns VIE_EUNDEF with NaN outputs when a denominator is zero.
 */
int hom_transfer(const double E[8], const double omega[2], double sigma, const double* dtau,
                 int n_tau, double* g2, double* Nc, double* visibility);

/*
 * vie_hom_map -- g2, HOM visibility and the normalised classical
 * intensity-product correlation (Eq. 27) for every detector pair (r1 in set A,
 * r2 in set B) of one channel pair, on the device.
 *   Ea [2][nA] complex: detector-projected amplitudes of channels 1, 2 at the
 *                       directions of set A (component e_a);
 *   Eb [2][nB] complex: same at set B (component e_b);
 *   g2, vis, p2 : host [nA][nB] doubles (any may be NULL); NaN where undefined;
 *                 p2 is divided by its maximum over the map.
 * Errors: VIE_EINVAL, VIE_ENOMEM, VIE_EDEVICE.
 */
int vie_hom_map(const double* Ea, int nA, const double* Eb, int nB, double sigma, double* g2,
                double* vis, double* p2);

/* Copy the stored current of RHS `rhs` to host out[3][n0][n1][n2] complex
 * (zero outside the body).  Errors: VIE_EINVAL, VIE_ESTATE. */
int vie_get_current(vie_handle* hd, int rhs, double* out);

/*
 * vie_apply -- one operator application y = w - chi (K * w) (Eq. 24 in the w
 * unknown) for n_rhs vectors, in the given precision, through the same FFT
 * kernels the solver uses.  w, y: host [n_rhs][3][n0][n1][n2] complex; w must
 * vanish outside the body (y is w there).  Errors: VIE_EINVAL, VIE_ENOMEM,
 * VIE_EDEVICE.
 */
int vie_apply(vie_handle* hd, const double* w, double* y, int n_rhs, int precision);

/* Device variant on the compact body-voxel layout: w_dev, y_dev are
 * [n_rhs][3][n_body] complex (float2 for VIE_PREC_MIXED, double2 for
 * VIE_PREC_FP64 and VIE_PREC_F32X2), body voxels in C order.  Enqueued on the handle's stream;
 * not synchronised. */
int vie_apply_device(vie_handle* hd, const void* w_dev, void* y_dev, int n_rhs, int precision);

/*
 * vie_apply_noalloc -- the FP32 operator of vie_apply_device for callers that
 * cannot let the library allocate device memory: their device memory belongs
 * to a framework's caching allocator or to a pool sized at start-up, or their
 * loop must not stall on cudaMalloc/cudaFree.  The paper has no counterpart;
 * this is a deployment variant of vie_apply_device that allocates nothing.
 * Its FFT workspace is a fixed 64 MiB file-scope device array, held by every
 * GPU that loads the library until the process exits.
 *   w_dev, y_dev : device [n_rhs][3][n_body] complex64 (float2), layout as in
 *                  vie_apply_device; 1 <= n_rhs <= 1024.
 * Limits: every padded size must be a power of two (16..512), and the
 * workspace of one RHS (3 n0 n1 P2 + 3 n0 P1 P2 complex64 words) must fit in
 * the array (grids up to 64^3 do); otherwise VIE_EINVAL, with the sizes in
 * vie_last_error().  It always runs the register FFT passes: a handle set to
 * the generic path (vie_set_fft_path(hd, 1)) is refused with VIE_EINVAL, as
 * are D2 handles.  Like every entry point it makes the handle's device current
 * (cudaSetDevice).  The first call on each device looks up the array's device
 * address with that device current; make that first call before any stream
 * capture.  All calls share the array and leave their data in it: calls that
 * can overlap on the GPU (other streams, unordered handles) race; calls on one
 * stream run in order.  Enqueued on the handle's stream; not synchronised.
 */
int vie_apply_noalloc(vie_handle* hd, const void* w_dev, void* y_dev, int n_rhs);

/* Kernel-level check: batched 1-D complex DFT of `count` contiguous lines of
 * length L (2,3,5,7-smooth, <= 8192; FP64 <= 6400) by the library's FFT engine, host
 * in/out [count][L] complex doubles, forward (sign -1) when inverse == 0,
 * unnormalised inverse otherwise, in FP32 (precision MIXED) or FP64. */
int vie_fft_lines(const double* in, double* out, int L, int count, int inverse, int precision);

int vie_get_info(const vie_handle* hd, vie_info* info);

/* ---- multi-body batches (many bodies of uneven grids in one launch) ----
 * Batching applied to bodies as well as right-hand sides: a batch holds bodies of
 * different grids (each its own n, h, origin and eps_r; one k0), each padded
 * to a power of two per body (the smallest >= 2n - 1 over its axes, 32..256,
 * so n <= 128 per axis).  Body b's RHS j is row b * n_rhs + j of batch-wide
 * compact vectors [rows][3][stride], stride = vie_batch_stride() = the
 * largest body's n_body; a body uses the first n_body entries of each
 * component (the rest is zero and ignored).  The FP32 operator runs its five
 * passes (Sec. II-C, Eq. 24) over all rows of all bodies that share a padded
 * size in one launch per pass, each row with its own grid, voxel map,
 * contrast and kernel spectrum; the FP64-accuracy residual runs each body's
 * own operator.  The handle owns all device memory; not thread-safe.
 * Errors: VIE_EINVAL (bad sizes, eps_r < 1, an empty body), VIE_ENOMEM,
 * VIE_EDEVICE. */
typedef struct vie_batch vie_batch;
int vie_batch_create(int n_bodies, const vie_grid* grids, const double* const* eps_r, double k0,
                     vie_batch** out);
void vie_batch_destroy(vie_batch* bt);
long long vie_batch_stride(const vie_batch* bt);
/* per-body n, P, n_body; device_bytes = the whole batch */
int vie_batch_info(const vie_batch* bt, int body, vie_info* info);
/* y = A w for n_rhs rows per body (all bodies): w_dev, y_dev device
 * [n_bodies * n_rhs][3][stride], float2 (VIE_PREC_MIXED) or double2 (VIE_PREC_FP64,
 * VIE_PREC_F32X2).  Enqueued on the batch's stream (synchronised by the call
 * that uploads the slot table). */
int vie_batch_apply_device(vie_batch* bt, const void* w_dev, void* y_dev, int n_rhs, int precision);
/* The same n_rhs channels for every body, solved together: mixed-precision
 * GMRES (opts: precision MIXED, solver GMRES, precond 0, use_x0 0) with the
 * refinement of vie_solve.  stats->iters / relres: [n_bodies * n_rhs].
 * Errors: as vie_solve. */
int vie_batch_solve(vie_batch* bt, const vie_channel* ch, int n_rhs, const vie_solve_opts* opts,
                    vie_solve_stats* stats);
/* current of (body, rhs) on the body's full grid, host out[3][n0][n1][n2] complex */
int vie_batch_get_current(vie_batch* bt, int body, int rhs, double* out);
/* far field of every RHS of one body at D directions (Eq. 25, FP64), host
 * out[n_rhs][D][3] complex in the basis of vie_farfield_dirs */
int vie_batch_farfield_dirs(vie_batch* bt, int body, const double* dirs, int D, int basis, double* out);

/* ---- learned initial guess ----------------------------------------------
 * A 4-level 3-D U-Net (channels c0..c3, 3x3x3 convolutions with ReLU, 2x2x2
 * average pooling, nearest upsampling, skip concatenations, 1x1x1 head) maps
 * 10 input channels on a coarse cubic grid of D^3 voxels (D % 8 == 0) --
 * block-averaged chi, Re/Im of the polarisation and the propagation direction
 * (constant channels) -- to 6 output channels, the scattered part of the
 * total field with the incident phase removed, (E_tot - E_inc) e^{-i k0 khat.r},
 * averaged over each block's body voxels.  The solver turns the prediction
 * into b + s, b = chi E_inc and s = chi (upsampled prediction e^{i k0 khat.r}),
 * and starts from the residual-minimising combination beta b + alpha s
 * (use_x0 = 2); plain GMRES from x0 = 0 is the fallback, chosen per RHS by
 * the FP64 residual.  The paper's method is not learned: this part is an
 * addition of this library.  Activations in bf16 (or FP32 for gradient checks), weights FP32
 * masters, every sum in FP32; trained with Adam on solver-generated data.
 * Device arrays: x [B][10][D^3], y / t [B][6][D^3], m [B][D^3] (float32),
 * on the current device; these calls synchronise the device's null stream. */
typedef struct vie_net vie_net;
int vie_net_create(const int channels[4], unsigned long long seed, int bf16, vie_net** out);
/* the same with `cin` input channels (10: initial guess; 7: preconditioner); VIE_EINVAL outside 1..64 */
int vie_net_create_io(const int channels[4], int cin, unsigned long long seed, int bf16, vie_net** out);
void vie_net_destroy(vie_net* net);
long long vie_net_num_params(const vie_net* net);
/* bf16 networks: run the 3x3x3 and 1x1x1 convolutions (forward, data and
 * weight gradients) as implicit GEMMs on the tensor cores (tcgen05.mma
 * kind::f16, BF16 operands, FP32 accumulation in tensor memory) when on != 0
 * (the default), or on the CUDA-core kernels.  Layers with more than 128
 * output or 256 input channels always take the CUDA cores.  VIE_EINVAL for a
 * NULL net; a tensor-core wait that runs out makes the next forward or
 * gradient call return VIE_ETIMEOUT. */
int vie_net_set_tensor_cores(vie_net* net, int on);
/* host float32 arrays of vie_net_num_params() entries: per layer w[co][ci][k^3] then b[co] */
int vie_net_get_params(const vie_net* net, float* host);
int vie_net_set_params(vie_net* net, const float* host);
int vie_net_forward(vie_net* net, const float* x_dev, float* y_dev, int B, int D);
/* masked mean-squared error sum m (y - t)^2 / (6 sum m) and its parameter
 * gradients (host, same layout as the parameters; NULL to skip) */
int vie_net_gradients(vie_net* net, const float* x_dev, const float* t_dev, const float* m_dev, int B, int D,
                      float* loss, float* grads_host);
/* one Adam step (beta 0.9, 0.999, eps 1e-8) on that loss */
int vie_net_train_step(vie_net* net, const float* x_dev, const float* t_dev, const float* m_dev, int B, int D,
                       float lr, float* loss);
/* training sample of every RHS of the handle's last solve on the grid
 * coarsened by `factor`: x [rhs][10][D^3]; when t_dev / m_dev are given also
 * the targets t [rhs][6][D^3] and mask m [rhs][D^3] (fraction of body voxels
 * per block) from the solved currents.  Errors: VIE_EINVAL, VIE_ESTATE. */
int vie_net_features(vie_handle* hd, int factor, float* x_dev, float* t_dev, float* m_dev);
/* attach (or detach with NULL) the network used by use_x0 = 2; not owned */
int vie_attach_net(vie_handle* hd, vie_net* net, int factor);
/* number of RHS of the last solve whose supplied initial guess was rejected */
int vie_guesses_rejected(const vie_handle* hd);

/* ---- block-Jacobi preconditioner (FGMRES, opts.precond = 2) ---------------
 * The paper's solver applies a block preconditioner over blocks of the volume
 * (7 x 7 lateral blocks of the metasurface, Sec. III-B) without further detail.
 * Here: M(v) approximately solves A_bd z = v, A_bd = I - diag(chi) K_bd with
 * K_bd keeping only interactions between voxels of the same block, by
 * `inner_iters` COCR steps from z = 0 (FP32 vectors, FP64 scalars).  The blocks
 * are the cells of the tiling given by interior cut positions per axis:
 * cuts = [axis 0 cuts..., axis 1 cuts..., axis 2 cuts...], ncuts[a] of them
 * on axis a, strictly increasing inside (0, n_a); no cut on an axis keeps it
 * whole.  Each block is cropped to the bounding box of its body voxels; A_bd
 * runs as one batched FFT operator on the largest box, one slot per non-empty
 * block.  Set up again after every change of the body (vie_set_eps drops it).
 * D1 only.  Errors: VIE_EINVAL (cuts, iterations, D2), VIE_ENOMEM. */
int vie_set_block_precond(vie_handle* hd, const int* cuts, const int ncuts[3], int inner_iters);
/* The block layout alone, on the host (no device work): for a grid n, body
 * voxels vox[n_body] (increasing C-order linear indices) and the cuts of
 * vie_set_block_precond, box_out = the block box (largest cropped extent per
 * axis), *blocks_out = non-empty blocks; map_out, when not NULL, receives
 * [blocks][box0][box1][box2] compact body indices (-1 where a block has no
 * voxel) and must hold blocks x box0 x box1 x box2 ints (call once with NULL
 * to size it).  Errors: VIE_EINVAL. */
int vie_block_layout(const int n[3], const int* vox, long long n_body, const int* cuts, const int ncuts[3],
                     int box_out[3], int* blocks_out, int* map_out);
/* y = A_bd w for one FP32 compact vector [3][n_body] (device, float2); for
 * checks of the block operator.  Enqueued on the handle's stream. */
int vie_block_apply_device(vie_handle* hd, const void* w_dev, void* y_dev);

/* ---- learned right preconditioner (FGMRES, opts.precond = 1) --------------
 * Each Krylov vector v (unit norm) is mapped to z = v + up(Net(x)) / sqrt(3 Nb)
 * with x [7][D^3] = (block-averaged chi, sqrt(3 Nb) times the block-averaged
 * Re/Im of v per component) on the grid coarsened by `factor`, and the solver
 * applies A to z and keeps the z vectors for the update (flexible GMRES; the
 * preconditioner may change between steps).  The network, made with cin = 7,
 * learns A^{-1} - I on pairs (u = A v, v): targets t = sqrt(3 Nb)/||u|| times
 * the block average of (v - u).  Not owned; NULL detaches.  Errors: VIE_EINVAL
 * (non-cubic grid, n not divisible by 8 x factor, network with cin != 7). */
int vie_attach_precond(vie_handle* hd, vie_net* net, int factor);
/* training pairs for the preconditioner: v_dev [n][3][Nb] complex64 (device,
 * the body layout of vie_apply_device) -> u = A v with the FP32 operator, then
 * x_dev [n][7][D^3], t_dev [n][6][D^3], m_dev [n][D^3] (float32, device) as
 * above.  Synchronises the handle's stream.  Errors: VIE_EINVAL, VIE_ENOMEM. */
int vie_precond_pairs(vie_handle* hd, int factor, const void* v_dev, int n, float* x_dev, float* t_dev,
                      float* m_dev);

/* Engine of the far-field contractions on (theta, phi) grids (vie_farfield):
 * 0 (default) tensor cores (tcgen05, TF32 split three ways: hi*hi + hi*lo +
 * lo*hi, FP32 accumulation in tensor memory), 1 CUDA-core FP32.
 * Errors: VIE_EINVAL. */
int vie_set_farfield_engine(vie_handle* hd, int engine);

/* Kernel-level check of the far-field GEMM engines: C = A B for complex
 * matrices (host, row-major, interleaved doubles): A [M][K], B [K][N],
 * C [M][N]; computed on the device in complex64 by the engine named as in
 * vie_set_farfield_engine.  Errors: VIE_EINVAL, VIE_ENOMEM, VIE_ETIMEOUT,
 * VIE_EDEVICE. */
int vie_cgemm(int M, int N, int K, const double* A, const double* B, double* C, int engine);

/* FFT kernel family of the FP32 operator passes: 0 (default) uses the
 * register four-step kernels on every axis whose padded length is a power of
 * two in 16..512 and the generic shared-memory Stockham kernels elsewhere;
 * 1 forces the generic kernels everywhere.  Results agree to FP32 round-off;
 * used for A/B timing.  Errors: VIE_EINVAL. */
int vie_set_fft_path(vie_handle* hd, int path);
/* Autotuner of the operator's FFT schedule on this handle's grid: times
 * `reps` FP32 operator applications on n_rhs deterministic test vectors for
 * each candidate configuration -- per axis the padded length of the default
 * rule and the other of (next power of two >= 2n-1, smallest 2,3,5,7-smooth
 * length), i.e. radix-16/8/4/2 four-step kernels or the mixed-radix Stockham
 * engine, and for power-of-two lengths the register or the generic path --
 * and keeps the fastest (rebuilding the kernel spectrum; body, solver state
 * and stored currents are kept).  P_out (optional) receives the padded
 * lengths, ms_per_apply (optional) the best time of one application.  The
 * operator's values do not depend on the choice (any P >= 2n-1 embeds the
 * same convolution); only rounding differs.  Errors: VIE_EINVAL, VIE_ENOMEM. */
int vie_autotune(vie_handle* hd, int n_rhs, int reps, int P_out[3], double* ms_per_apply);

/* Launch statistics: number of library kernels launched by this process. */
long long vie_kernel_launches(void);

/* Optional per-kernel timing: when enabled, every library kernel launch is
 * bracketed by CUDA events on its stream and its duration accumulated under
 * a kernel id (0 .. vie_timer_count()-1; names from vie_timer_name), together
 * with the algorithmic bytes of the launch (each input read once, each output
 * written once).  Adds two event records per launch; off by default. */
void vie_timer_enable(int on);
void vie_timer_reset(void);
int vie_timer_read(int id, double* total_ms, long long* launches, double* bytes);
const char* vie_timer_name(int id);
int vie_timer_count(void);

/* Device stream used by the handle (cudaStream_t as void*). */
void* vie_stream(vie_handle* hd);

void vie_destroy(vie_handle* hd);

const char* vie_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* VIE_H */
