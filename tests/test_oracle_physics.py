"""Physics pins of the oracle's discrete VIE: energy conservation and
S-matrix unitarity for lossless bodies (Sec. II-A, Eq. SmatrixFull),
reciprocity, grid symmetries, the Lorenz-Mie series for spheres (Sec. III-A)
and the Rayleigh-dipole limit of g2 (Eq. 26)."""
import math

import numpy as np
import pytest

from oracle import hom, mie, vie
from paper_2508_16471_gb300 import inputs

K0 = 2.0 * math.pi


def _random_body(n, seed):
    rng = np.random.default_rng(seed)
    eps = 1.0 + rng.uniform(0.5, 4.0, n) * (rng.uniform(size=n) < 0.7)
    return eps


def _lu_solver(n, h, eps):
    chi = vie.contrast(eps)
    A = vie.dense_operator(n, h, K0, chi)
    lu = np.linalg.inv(A)

    def solve(khat, pol):
        b = vie.rhs(chi, vie.incident_field(n, h, K0, khat, pol))
        return (lu @ b.reshape(-1)).reshape(b.shape)
    return solve


def _quad(n, h):
    Rb = h * math.sqrt(sum((v / 2.0) ** 2 for v in n))
    return vie.sphere_quadrature(int(K0 * Rb) + 20)


def test_optical_theorem_lossless_exact():
    n, h = (5, 4, 6), 0.09
    eps = _random_body(n, 11)
    solve = _lu_solver(n, h, eps)
    d, wq = _quad(n, h)
    for khat, pol in [((0, 0, 1.0), (1.0, 0, 0)), ((0.6, 0, 0.8), (0, 1j, 0)),
                      ((0, 1.0, 0), (0.6, 0, 0.8j))]:
        khat = np.array(khat, float)
        pol = np.array(pol, complex)
        pol = pol / np.linalg.norm(pol)
        w = solve(khat, pol)
        Ff = vie.farfield(w, n, h, K0, khat[None])[0]
        ext = 4 * math.pi / K0 * np.imag(np.conj(pol) @ Ff)
        F = vie.farfield(w, n, h, K0, d)
        sca = float(np.sum(wq * np.sum(np.abs(F) ** 2, axis=1)))
        assert abs(ext - sca) <= 1e-9 * sca


def test_generalized_optical_theorem():
    """(f_ij - f_ji*)/(2i) = (k/4pi) oint F_i* . F_j dOmega with
    f_ij = conj(p_i) . F_j(k_i): unitarity of S for a lossless body."""
    n, h = (4, 5, 4), 0.1
    eps = _random_body(n, 12)
    solve = _lu_solver(n, h, eps)
    d, wq = _quad(n, h)
    ch = [(np.array([0, 0, 1.0]), np.array([1.0, 0, 0], complex)),
          (np.array([0.8, 0.0, 0.6]), np.array([0.0, 1.0, 0.0], complex)),
          (np.array([0.0, -1.0, 0.0]), np.array([1.0, 0.0, 1j]) / math.sqrt(2))]
    W = [solve(k, p) for k, p in ch]
    Fd = [vie.farfield(w, n, h, K0, d) for w in W]
    for i in range(3):
        for j in range(3):
            fij = np.conj(ch[i][1]) @ vie.farfield(W[j], n, h, K0, ch[i][0][None])[0]
            fji = np.conj(ch[j][1]) @ vie.farfield(W[i], n, h, K0, ch[j][0][None])[0]
            lhs = (fij - np.conj(fji)) / 2j
            rhs = K0 / (4 * math.pi) * np.sum(wq * np.sum(np.conj(Fd[i]) * Fd[j], axis=1))
            assert abs(lhs - rhs) <= 1e-9 * max(abs(rhs), 1e-3 * abs(fij))


def test_reciprocity():
    """p_s . F(r_s; k_i, p_i) = p_i . F(-k_i; -r_s, p_s)."""
    n, h = (5, 5, 3), 0.1
    eps = _random_body(n, 13)
    solve = _lu_solver(n, h, eps)
    ki, pi_ = np.array([0.0, 0.6, 0.8]), np.array([1.0, 0.0, 0.0], complex)
    rs = np.array([0.48, 0.6, -0.64])
    ps = np.cross(rs, [0.0, 0.0, 1.0])
    ps = (ps / np.linalg.norm(ps)).astype(complex) + 0.3j * np.cross(rs, ps / np.linalg.norm(ps))
    wi = solve(ki, pi_)
    wr = solve(-rs, ps)
    a = ps @ vie.farfield(wi, n, h, K0, rs[None])[0]
    b = pi_ @ vie.farfield(wr, n, h, K0, -ki[None])[0]
    assert abs(a - b) <= 1e-12 * abs(a)


def test_rotation_symmetry_of_centred_sphere():
    """Rotating a centred cubic grid by 90 deg about y maps channel
    (+z, x-pol) onto (+x, -z-pol): far fields map exactly."""
    g = inputs.Grid((8, 8, 8), 1.0 / 20.0)
    eps = inputs.sphere(g, 0.17, 2.25)
    solve = _lu_solver(g.n, g.h, eps)
    w1 = solve(np.array([0, 0, 1.0]), np.array([1.0, 0, 0], complex))
    w2 = solve(np.array([1.0, 0, 0]), np.array([0, 0, 1.0], complex))
    R = np.array([[0, 0, 1.0], [0, 1.0, 0], [-1.0, 0, 0]])
    rng = np.random.default_rng(0)
    d = rng.standard_normal((20, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    F1 = vie.farfield(w1, g.n, g.h, K0, d)
    F2 = vie.farfield(w2, g.n, g.h, K0, d @ R.T)
    assert np.abs(F2 + F1 @ R.T).max() <= 1e-12 * np.abs(F1).max()


def _mie_dirs():
    th = np.radians(np.arange(0, 181, 5.0))
    ph = np.radians(np.arange(0, 356, 5.0))
    T, P = np.meshgrid(th, ph, indexing="ij")
    T, P = T.ravel(), P.ravel()
    d = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], -1)
    return T, P, d


def test_mie_extinction_convention():
    # Q_ext from the coefficients equals (4/x^2) Re S(0), and F(0) carries it
    x, m = 2.5, 1.5
    S1, S2 = mie.amplitudes(x, m, np.array([0.0]))
    assert abs(S1[0] - S2[0]) < 1e-12
    assert abs(mie.extinction_efficiency(x / K0, m * m, K0) - 4 / x ** 2 * S1[0].real) < 1e-12


def test_vie_converges_to_mie_sphere():
    """Sphere R = 0.4 lambda, eps_r = 2.25 (the 16^3 sphere workload): the far
    field approaches the Mie series as the grid is refined; 16^3 within 5 %."""
    T, P, d = _mie_dirs()
    Fm = mie.farfield(0.4, 2.25, K0, T, P)
    errs = []
    for N in (12, 16, 32):
        h = 0.8 / N
        g = inputs.Grid((N, N, N), h)
        eps = inputs.sphere(g, 0.4, 2.25)
        w, info = vie.solve_channels(g.n, h, K0, eps, [((0, 0, 1.0), (1.0, 0, 0))], tol=1e-10)
        F = vie.farfield(w[0], g.n, h, K0, d)
        errs.append(np.linalg.norm(F - Fm) / np.linalg.norm(Fm))
    assert errs[1] < 0.05
    assert errs[0] > errs[1] > errs[2]


def test_single_voxel_is_small_mie_sphere():
    """One voxel = a sphere of radius a: error vs Mie falls as (k a)^2
    (Clausius-Mossotti polarisability with its radiative correction)."""
    T, P, d = _mie_dirs()
    sel = slice(None, None, 37)
    errs = []
    for h in (0.02, 0.01):
        a = vie.equivalent_radius(h)
        w, _ = vie.solve_channels((1, 1, 1), h, K0, np.full((1, 1, 1), 2.1),
                                  [((0, 0, 1.0), (1.0, 0, 0))], method="lu")
        F = vie.farfield(w[0], (1, 1, 1), h, K0, d[sel])
        Fm = mie.farfield(a, 2.1, K0, T[sel], P[sel])
        errs.append(np.linalg.norm(F - Fm) / np.linalg.norm(Fm))
    assert errs[0] < 2e-3
    assert 3.5 < errs[0] / errs[1] < 4.5


def test_rayleigh_limit_g2():
    """Dipole scatterer, the paper's channels (y-pol along +x, x-pol along +y),
    a = b = z: g2 = sin^2(phi1 + phi2) for any theta (Sec. III-A)."""
    h = 0.01
    chs = [(c.khat, c.pol) for c in inputs.channels_paper_sphere()]
    w, _ = vie.solve_channels((1, 1, 1), h, K0, np.full((1, 1, 1), 2.1), chs, method="lu")
    rng = np.random.default_rng(3)
    for _ in range(10):
        t1, t2 = rng.uniform(0.2, 2.9, 2)
        p1, p2 = rng.uniform(0, 2 * math.pi, 2)
        r1 = np.array([math.sin(t1) * math.cos(p1), math.sin(t1) * math.sin(p1), math.cos(t1)])
        r2 = np.array([math.sin(t2) * math.cos(p2), math.sin(t2) * math.sin(p2), math.cos(t2)])
        E = np.zeros((2, 2), complex)
        for j in range(2):
            F = vie.farfield(w[j], (1, 1, 1), h, K0, np.stack([r1, r2]))
            E[0, j], E[1, j] = F[0, 2], F[1, 2]
        assert abs(hom.g2_degenerate(E) - math.sin(p1 + p2) ** 2) < 1e-12


def test_g2_invariant_under_phase_origin_shift():
    g = inputs.Grid((4, 4, 4), 0.08)
    eps = _random_body(g.n, 14)
    chs = [(c.khat, c.pol) for c in inputs.channels_two_plane_waves()]
    r = np.array([[0.5, 0.5, math.sqrt(0.5)], [-0.5, 0.5, math.sqrt(0.5)]])
    vals = []
    for origin in ((0, 0, 0), (0.13, -0.21, 0.34)):
        chi = vie.contrast(eps)
        A = vie.dense_operator(g.n, g.h, K0, chi)
        E = np.zeros((2, 2), complex)
        for j, (k, p) in enumerate(chs):
            b = vie.rhs(chi, vie.incident_field(g.n, g.h, K0, k, p, origin))
            w = np.linalg.solve(A, b.reshape(-1)).reshape(b.shape)
            F = vie.farfield(w, g.n, g.h, K0, r, origin)
            E[0, j], E[1, j] = F[0, 2], F[1, 2]
        vals.append(hom.g2_degenerate(E))
    assert abs(vals[0] - vals[1]) < 1e-12


def test_detector_projection_bases():
    """e_theta = d rhat/d theta, e_phi = (d rhat/d phi)/sin(theta) by finite
    differences; components reassemble F; L/R follow Eq. 30."""
    rng = np.random.default_rng(7)
    th = rng.uniform(0.1, 3.0, 8)
    ph = rng.uniform(-3.0, 3.0, 8)
    rhat = lambda t, p: np.stack([np.sin(t) * np.cos(p), np.sin(t) * np.sin(p), np.cos(t)], -1)
    d = rhat(th, ph)
    eth, eph = vie.spherical_unit_vectors(d)
    e = 1e-6
    assert np.abs(eth - (rhat(th + e, ph) - rhat(th - e, ph)) / (2 * e)).max() < 1e-8
    dph = (rhat(th, ph + e) - rhat(th, ph - e)) / (2 * e) / np.sin(th)[:, None]
    assert np.abs(eph - dph).max() < 1e-8
    F = rng.standard_normal((8, 3)) + 1j * rng.standard_normal((8, 3))
    S = vie.project(F, d, 1)
    back = S[:, 0:1] * eth + S[:, 1:2] * eph + S[:, 2:3] * d
    assert np.abs(back - F).max() < 1e-14
    C = vie.project(F, d, 2)
    assert np.allclose(C[:, 0], (S[:, 0] + 1j * S[:, 1]) / math.sqrt(2), atol=1e-15)
    assert np.allclose(C[:, 1], (S[:, 0] - 1j * S[:, 1]) / math.sqrt(2), atol=1e-15)
    assert np.allclose(vie.project(F, d, 0), F)


def test_mie_components_in_spherical_basis():
    """The Mie field in (theta, phi) components is (i/k)(S2 cos phi, -S1 sin phi)."""
    th = np.array([0.3, 1.2, 2.5])
    ph = np.array([0.4, 2.0, -1.0])
    F = mie.farfield(0.3, 2.25, K0, th, ph)
    d = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], -1)
    S = vie.project(F, d, 1)
    S1, S2 = mie.amplitudes(K0 * 0.3, 1.5, th)
    assert np.allclose(S[:, 0], 1j / K0 * S2 * np.cos(ph), atol=1e-14)
    assert np.allclose(S[:, 1], -1j / K0 * S1 * np.sin(ph), atol=1e-14)
    assert np.abs(S[:, 2]).max() < 1e-14


def test_mie_general_incidence_pins():
    """The arbitrary-incidence Mie far field reduces to the z/x case and is
    covariant under a rotation of incidence, polarisation and directions."""
    T, P, d = _mie_dirs()
    sel = slice(None, None, 7)
    F0 = mie.farfield(0.3, 2.1, K0, T[sel], P[sel])
    Fg = mie.farfield_general(0.3, 2.1, K0, (0, 0, 1.0), (1.0, 0, 0), d[sel])
    assert np.abs(Fg - F0).max() <= 1e-13 * np.abs(F0).max()
    rng = np.random.default_rng(5)
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    Q *= np.sign(np.linalg.det(Q))
    Fr = mie.farfield_general(0.3, 2.1, K0, Q @ (0, 0, 1.0), Q @ np.array([1.0, 0, 0]), d[sel] @ Q.T)
    assert np.abs(Fr - F0 @ Q.T).max() <= 1e-12 * np.abs(F0).max()
    # transversality
    assert np.abs(np.sum(Fr * (d[sel] @ Q.T), axis=1)).max() <= 1e-13 * np.abs(F0).max()


def test_na_rule_pins():
    """The finite-NA quadrature: weights sum to one, the weighted mean
    direction is the axis times the W-weighted mean of cos(t) (a 1-D integral
    done here by scipy.integrate.quad), and a vanishing aperture returns the
    axis value of a smooth field."""
    from scipy.integrate import quad
    c = np.array([0.3, -0.5, 0.8])
    c /= np.linalg.norm(c)
    tna, sg = 0.4, 0.25
    dirs, W = vie.na_rule(c, tna, sg, 12, 16)
    assert abs(W.sum() - 1.0) < 1e-14
    num = quad(lambda t: np.exp(-t * t / (2 * sg * sg)) * np.sin(t) * np.cos(t), 0, tna)[0]
    den = quad(lambda t: np.exp(-t * t / (2 * sg * sg)) * np.sin(t), 0, tna)[0]
    assert np.abs(W @ dirs - c * num / den).max() < 1e-12
    assert np.abs(np.linalg.norm(dirs, axis=1) - 1).max() < 1e-14
    f = lambda d: np.exp(1j * 3.0 * (d @ np.array([1.0, 2.0, -0.5])))
    d0, W0 = vie.na_rule(c, 1e-4, 1.0, 4, 8)
    assert abs(np.sum(W0 * f(d0)) - f(c[None])[0]) < 1e-6


def test_axis_swap_covariance_of_circular_amplitudes():
    """The paper-scale grid is stored with the x and z axes swapped (a
    reflection).  Solving a chiral body in the swapped frame, with incidence,
    polarisation and directions mapped by the same swap, and mapping the far
    field back must give the paper-frame circular amplitudes (Eq. 30) exactly:
    the dyadic kernel is covariant under any orthogonal map.  A handedness
    slip (recomputing the circular basis in the swapped frame) fails this."""
    n = (6, 5, 7)
    h = 0.08
    rng = np.random.default_rng(31)
    eps = np.where(rng.uniform(size=n) < 0.5, rng.uniform(1.5, 4.0, n), 1.0)  # no mirror symmetry
    chs = [(c.khat, c.pol) for c in inputs.channels_metasurface([10.0])]      # L, R
    deg = np.array([-25.0, -10.0, 0.0, 10.0, 25.0])
    t = np.radians(deg)
    d_p = np.stack([np.sin(t), np.zeros_like(t), np.cos(t)], -1)
    W, _ = vie.solve_channels(n, h, K0, eps, chs, method="lu")
    F_p = np.stack([vie.farfield(W[r], n, h, K0, d_p) for r in range(2)])
    # the same problem on the swapped grid
    eps_g = np.ascontiguousarray(np.transpose(eps, inputs.PAPER_AXES))
    n_g = eps_g.shape
    chs_g = [(inputs.to_grid_frame(k), inputs.to_grid_frame(p)) for k, p in chs]
    W_g, _ = vie.solve_channels(n_g, h, K0, eps_g, chs_g, method="lu")
    F_g = np.stack([vie.farfield(W_g[r], n_g, h, K0, inputs.to_grid_frame(d_p)) for r in range(2)])
    F_back = inputs.to_grid_frame(F_g)
    assert np.abs(F_back - F_p).max() <= 1e-10 * np.abs(F_p).max()
    # circular amplitudes in the paper frame agree; in the swapped frame's own basis they do not
    C_p = np.stack([vie.project(F_p[r], d_p, 2) for r in range(2)])
    C_b = np.stack([vie.project(F_back[r], d_p, 2) for r in range(2)])
    assert np.abs(C_b - C_p).max() <= 1e-10 * np.abs(C_p).max()
    C_wrong = np.stack([vie.project(F_g[r], inputs.to_grid_frame(d_p), 2) for r in range(2)])
    assert np.abs(C_wrong - C_p).max() > 1e-3 * np.abs(C_p).max()


def test_bench_circular_projection_matches_eq30():
    """The paper-scale bench mode takes the circular components (Eq. 30) of
    paper-frame far fields itself; they must equal the oracle's projection
    onto (E_L, E_R) at the same signed xz-plane directions."""
    import bench
    rng = np.random.default_rng(4)
    deg = np.arange(-30.0, 30.0 + 1e-9, 7.5)
    t = np.radians(deg)
    d = np.stack([np.sin(t), np.zeros_like(t), np.cos(t)], -1)
    F = rng.standard_normal((2, len(deg), 3)) + 1j * rng.standard_normal((2, len(deg), 3))
    F = F - d[None] * np.sum(F * d[None], axis=-1, keepdims=True)  # transverse
    got = bench.circular_components(F, deg)
    for r in range(2):
        ref = vie.project(F[r], d, 2)[:, :2]
        assert np.abs(got[r] - ref).max() <= 1e-13 * np.abs(ref).max()
