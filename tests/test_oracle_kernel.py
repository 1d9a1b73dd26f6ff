"""Pins of the oracle's Green's tensor and discrete kernel (Sec. II-C,
Eq. dyadicG) against independent mathematics: finite differences, ball
quadrature, static limits and symmetry."""
import math

import numpy as np
import pytest

from oracle import vie

K0 = 2.0 * math.pi


def scalar_g(R, k):
    r = np.linalg.norm(R)
    return np.exp(1j * k * r) / (4.0 * math.pi * r)


@pytest.mark.parametrize("R", [(0.3, 0.1, -0.2), (0.05, 0.0, 0.0), (1.1, -0.7, 0.4), (0.0, 0.2, 0.2)])
def test_green_closed_form_matches_finite_differences(R):
    """(I + grad grad / k^2) g by 4th-order central differences of the scalar
    Green's function: catches a dropped term or wrong sign in the closed form."""
    R = np.asarray(R, float)
    k = K0
    d = 1e-3 * max(np.linalg.norm(R), 0.05)
    H = np.zeros((3, 3), complex)
    e = np.eye(3)
    f = lambda p: scalar_g(p, k)
    for i in range(3):
        for j in range(3):
            if i == j:
                H[i, i] = (-f(R + 2 * d * e[i]) + 16 * f(R + d * e[i]) - 30 * f(R)
                           + 16 * f(R - d * e[i]) - f(R - 2 * d * e[i])) / (12 * d * d)
            else:
                s = 0
                for a, b, w in ((1, 1, 1), (1, -1, -1), (-1, 1, -1), (-1, -1, 1)):
                    s += w * f(R + a * d * e[i] + b * d * e[j])
                H[i, j] = s / (4 * d * d)
    G_fd = f(R) * np.eye(3) + H / k ** 2
    G = vie.green_dyadic(R, k)
    G_cf = np.array([[G[vie.CIDX[i][j]] for j in range(3)] for i in range(3)])
    assert np.abs(G_cf - G_fd).max() <= 2e-5 * np.abs(G_cf).max()


def _ball_nodes(a, nr=24, nt=24):
    """Product Gauss rule on a ball of radius a: GL in r (r^2 weight) x GL in
    cos(theta) x trapezoid in phi."""
    xr, wr = np.polynomial.legendre.leggauss(nr)
    r = 0.5 * a * (xr + 1.0)
    wr = 0.5 * a * wr * r ** 2
    xc, wc = np.polynomial.legendre.leggauss(nt)
    nph = 2 * nt
    ph = 2 * math.pi * np.arange(nph) / nph
    pts, wts = [], []
    for ri, wri in zip(r, wr):
        for ci, wci in zip(xc, wc):
            s = math.sqrt(1 - ci * ci)
            for p in ph:
                pts.append(ri * np.array([s * math.cos(p), s * math.sin(p), ci]))
                wts.append(wri * wci * 2 * math.pi / nph)
    return np.array(pts), np.array(wts)


def test_mean_value_factor_is_ball_average_of_helmholtz_solutions():
    h = 0.07
    a = vie.equivalent_radius(h)
    pts, wts = _ball_nodes(a)
    vol = 4.0 / 3.0 * math.pi * a ** 3
    assert abs(wts.sum() - vol) < 1e-12 * vol
    kap = vie.mean_value_factor(K0 * a)
    # plane wave
    u = np.exp(1j * K0 * pts[:, 2])
    assert abs(np.sum(wts * u) / vol - kap) < 1e-12
    # outgoing spherical wave from a source one cell away
    src = np.array([h, 0.0, 0.0])
    g = np.array([scalar_g(p - src, K0) for p in pts])
    avg = np.sum(wts * g) / vol
    assert abs(avg - kap * scalar_g(-src, K0)) < 1e-9 * abs(scalar_g(src, K0))


def test_self_term_static_limit_and_radiative_part():
    # static limit: depolarisation dyad -I/3
    assert abs(vie.self_term(K0, 1e-6) - (-1.0 / 3.0)) < 1e-9
    # Im K(0) = kappa (2/9) (k a)^3 = kappa k^3 V / (6 pi)
    for h in (0.01, 0.05, 0.1):
        a = vie.equivalent_radius(h)
        ka = K0 * a
        kap = vie.mean_value_factor(ka)
        assert abs(vie.self_term(K0, h).imag - kap * 2.0 / 9.0 * ka ** 3) < 1e-14
        assert abs(kap * 2.0 / 9.0 * ka ** 3 - kap * K0 ** 3 * h ** 3 / (6 * math.pi)) < 1e-14


def test_self_term_imaginary_part_is_ball_integral_of_im_g():
    """Im of k^2 int_ball G dV by quadrature of the (regular) imaginary part."""
    h = 0.08
    a = vie.equivalent_radius(h)
    pts, wts = _ball_nodes(a, nr=16, nt=16)
    G = vie.green_dyadic(pts, K0)
    ImGxx = np.sum(wts * G[:, 0].imag) * K0 ** 2
    ImGxy = np.sum(wts * G[:, 1].imag) * K0 ** 2
    assert abs(ImGxx - vie.self_term(K0, h).imag) < 1e-10
    assert abs(ImGxy) < 1e-10


def test_kernel_parity_and_symmetry():
    m = np.array([[2, -1, 3], [1, 1, 0], [0, 0, 4]])
    h = 0.05
    K = vie.kernel_at(m, h, K0)
    Km = vie.kernel_at(-m, h, K0)
    assert np.allclose(K, Km, rtol=0, atol=1e-15 * np.abs(K).max())
    # reflection x -> -x flips xy and xz, keeps the rest
    mr = m * np.array([-1, 1, 1])
    Kr = vie.kernel_at(mr, h, K0)
    sgn = np.array([1, -1, -1, 1, 1, 1])
    assert np.allclose(Kr, K * sgn, rtol=0, atol=1e-15 * np.abs(K).max())
    # isotropy: trace of the far-zone Green's tensor of a rotated offset is unchanged
    K1 = vie.kernel_at(np.array([3, 4, 0]), h, K0)
    K2 = vie.kernel_at(np.array([0, 0, 5]), h, K0)
    assert abs((K1[0] + K1[3] + K1[5]) - (K2[0] + K2[3] + K2[5])) < 1e-14


def test_kernel_table_indexing():
    n = (3, 4, 2)
    h = 0.1
    T = vie.kernel_table(n, h, K0)
    assert T.shape == (6, 5, 7, 3)
    for m in ([0, 0, 0], [-2, 3, 1], [1, -3, -1]):
        idx = tuple(np.array(m) + np.array(n) - 1)
        assert np.allclose(T[(slice(None),) + idx], vie.kernel_at(np.array(m), h, K0))
