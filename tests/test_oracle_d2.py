"""Pins of the oracle's rooftop / pulse-tested discretisation (D2): the FFT
operator against brute-force direct sums, the complex symmetry of the discrete
operator (reciprocity of the Galerkin-like scheme), exact far-field
reciprocity of its solutions, and convergence to the Mie series."""
import math

import numpy as np

from oracle import d2, mie, vie
from paper_2508_16471_gb300 import inputs

K0 = 2.0 * math.pi


def test_fft_operator_matches_direct_sums():
    rng = np.random.default_rng(0)
    n, h = (3, 4, 5), 0.07
    chi = rng.uniform(0.0, 3.0, n) * (rng.uniform(size=n) < 0.7)
    w = (rng.standard_normal((3,) + n) + 1j * rng.standard_normal((3,) + n)) * (d2.face_contrast(chi) > 0)
    op = d2.FFTOperator(n, h, K0, chi)
    y_fft = op(w)
    y_dir = d2.apply_direct(n, h, K0, d2.face_contrast(chi), w)
    assert np.abs(y_fft - y_dir).max() <= 1e-12 * np.abs(y_dir).max()


def test_operator_is_complex_symmetric():
    """K_ab(c, c') = K_ba(c', c): u^T (K v) = v^T (K u) for any u, v."""
    rng = np.random.default_rng(1)
    n, h = (4, 3, 5), 0.05
    op = d2.FFTOperator(n, h, K0, np.ones(n))
    u = rng.standard_normal((3,) + n) + 1j * rng.standard_normal((3,) + n)
    v = rng.standard_normal((3,) + n) + 1j * rng.standard_normal((3,) + n)
    a = np.sum(u * op.kernel_apply(v))
    b = np.sum(v * op.kernel_apply(u))
    assert abs(a - b) <= 1e-12 * abs(a)


def test_scalar_kernel_self_term_small_ball():
    """G_h(0) is the ball integral of g: a^2/2 + i k a^3/3 + O(k^2 a^4)."""
    h = 1e-3
    a = vie.equivalent_radius(h)
    g0 = d2.scalar_kernel(np.zeros(3, dtype=np.int64), h, K0)
    ref = a * a / 2 + 1j * K0 * a ** 3 / 3
    assert abs(g0 - ref) <= 1e-4 * abs(ref)


def test_farfield_reciprocity_of_solutions():
    """p2 . F(-k2; k1, p1) = p1 . F(-k1; k2, p2) for a random body."""
    g, eps = inputs.random_body(3, n_axis=8, h=0.06)
    k1, k2 = np.array([0.0, 0.6, 0.8]), np.array([1.0, 0.0, 0.0])
    p1, p2 = np.array([1.0, 0.0, 0.0], complex), np.array([0.0, 0.8, -0.6], complex)
    W, infos = d2.solve(g.n, g.h, K0, eps, [(k1, p1), (k2, p2)], tol=1e-13)
    F12 = d2.farfield(W[0], g.n, g.h, K0, -k2[None])[0]
    F21 = d2.farfield(W[1], g.n, g.h, K0, -k1[None])[0]
    a, b = p2 @ F12, p1 @ F21
    assert abs(a - b) <= 1e-10 * abs(a)


def test_converges_to_mie():
    """Sphere R = 0.3 lambda, eps_r = 2.1 (one empty cell layer around it),
    x-polarised along +z: the far-field error against Mie falls to ~1.5 % at
    24 cells across the diameter."""
    th = np.radians(np.arange(0, 181, 10.0))
    ph = np.radians(np.arange(0, 356, 20.0))
    T, P = np.meshgrid(th, ph, indexing="ij")
    T, P = T.ravel(), P.ravel()
    dirs = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], -1)
    R = 0.3
    Fm = mie.farfield(R, 2.1, K0, T, P)
    errs = []
    for N in (12, 24):
        h = 2 * R / N
        g = inputs.Grid((N + 2,) * 3, h)
        eps = inputs.sphere(g, R, 2.1)
        W, _ = d2.solve(g.n, h, K0, eps, [((0, 0, 1.0), (1.0, 0, 0))], tol=1e-10)
        F = d2.farfield(W[0], g.n, h, K0, dirs)
        errs.append(np.linalg.norm(F - Fm) / np.linalg.norm(Fm))
    assert errs[0] < 0.05 and errs[1] < 0.02 and errs[1] < errs[0]
