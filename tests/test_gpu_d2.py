"""GPU parity of the rooftop / pulse-tested discretisation (D2) against the
oracle's D2 (``oracle/d2.py``): the operator on small ragged grids (generic
and power-of-two FFT paths, FP64 and FP32), a sphere solve (currents and far
fields), and the paper's Mie validation case solved with D2."""
import json
import math
import os

import numpy as np
import pytest

from oracle import d2 as od2
from oracle import hom as ohom
from oracle import mie as omie
from oracle import vie as ovie
from paper_2508_16471_gb300 import inputs

pytestmark = pytest.mark.gpu
K0 = 2.0 * math.pi
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


def _support(chi):
    return np.any(od2.face_contrast(chi) > 0, axis=0)


@pytest.mark.parametrize("n", [(5, 6, 7), (8, 8, 8), (12, 10, 9)])
def test_d2_operator_matches_oracle(vielib, n):
    rng = np.random.default_rng(sum(n))
    h = 0.05
    eps = np.where(rng.uniform(size=n) < 0.5, rng.uniform(1.5, 5.0, n), 1.0)
    eps[0] = 1.0  # empty first layer along x (faces below it are not represented)
    chi = ovie.contrast(eps)
    S = _support(chi)
    w = (rng.standard_normal((2, 3) + n) + 1j * rng.standard_normal((2, 3) + n)) * S
    ref = np.stack([od2.apply_direct(n, h, K0, od2.face_contrast(chi), w[r]) for r in range(2)])
    with vielib.Handle(n, h, eps, K0, disc=vielib.DISC_D2) as hd:
        y64 = hd.apply(w, precision=vielib.PREC_FP64)
        y32 = hd.apply(w, precision=vielib.PREC_MIXED)
    s = np.abs(ref).max()
    assert np.abs(y64 - ref).max() <= 1e-11 * s
    assert np.abs(y32 - ref).max() <= 2e-5 * s


def test_d2_operator_long_axis(vielib):
    """D2 with a padded z length of 4410 (generic line kernels, twiddles from
    global memory), against the oracle's FFT form of the D2 operator."""
    n = (3, 4, 2200)
    rng = np.random.default_rng(5)
    h = 0.02
    eps = np.where(rng.uniform(size=n) < 0.5, rng.uniform(1.5, 5.0, n), 1.0)
    eps[0] = 1.0
    chi = ovie.contrast(eps)
    S = _support(chi)
    w = (rng.standard_normal((2, 3) + n) + 1j * rng.standard_normal((2, 3) + n)) * S
    op = od2.FFTOperator(n, h, K0, chi, workers=-1)
    ref = np.stack([op(w[r]) for r in range(2)])
    with vielib.Handle(n, h, eps, K0, disc=vielib.DISC_D2) as hd:
        assert hd.info()["P"][2] > 4096
        y64 = hd.apply(w, precision=vielib.PREC_FP64)
        y32 = hd.apply(w, precision=vielib.PREC_MIXED)
    s = np.abs(ref).max()
    assert np.abs(y64 - ref).max() <= 1e-11 * s
    assert np.abs(y32 - ref).max() <= 2e-5 * s


def test_d2_sphere_solve_matches_oracle(vielib):
    N, R = 16, 0.3
    h = 2 * R / N
    g = inputs.Grid((N + 2,) * 3, h)
    eps = inputs.sphere(g, R, 2.25)
    chs = [((0, 0, 1.0), (1.0, 0, 0)), ((1.0, 0, 0), (0, 0, 1.0))]
    W_or, infos = od2.solve(g.n, h, K0, eps, chs, tol=1e-12)
    assert all(i["converged"] for i in infos)
    th, ph = np.radians(np.arange(0, 181, 15.0)), np.radians(np.arange(0, 360, 30.0))
    T, P = np.meshgrid(th, ph, indexing="ij")
    dirs = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], -1).reshape(-1, 3)
    with vielib.Handle(g.n, h, eps, K0, disc=vielib.DISC_D2) as hd:
        st = hd.solve(chs, tol=1e-10, restart=40)
        assert st["converged"] == 2
        W = np.stack([hd.get_current(r) for r in range(2)])
        Fd = hd.farfield_dirs(dirs)
        Fg = hd.farfield(th, ph).reshape(2, -1, 3)
        # COCR on the face unknowns (weights 1/chi_f; faces with chi_f = 0 stay zero)
        st = hd.solve(chs, tol=1e-10, restart=4, solver=vielib.SOLVER_COCR)
        assert st["converged"] == 2
        Wc = np.stack([hd.get_current(r) for r in range(2)])
    assert np.abs(W - W_or).max() <= 1e-8 * np.abs(W_or).max()
    assert np.abs(Wc - W_or).max() <= 1e-8 * np.abs(W_or).max()
    F_or = np.stack([od2.farfield(W_or[j], g.n, h, K0, dirs) for j in range(2)])
    assert np.linalg.norm(Fd - F_or) <= 1e-8 * np.linalg.norm(F_or)
    assert np.linalg.norm(Fg - F_or) <= 1e-5 * np.linalg.norm(F_or)


@pytest.mark.parametrize("idx", [0, 1, 2])
def test_d2_sphere_g2_against_mie(vielib, idx):
    """The paper's validation case (Sec. III-A) with the D2 discretisation on
    64 cells across the diameter (one empty cell layer around the sphere);
    the relative l2 error of g2_zz against Mie is printed beside the paper's."""
    G = GOLD["sphere_g2_validation"]
    lam_nm = 299792.458 / G["freq_THz"]
    r = G["radii_nm"][idx] / lam_nm
    N = 64
    grid = inputs.Grid((N + 2,) * 3, 2.0 * r / N)
    eps = inputs.sphere(grid, r, G["eps_r"])
    chs = [((1.0, 0.0, 0.0), (0.0, 1.0, 0.0)), ((0.0, 1.0, 0.0), (1.0, 0.0, 0.0))]
    phi1 = np.radians(np.arange(G["phi1_deg"][0], G["phi1_deg"][1] + 1e-9, 1.0))
    t1 = np.radians(G["theta1_deg"])
    d1 = np.stack([np.sin(t1) * np.cos(phi1), np.sin(t1) * np.sin(phi1), np.full_like(phi1, np.cos(t1))], -1)
    t2, p2 = np.radians(G["theta2_deg"]), np.radians(G["phi2_deg"])
    d2v = np.array([[np.sin(t2) * np.cos(p2), np.sin(t2) * np.sin(p2), np.cos(t2)]])
    with vielib.Handle(grid.n, grid.h, eps, K0, disc=vielib.DISC_D2) as hd:
        st = hd.solve(chs, tol=1e-9, restart=64, max_iter=20000)
        assert st["converged"] == 2
        F1 = hd.farfield_dirs(d1)
        F2 = hd.farfield_dirs(d2v)
    g2, _, _ = vielib.hom_map(np.stack([F1[0][:, 2], F1[1][:, 2]]), np.stack([F2[0][:, 2], F2[1][:, 2]]))
    g2 = g2[:, 0]
    M1 = [omie.farfield_general(r, G["eps_r"], K0, k, p, d1) for k, p in chs]
    M2 = [omie.farfield_general(r, G["eps_r"], K0, k, p, d2v) for k, p in chs]
    ref = np.array([ohom.g2_degenerate([[M1[0][i, 2], M1[1][i, 2]], [M2[0][0, 2], M2[1][0, 2]]])
                    for i in range(len(phi1))])
    err = np.linalg.norm(g2 - ref) / np.linalg.norm(ref)
    print(f"D2 sphere r = {G['radii_nm'][idx]:.0f} nm: g2_zz relative l2 error vs Mie {100 * err:.2f} % "
          f"(paper: {G['rel_l2_err_pct'][idx]:.2f} %)")
    assert err < 0.05
