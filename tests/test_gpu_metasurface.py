"""PB-phase metasurface workflow (Sec. III-B) at reduced size (2 x 2 fins on a
64 x 64 x 32 grid, h = p/32): circular-polarisation channels, circular
far-field components at detector angles theta in [-30, 30] deg in the xz-plane
(signed-angle reading), H/V by linearity of the solution in the incident
polarisation (Eq. 28), and the g_LR / visibility maps of Eq. 31 from the
device map kernel, checked against the oracle."""
import math

import numpy as np
import pytest

from oracle import hom as ohom
from oracle import vie as ovie
from paper_2508_16471_gb300 import inputs
from sample_points import pick_voxels

pytestmark = pytest.mark.gpu


def _dirs(deg, phi_sign):
    t = np.radians(deg)
    return np.stack([phi_sign * np.sin(t), np.zeros_like(t), np.cos(t)], -1)


def test_metasurface_reduced_glr_map(vielib):
    grid, eps, _ = inputs.metasurface(seed=0, n=(64, 64, 32), fins=(2, 2))
    k0 = 2 * math.pi
    LR = inputs.channels_metasurface([0.0])  # normal incidence: L then R
    HV = [(np.array([0, 0, 1.0]), np.array([1.0, 0, 0], complex)),   # H = e_theta at theta = 0
          (np.array([0, 0, 1.0]), np.array([0, 1.0, 0], complex))]   # V = e_phi
    chs = [(c.khat, c.pol) for c in LR] + HV
    deg = np.arange(-30.0, 30.0 + 1e-9, 2.0)
    d1 = _dirs(np.abs(deg), np.where(deg < 0, -1.0, 1.0))  # r1: signed angle, phi = 180 deg for negative
    d2 = _dirs(np.abs(deg), np.where(deg < 0, -1.0, 1.0))
    with vielib.Handle(grid.n, grid.h, eps, k0) as hd:
        st = hd.solve(chs, tol=1e-8, restart=128, max_iter=20000)
        assert st["converged"] == 4
        W = np.stack([hd.get_current(r) for r in range(4)])
        C1 = hd.farfield_dirs(d1, basis=vielib.BASIS_CIRC)  # [4][D][3]: (F_L, F_R, F_r)
    s2 = math.sqrt(2.0)
    # linearity: H = (L + R)/sqrt2, V = (L - R)/(i sqrt2)  (inverse of Eq. 28)
    assert np.abs(C1[2] - (C1[0] + C1[1]) / s2).max() <= 1e-6 * np.abs(C1[2]).max()
    assert np.abs(C1[3] - (C1[0] - C1[1]) / (1j * s2)).max() <= 1e-6 * np.abs(C1[3]).max()
    # F_r vanishes (transverse far field)
    assert np.abs(C1[:, :, 2]).max() <= 1e-9 * np.abs(C1[:, :, :2]).max()
    # oracle far field of the GPU currents in the circular basis
    for r in range(4):
        F_or = ovie.project(ovie.farfield(W[r], grid.n, grid.h, k0, d1), d1, 2)
        assert np.linalg.norm(C1[r] - F_or) <= 1e-8 * np.linalg.norm(F_or)
    # Eq. 31: channels H, V; detector a = R at r1, detector b = L at r2
    Ea = np.stack([C1[2][:, 1], C1[3][:, 1]])
    Eb = np.stack([C1[2][:, 0], C1[3][:, 0]])
    g2, vis, p2 = vielib.hom_map(Ea, Eb)
    for i in range(0, len(deg), 7):
        for j in range(0, len(deg), 5):
            E = [[Ea[0, i], Ea[1, i]], [Eb[0, j], Eb[1, j]]]
            assert abs(g2[i, j] - ohom.g2_degenerate(E)) < 1e-12
            assert abs(vis[i, j] - ohom.visibility(E)) < 1e-12
    assert np.all((g2 >= -1e-14) & (g2 <= 1 + 1e-12))
    assert abs(p2.max() - 1.0) < 1e-14


def test_metasurface_full_size(vielib):
    """The full PB-phase configuration: 8 x 8 fins on the 256 x 256 x 32 grid,
    32 incidence angles x L/R (64 RHS) in one batched mixed-precision solve to
    an FP64 residual of 1e-6.  Checked against the oracle: its equation at
    32 fin voxels (the extreme ones, the ones nearest the grid corners, surface
    and random ones) for the two channels at theta_s = +1 deg, the far field
    of those currents, and the g_LR / visibility map of Eq. 31 (H/V by
    linearity, Eq. 28) at sampled detector pairs."""
    grid, eps, _ = inputs.metasurface(seed=0)
    k0 = 2 * math.pi
    chs = [(c.khat, c.pol) for c in inputs.channels_metasurface()]
    assert len(chs) == 64
    iL, iR = 32, 33  # theta_s = +1 deg
    deg = np.arange(-30.0, 30.0 + 1e-9, 0.5)
    d = _dirs(np.abs(deg), np.where(deg < 0, -1.0, 1.0))
    with vielib.Handle(grid.n, grid.h, eps, k0) as hd:
        st = hd.solve(chs, tol=1e-6, restart=128, max_iter=20000)
        assert st["converged"] == 64 and st["relres_max"] <= 1e-6
        W = np.stack([hd.get_current(r) for r in (iL, iR)])
        C = hd.farfield_dirs(d, basis=vielib.BASIS_CIRC)[[iL, iR]]  # [2][D][3]
    # the oracle's equation at sampled fin voxels
    chi = ovie.contrast(eps)
    body = np.argwhere(chi > 0)
    pts = pick_voxels(chi > 0, 32, 3)
    conv = ovie.convolve_points_sparse(body, W[:, :, body[:, 0], body[:, 1], body[:, 2]], grid.h, k0, pts)
    for q, r in enumerate((iL, iR)):
        b = ovie.rhs(chi, ovie.incident_field(grid.n, grid.h, k0, *chs[r]))
        res = np.array([[W[q][c][tuple(p)] - chi[tuple(p)] * conv[q, c, i] - b[c][tuple(p)] for c in range(3)]
                        for i, p in enumerate(pts)])
        assert np.abs(res).max() <= 1.05e-6 * np.linalg.norm(b)
    # far field of the GPU currents at every 10th detector direction
    sel = np.arange(0, len(deg), 10)
    for q in range(2):
        F_or = ovie.project(ovie.farfield(W[q], grid.n, grid.h, k0, d[sel]), d[sel], 2)
        assert np.linalg.norm(C[q][sel] - F_or) <= 1e-8 * np.linalg.norm(F_or)
    # Eq. 31 map: channels H = (L + R)/sqrt2, V = (L - R)/(i sqrt2); a = R at r1, b = L at r2
    s2 = math.sqrt(2.0)
    H = (C[0] + C[1]) / s2
    Vv = (C[0] - C[1]) / (1j * s2)
    Ea = np.stack([H[:, 1], Vv[:, 1]])
    Eb = np.stack([H[:, 0], Vv[:, 0]])
    g2, vis, p2 = vielib.hom_map(Ea, Eb)
    assert g2.shape == (len(deg), len(deg))
    for i in range(0, len(deg), 17):
        for j in range(0, len(deg), 13):
            E = [[Ea[0, i], Ea[1, i]], [Eb[0, j], Eb[1, j]]]
            assert abs(g2[i, j] - ohom.g2_degenerate(E)) < 1e-12
            assert abs(vis[i, j] - ohom.visibility(E)) < 1e-12
    assert np.all((g2 >= -1e-14) & (g2 <= 1 + 1e-12))
