"""The stored oracle far fields (tests/golden/*_farfield.npz, written by
tests/golden/make_golden.py from the oracle alone) checked against physics
that fixes them independently of any solver: the optical theorem of a
lossless body, (4 pi / k0) Im(p* . F(k)) = integral of |F|^2 over the sphere
(exact in the discrete model, so only the quadrature of the stored grid and
the 1e-10 solve limit it), and the records of the run that wrote them."""
import math
import os

import numpy as np
import pytest

from paper_2508_16471_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")
K0 = 2.0 * math.pi


def _load(name):
    p = os.path.join(GOLD, f"{name}_farfield.npz")
    if not os.path.exists(p):
        pytest.fail(f"missing stored oracle result {p}: run tests/golden/make_golden.py {name}")
    return np.load(p)


def _sphere_integral(F, th, ph):
    """Integral of |F_theta|^2 + |F_phi|^2 over the sphere on a product grid
    theta = 0..pi (inclusive), phi uniform over [0, 2 pi): composite Simpson in
    theta (sin(theta) weight), the periodic trapezoid (exact for band-limited
    data) in phi."""
    p = np.sum(np.abs(F) ** 2, axis=-1)  # [nt][np]
    ring = p.mean(axis=1) * 2.0 * math.pi * np.sin(th)
    nt = len(th)
    assert nt % 2 == 1
    w = np.ones(nt)
    w[1:-1:2], w[2:-1:2] = 4.0, 2.0
    return float(np.sum(w * ring) * (th[1] - th[0]) / 3.0)


@pytest.mark.parametrize("name", ["sphere64", "body64"])
def test_stored_oracle_farfields_satisfy_the_optical_theorem(name):
    gold = _load(name)
    F, th, ph = gold["F_theta_phi"].astype(np.complex128), gold["theta"], gold["phi"]
    assert np.all(gold["relres"] <= 1e-10) and float(gold["tol"]) <= 1e-10
    assert F.shape[0] == len(gold["khat"]) == len(gold["F_forward"])
    for j, pol in enumerate(gold["pol"]):
        ext = 4.0 * math.pi / K0 * np.imag(np.conj(pol) @ gold["F_forward"][j])
        sca = _sphere_integral(F[j], th, ph)
        assert abs(ext - sca) <= 5e-5 * sca, (j, ext, sca)


def test_stored_sphere_farfield_forward_value_on_the_grid():
    """For the sphere's channels the forward direction lies on the stored grid:
    the grid value there equals the separately stored forward far field."""
    gold = _load("sphere64")
    F, th, ph = gold["F_theta_phi"].astype(np.complex128), gold["theta"], gold["phi"]
    for j, k in enumerate(gold["khat"]):
        t = math.acos(max(-1.0, min(1.0, k[2])))
        it = int(np.argmin(np.abs(th - t)))
        assert abs(th[it] - t) < 1e-9 and abs(math.atan2(k[1], k[0])) < 1e-12
        _, et, ep = inputs.spherical_basis(t, 0.0)
        Ff = gold["F_forward"][j]
        assert abs(F[j, it, 0, 0] - et @ Ff) <= 1e-6 * np.abs(Ff).max()
        assert abs(F[j, it, 0, 1] - ep @ Ff) <= 1e-6 * np.abs(Ff).max()
