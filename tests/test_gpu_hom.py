"""Two-photon observables from the library (host scalar entry point and the
device map kernel) against the oracle's Eq. 10 / Eqs. 18-22 / Eq. 27."""
import numpy as np
import pytest

from oracle import hom as ohom

pytestmark = pytest.mark.gpu


def test_hom_transfer_matches_oracle(vielib):
    rng = np.random.default_rng(0)
    dt = np.linspace(-4, 4, 33)
    for _ in range(50):
        E = rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))
        om = rng.uniform(0.5, 2.0, 2)
        g2, nc, vis, code = vielib.hom_transfer(E, omega=om, sigma=1.2, dtau=dt)
        assert code == 0
        assert abs(g2 - ohom.g2_degenerate(E, om)) < 1e-12
        assert np.abs(nc - ohom.coincidence_closed(E, dt, 1.2, om)).max() < 1e-12
        assert abs(vis - ohom.visibility(E, 1.2, om)) < 1e-12


def test_hom_transfer_undefined(vielib):
    E = np.array([[0.3, 0.0], [0.2j, 0.0]])
    g2, nc, vis, code = vielib.hom_transfer(E, dtau=[0.0])
    assert code == vielib.VIE_EUNDEF and g2 == 0.0 and np.isnan(nc[0]) and np.isnan(vis)


def test_hom_map_device(vielib):
    rng = np.random.default_rng(1)
    nA, nB = 37, 53
    Ea = rng.standard_normal((2, nA)) + 1j * rng.standard_normal((2, nA))
    Eb = rng.standard_normal((2, nB)) + 1j * rng.standard_normal((2, nB))
    g2, vis, p2 = vielib.hom_map(Ea, Eb)
    ref_g2 = np.array([[ohom.g2_degenerate([[Ea[0, i], Ea[1, i]], [Eb[0, j], Eb[1, j]]])
                        for j in range(nB)] for i in range(nA)])
    ref_v = np.array([[ohom.visibility([[Ea[0, i], Ea[1, i]], [Eb[0, j], Eb[1, j]]])
                       for j in range(nB)] for i in range(nA)])
    ref_p = np.array([[ohom.classical_p2((Ea[0, i], Ea[1, i]), (Eb[0, j], Eb[1, j]))
                       for j in range(nB)] for i in range(nA)])
    ref_p /= ref_p.max()
    assert np.abs(g2 - ref_g2).max() < 1e-12
    assert np.abs(vis - ref_v).max() < 1e-12
    assert np.abs(p2 - ref_p).max() < 1e-12
