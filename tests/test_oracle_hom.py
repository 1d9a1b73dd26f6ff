"""Pins of the oracle's two-photon observables (Sec. II-A/B): Eq. 10 against
a brute-force Fock-space evaluation of Eq. 11, the permanent law for unitary
transfer matrices, the beam-splitter reduction of Eq. G2_scatter to Eq. 17,
the closed-form coincidence curve against tau-quadrature, bounds, limits and
invariances."""
import math

import numpy as np
import pytest

from oracle import hom


def _rand_E(rng):
    return rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))


def test_eq10_equals_brute_force_eq11():
    rng = np.random.default_rng(0)
    for _ in range(20):
        E = _rand_E(rng)
        assert abs(hom.g2_degenerate(E) - hom.g2_fock(E)) < 1e-12
        om = rng.uniform(0.5, 2.0, 2)
        assert abs(hom.g2_degenerate(E, om) - hom.g2_fock(E, om)) < 1e-12


def test_bounds_0_1():
    rng = np.random.default_rng(1)
    for _ in range(500):
        g = hom.g2_degenerate(_rand_E(rng), rng.uniform(0.2, 3.0, 2))
        assert -1e-15 <= g <= 1 + 1e-12


def _random_unitary(rng):
    z = rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def test_unitary_transfer_gives_permanent():
    """For a unitary 2x2 transfer, g2 = |perm U|^2, the textbook probability of
    one photon in each output port of a lossless two-mode network."""
    rng = np.random.default_rng(2)
    for _ in range(20):
        U = _random_unitary(rng)
        perm = U[0, 0] * U[1, 1] + U[0, 1] * U[1, 0]
        assert abs(hom.g2_degenerate(U) - abs(perm) ** 2) < 1e-12


def test_beam_splitter_reduction():
    """A_dir = T, A_ex = -R (Eq. 17): g2 = (T - R)^2, N~c(0) = 1 - 2TR/(T^2+R^2)."""
    for Tt in (0.5, 0.3, 0.8):
        R = 1 - Tt
        E = np.array([[math.sqrt(Tt), 1j * math.sqrt(R)], [1j * math.sqrt(R), math.sqrt(Tt)]])
        assert abs(hom.g2_degenerate(E) - (Tt - R) ** 2) < 1e-14
        Ad, Ae = hom.path_amplitudes(E)
        assert abs(Ad - Tt) < 1e-15 and abs(Ae + R) < 1e-15
        nc0 = hom.coincidence_closed(E, [0.0])[0]
        assert abs(nc0 - (1 - 2 * Tt * R / (Tt * Tt + R * R))) < 1e-14
    E = np.array([[1, 1j], [1j, 1]]) / math.sqrt(2)
    assert hom.visibility(E) == pytest.approx(1.0, abs=1e-14)


def test_coincidence_closed_form_matches_quadrature():
    rng = np.random.default_rng(4)
    dt = np.array([-3.0, -1.1, -0.2, 0.0, 0.4, 1.7, 4.0])
    for _ in range(5):
        E = _rand_E(rng)
        a = hom.coincidence_closed(E, dt, sigma=1.2)
        b = hom.coincidence_quadrature(E, dt, sigma=1.2)
        assert np.abs(a - b).max() < 1e-9


def test_coincidence_limits_and_range():
    rng = np.random.default_rng(5)
    for _ in range(50):
        E = _rand_E(rng)
        nc = hom.coincidence_closed(E, np.array([-1e3, -2.0, 0.0, 0.5, 1e3]))
        assert abs(nc[0] - 1) < 1e-14 and abs(nc[-1] - 1) < 1e-14
        assert np.all(nc >= -1e-14) and np.all(nc <= 2 + 1e-14)
        # N~c(0) = |A_dir + A_ex|^2 / (|A_dir|^2 + |A_ex|^2)
        Ad, Ae = hom.path_amplitudes(E)
        assert abs(nc[2] - abs(Ad + Ae) ** 2 / (abs(Ad) ** 2 + abs(Ae) ** 2)) < 1e-13


def test_trivial_single_path_zero():
    """Channel 2 absent at both detectors: g2 = 0 but N~c is undefined (0/0)."""
    E = np.array([[0.3 + 0.1j, 0.0], [0.7 - 0.2j, 0.0]])
    assert hom.g2_degenerate(E) == 0.0
    assert np.isnan(hom.coincidence_closed(E, [0.0])[0])
    # one path amplitude vanishing (A_ex = 0, A_dir != 0): flat N~c = 1
    E = np.array([[0.3, 0.0], [0.5, 0.4]])
    assert np.allclose(hom.coincidence_closed(E, [-1.0, 0.0, 1.0]), 1.0)


def test_invariances():
    rng = np.random.default_rng(6)
    for _ in range(10):
        E = _rand_E(rng)
        ph = np.exp(1j * rng.uniform(0, 2 * math.pi, 2))
        g0 = hom.g2_degenerate(E)
        assert abs(hom.g2_degenerate(E * ph[None, :]) - g0) < 1e-12
        assert abs(hom.g2_degenerate(E * (2.5 - 1.3j)) - g0) < 1e-12
        v0 = hom.visibility(E)
        assert abs(hom.visibility(E * ph[None, :]) - v0) < 1e-12


def test_classical_p2():
    E1 = (1.0 + 0j, 1.0j)
    E2 = (0.5, -0.5)
    assert hom.classical_p2(E1, E2) == pytest.approx(2.0 * 0.0)
    assert hom.classical_p2((1.0, 1.0), (1.0, 0.0)) == pytest.approx(4.0)
