"""Mie series for a homogeneous dielectric sphere (test infrastructure only).

Only ``tests/`` may import this module.  It validates the physics of the
discrete model (it is not a parity pin): the far field of a sphere of radius a,
relative permittivity eps_r, illuminated by an x-polarised plane wave along +z
with exp(-i omega t), written from the standard Lorenz-Mie solution (Bohren &
Huffman, ch. 4):

  a_n = [m psi_n(mx) psi_n'(x) - psi_n(x) psi_n'(mx)] /
        [m psi_n(mx) xi_n'(x)  - xi_n(x)  psi_n'(mx)]
  b_n = [psi_n(mx) psi_n'(x) - m psi_n(x) psi_n'(mx)] /
        [psi_n(mx) xi_n'(x)  - m xi_n(x)  psi_n'(mx)]
  S1 = sum (2n+1)/(n(n+1)) (a_n pi_n + b_n tau_n)
  S2 = sum (2n+1)/(n(n+1)) (a_n tau_n + b_n pi_n)

with psi_n(r) = r j_n(r), xi_n(r) = r h_n^(1)(r), x = k a, m = sqrt(eps_r), and
F(theta, phi) = (i/k) [S2 cos(phi) e_theta - S1 sin(phi) e_phi] so that
E_sca ~ F exp(ikr)/r.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import spherical_jn, spherical_yn


def _psi(n, z):
    return z * spherical_jn(n, z)


def _dpsi(n, z):
    return spherical_jn(n, z) + z * spherical_jn(n, z, derivative=True)


def _xi(n, z):
    return z * (spherical_jn(n, z) + 1j * spherical_yn(n, z))


def _dxi(n, z):
    h = spherical_jn(n, z) + 1j * spherical_yn(n, z)
    dh = spherical_jn(n, z, derivative=True) + 1j * spherical_yn(n, z, derivative=True)
    return h + z * dh


def coefficients(x, m, nmax=None):
    """Mie coefficients a_n, b_n for n = 1..nmax (Wiscombe's nmax by default)."""
    if nmax is None:
        nmax = int(math.ceil(x + 4.05 * x ** (1.0 / 3.0) + 2.0))
    n = np.arange(1, nmax + 1)
    mx = m * x
    a = (m * _psi(n, mx) * _dpsi(n, x) - _psi(n, x) * _dpsi(n, mx)) / \
        (m * _psi(n, mx) * _dxi(n, x) - _xi(n, x) * _dpsi(n, mx))
    b = (_psi(n, mx) * _dpsi(n, x) - m * _psi(n, x) * _dpsi(n, mx)) / \
        (_psi(n, mx) * _dxi(n, x) - m * _xi(n, x) * _dpsi(n, mx))
    return n, a, b


def angular(nmax, mu):
    """pi_n(mu) and tau_n(mu), n = 1..nmax, by upward recurrence."""
    mu = np.asarray(mu, float)
    pi = np.zeros((nmax + 1,) + mu.shape)
    tau = np.zeros((nmax + 1,) + mu.shape)
    pi[1] = 1.0
    if nmax >= 2:
        pi[2] = 3.0 * mu
    for n in range(3, nmax + 1):
        pi[n] = ((2 * n - 1) * mu * pi[n - 1] - n * pi[n - 2]) / (n - 1)
    for n in range(1, nmax + 1):
        tau[n] = n * mu * pi[n] - (n + 1) * pi[n - 1]
    return pi[1:], tau[1:]


def amplitudes(x, m, theta):
    """S1(theta), S2(theta)."""
    n, a, b = coefficients(x, m)
    pi, tau = angular(len(n), np.cos(theta))
    f = ((2 * n + 1) / (n * (n + 1)))[:, None]
    pi = pi.reshape(len(n), -1)
    tau = tau.reshape(len(n), -1)
    S1 = np.sum(f * (a[:, None] * pi + b[:, None] * tau), axis=0)
    S2 = np.sum(f * (a[:, None] * tau + b[:, None] * pi), axis=0)
    return S1, S2


def farfield(radius, eps_r, k0, theta, phi):
    """Cartesian far field F (D, 3) for x-polarised incidence along +z."""
    theta = np.asarray(theta, float).reshape(-1)
    phi = np.asarray(phi, float).reshape(-1)
    S1, S2 = amplitudes(k0 * radius, math.sqrt(eps_r), theta)
    Ft = (1j / k0) * S2 * np.cos(phi)
    Fp = -(1j / k0) * S1 * np.sin(phi)
    eth = np.stack([np.cos(theta) * np.cos(phi), np.cos(theta) * np.sin(phi), -np.sin(theta)], -1)
    eph = np.stack([-np.sin(phi), np.cos(phi), np.zeros_like(phi)], -1)
    return Ft[:, None] * eth + Fp[:, None] * eph


def farfield_general(radius, eps_r, k0, khat, pol, dirs):
    """Cartesian far field F (D, 3) for a plane wave along unit ``khat`` with
    polarisation ``pol`` (transverse), by rotational symmetry of the sphere:
    with the scattering plane spanned by khat and the direction r, e_perp =
    khat x r / |khat x r|, the incident parallel axis e_perp x khat and the
    scattered one e_perp x r,
        F = (i/k0) [S2(Theta) (pol . e_perp x khat) e_perp x r + S1(Theta) (pol . e_perp) e_perp],
    Theta the angle between khat and r; khat = z, pol = x gives ``farfield``."""
    khat = np.asarray(khat, float)
    pol = np.asarray(pol, complex)
    dirs = np.asarray(dirs, float).reshape(-1, 3)
    theta = np.arccos(np.clip(dirs @ khat, -1.0, 1.0))
    S1, S2 = amplitudes(k0 * radius, math.sqrt(eps_r), theta)
    out = np.zeros((len(dirs), 3), dtype=np.complex128)
    for i, r in enumerate(dirs):
        c = np.cross(khat, r)
        nc = np.linalg.norm(c)
        if nc < 1e-12:  # forward / backward: any axis normal to khat
            c = np.cross(khat, (1.0, 0.0, 0.0) if abs(khat[0]) < 0.9 else (0.0, 1.0, 0.0))
            nc = np.linalg.norm(c)
        ep = c / nc
        out[i] = (1j / k0) * (S2[i] * (pol @ np.cross(ep, khat)) * np.cross(ep, r) + S1[i] * (pol @ ep) * ep)
    return out


def extinction_efficiency(radius, eps_r, k0):
    """Q_ext = (2/x^2) sum (2n+1) Re(a_n + b_n)."""
    x = k0 * radius
    n, a, b = coefficients(x, math.sqrt(eps_r))
    return 2.0 / x ** 2 * float(np.sum((2 * n + 1) * (a + b).real))
