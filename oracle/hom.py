"""FP64 CPU oracle of the two-photon observables (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.

Follows Sec. II of the paper:
* the two-channel transfer relation (Eqs. field_transfer1/2, eq8-eq9) with
  T_{aj} = sqrt(omega_j) E_{aj} (the constant C cancels in every ratio);
* g2 in its general operator form (Eq. 11) evaluated by brute force in a
  truncated two-mode Fock space, and in the compact degenerate form (Eq. 10);
* the path amplitudes A_dir, A_ex (Eq. path_amplitudes) and the normalised
  coincidence number (Eqs. 18-22, HOM_envelope), both as a closed form and by
  numerical tau-quadrature of Eq. G2_scatter;
* the classical intensity-product correlation (Eq. 27).

Readings of the paper used here:
* h(tau) is the envelope exp(-tau^2/(2 sigma^2)); the carrier exp(-i w0 tau)
  of Eq. h_gauss is already factored out of the transfer relation (with it the
  overlap integral would oscillate at 2 w0 and contradict Eq. HOM_envelope).
* D_c is fixed by the stated limit N~c -> 1 for |dtau| -> inf:
  D_c = (|A_dir|^2 + |A_ex|^2) * int |h|^2.
* HOM visibility V = 1 - N~c(0).
* When A_dir = A_ex = 0 (a channel absent at both detectors) N~c is 0/0 and is
  reported as NaN.
"""
from __future__ import annotations

import math

import numpy as np


def transfer_matrix(E, omega=(1.0, 1.0)):
    """T[det][ch] = sqrt(omega_ch) * E[det][ch]; E[0] is detector a (r1),
    E[1] detector b (r2)."""
    E = np.asarray(E, dtype=np.complex128).reshape(2, 2)
    w = np.sqrt(np.asarray(omega, float))
    return E * w[None, :]


def g2_degenerate(E, omega=(1.0, 1.0)):
    """Eq. 10: omega1 omega2 |E_a1 E_b2 + E_a2 E_b1|^2 divided by
    (sum_l omega_l |E_al|^2)(sum_l omega_l |E_bl|^2)."""
    E = np.asarray(E, dtype=np.complex128).reshape(2, 2)
    w1, w2 = omega
    num = w1 * w2 * abs(E[0, 0] * E[1, 1] + E[0, 1] * E[1, 0]) ** 2
    den = (w1 * abs(E[0, 0]) ** 2 + w2 * abs(E[0, 1]) ** 2) * \
          (w1 * abs(E[1, 0]) ** 2 + w2 * abs(E[1, 1]) ** 2)
    if den == 0.0:
        return float("nan")
    return num / den


# ---- brute-force Fock-space evaluation of Eq. 11 -------------------------------- #
def _mode_ops(nmax=2):
    """Annihilation operators a_1, a_2 on the two-mode Fock space truncated at
    nmax photons per mode (basis |n1, n2>, index n1*(nmax+1)+n2)."""
    d = nmax + 1
    a = np.zeros((d, d))
    for k in range(1, d):
        a[k - 1, k] = math.sqrt(k)
    eye = np.eye(d)
    return np.kron(a, eye), np.kron(eye, a)


def g2_fock(E, omega=(1.0, 1.0), state=None):
    """Eq. 11 with explicit operators: numerator sum over m,n,p,q of
    T*_am T*_bn T_bp T_aq <a+_m a+_n a_p a_q>, denominator the product of the
    two first-order sums.  ``state``: Fock-space vector (default |1,1>)."""
    a1, a2 = _mode_ops(2)
    d = 3
    if state is None:
        state = np.zeros(d * d)
        state[1 * d + 1] = 1.0
    ops = [a1, a2]
    T = transfer_matrix(E, omega)
    Ea = T[0, 0] * ops[0] + T[0, 1] * ops[1]  # E_a^(+) at r1
    Eb = T[1, 0] * ops[0] + T[1, 1] * ops[1]  # E_b^(+) at r2
    psi = np.asarray(state, dtype=np.complex128)
    G2 = np.vdot(psi, Ea.conj().T @ Eb.conj().T @ Eb @ Ea @ psi).real
    G1a = np.vdot(psi, Ea.conj().T @ Ea @ psi).real
    G1b = np.vdot(psi, Eb.conj().T @ Eb @ psi).real
    if G1a * G1b == 0.0:
        return float("nan")
    return G2 / (G1a * G1b)


# ---- time domain ---------------------------------------------------------------- #
def path_amplitudes(E, omega=(1.0, 1.0)):
    """A_dir = T_a1 T_b2, A_ex = T_a2 T_b1 (Eq. path_amplitudes; equal to
    omega0 E_a1 E_b2 and omega0 E_a2 E_b1 in the degenerate case)."""
    T = transfer_matrix(E, omega)
    return T[0, 0] * T[1, 1], T[0, 1] * T[1, 0]


def envelope(tau, sigma):
    """h(tau) = exp(-tau^2/(2 sigma^2)) (Eq. h_gauss without the carrier)."""
    return np.exp(-np.asarray(tau, float) ** 2 / (2.0 * sigma * sigma))


def coincidence_closed(E, dtau, sigma=1.2, omega=(1.0, 1.0)):
    """N~c(dtau) = (N1+N2+N3+N4)/D_c with the Gaussian integrals in closed form:
    int |h|^2 = sigma sqrt(pi), int h(t) h*(2 dtau - t) dt =
    sigma sqrt(pi) exp(-dtau^2/sigma^2)."""
    Ad, Ae = path_amplitudes(E, omega)
    dtau = np.asarray(dtau, float)
    s = sigma * math.sqrt(math.pi)
    N1 = abs(Ad) ** 2 * s
    N2 = abs(Ae) ** 2 * s
    ov = s * np.exp(-dtau ** 2 / sigma ** 2)
    N3 = Ad * np.conj(Ae) * ov
    N4 = np.conj(Ad) * Ae * ov
    Dc = (abs(Ad) ** 2 + abs(Ae) ** 2) * s
    if Dc == 0.0:
        return np.full(dtau.shape, np.nan)
    return ((N1 + N2 + N3 + N4).real) / Dc


def coincidence_quadrature(E, dtau, sigma=1.2, omega=(1.0, 1.0), tmax=None, nt=20001):
    """N~c(dtau) by trapezoidal tau-integration of Eq. G2_scatter (K = 1)
    normalised by its large-delay value."""
    Ad, Ae = path_amplitudes(E, omega)
    if tmax is None:
        tmax = 12.0 * sigma + 2.0 * float(np.max(np.abs(dtau)))
    t = np.linspace(-tmax, tmax, nt)
    out = []
    for d in np.atleast_1d(dtau):
        h1 = envelope(t, sigma)
        h2 = envelope(2.0 * d - t, sigma)
        G2 = (abs(Ad) ** 2 * np.abs(h1) ** 2 + abs(Ae) ** 2 * np.abs(h2) ** 2
              + Ad * np.conj(Ae) * h1 * np.conj(h2) + np.conj(Ad) * Ae * np.conj(h1) * h2)
        Nc = np.trapezoid(G2.real, t)
        Dc = (abs(Ad) ** 2 + abs(Ae) ** 2) * np.trapezoid(np.abs(h1) ** 2, t)
        out.append(Nc / Dc if Dc != 0 else np.nan)
    return np.array(out)


def visibility(E, sigma=1.2, omega=(1.0, 1.0)):
    """V = 1 - N~c(0)."""
    return 1.0 - float(coincidence_closed(E, [0.0], sigma, omega)[0])


def classical_p2(E1, E2):
    """Eq. 27: P2 = |E(r1)|^2 |E(r2)|^2 with E = E_k1 + E_k2 (unnormalised).
    ``E1``, ``E2``: (E_k1, E_k2) at r1 and at r2."""
    a = abs(E1[0] + E1[1]) ** 2
    b = abs(E2[0] + E2[1]) ** 2
    return a * b
