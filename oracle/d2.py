"""FP64 CPU oracle of the rooftop / pulse-tested discretisation ("D2") of the
VIE (test infrastructure only; same import rules as ``oracle.vie``).

Sec. II-C expands the current on the uniform grid in rooftop (piecewise
linear) functions along x, y and z, one per Cartesian component per cell, and
tests with pulses; it does not give the integration rules.  The reading used
here (a weak-form scheme with the scalar Green's function and a discrete
grad-div, the structure of the classical weak-form CGFFT):

* unknown w_a(c) = chi E_a at the +a face of cell c (the peak of the rooftop
  along a spanning cells c and c + e_a), a = x, y, z; face contrast
  chi_a(c) = (chi(c) + chi(c + e_a)) / 2, chi = 0 outside the grid;
* vector potential A(r) = int g(r - r') w(r') dr', g = e^{ikR}/(4 pi R); each
  rooftop carries the volume h^3 and acts as a source at its face centre with
  the ball-averaged scalar kernel
      G_h(m != 0) = kappa h^3 g(m h),  G_h(0) = ((1 - i k a) e^{i k a} - 1)/k^2
  (a = h (3/4 pi)^{1/3}, kappa the ball mean-value factor, as in the D1
  reading of ``oracle.vie``);
* grad-div by differences on the staggered grid: at cell centres
  (div A)(c) = sum_b (A_b(c) - A_b(c - e_b)) / h, at the +a face
  (d_a div A)(c) = ((div A)(c + e_a) - (div A)(c)) / h;
* pulse testing at the face centres of Eq. 24 with E = w/chi:
      y_a(c) = w_a(c) - chi_a(c) [k^2 A_a(c) + (d_a div A)(c)] = chi_a(c) E_inc,a(face).
* far field (Eq. 25) of the face sources: F = kappa k^2 h^3/(4 pi) (I - rr) sum w e^{-i k r.r_face}.

Faces at the low grid boundary (between the first cell and the outside) carry
no unknown: bodies are expected to leave the first layer of cells empty.
The parity of the CUDA path is pinned here by brute force (direct sums),
the complex symmetry of the discrete operator (reciprocity) and convergence
to the Mie series.
"""
from __future__ import annotations

import math

import numpy as np

from . import vie as _vie


def face_contrast(chi):
    """chi_a(c) = (chi(c) + chi(c + e_a))/2, shape (3, n0, n1, n2)."""
    chi = np.asarray(chi, dtype=np.float64)
    out = np.zeros((3,) + chi.shape)
    for a in range(3):
        nb = np.zeros_like(chi)
        sl = [slice(None)] * 3
        sl2 = [slice(None)] * 3
        sl[a] = slice(0, chi.shape[a] - 1)
        sl2[a] = slice(1, None)
        nb[tuple(sl)] = chi[tuple(sl2)]
        out[a] = 0.5 * (chi + nb)
    return out


def face_positions(n, h, a, origin=(0.0, 0.0, 0.0)):
    """Centres of the +a faces, shape (n0, n1, n2, 3)."""
    r = _vie.voxel_positions(n, h, origin).copy()
    r[..., a] += 0.5 * h
    return r


def scalar_kernel(m, h, k0):
    """G_h(m) for integer offsets ``m`` (shape (..., 3))."""
    m = np.asarray(m, dtype=np.int64)
    a = _vie.equivalent_radius(h)
    ka = k0 * a
    kap = _vie.mean_value_factor(ka)
    zero = np.all(m == 0, axis=-1)
    R = np.sqrt(np.sum((m * h).astype(np.float64) ** 2, axis=-1))
    Rs = np.where(zero, 1.0, R)
    out = kap * h ** 3 * np.exp(1j * k0 * Rs) / (4.0 * math.pi * Rs)
    out = np.where(zero, ((1.0 - 1j * ka) * np.exp(1j * ka) - 1.0) / (k0 * k0), out)
    return out


def _potential_direct(n, h, k0, w, lo=-1, hi=None):
    """A_a on cells lo..hi (inclusive, every axis) by direct sums over the
    face sources; returns (3, L, L, L) with L = hi - lo + 1 per axis."""
    n = tuple(n)
    hi = [n[a] if hi is None else hi for a in range(3)]
    src = np.argwhere(np.any(w != 0, axis=0))
    tgt = np.stack(np.meshgrid(*[np.arange(lo, hi[a] + 1) for a in range(3)], indexing="ij"), -1)
    shp = tgt.shape[:-1]
    tgt = tgt.reshape(-1, 3)
    A = np.zeros((3, len(tgt)), dtype=np.complex128)
    for s in src:
        G = scalar_kernel(tgt - s, h, k0)
        for a in range(3):
            A[a] += G * w[a][tuple(s)]
    return A.reshape((3,) + shp)


def _grad_div(A, h):
    """d_a div A on the +a faces of cells 0..n-1 from A on cells -1..n
    (array offset 1); returns (3, n0, n1, n2)."""
    L = A.shape[1:]
    n = tuple(v - 2 for v in L)
    # div at cells 0..n from A(c) - A(c - e_b)
    div = np.zeros(tuple(n[a] + 1 for a in range(3)), dtype=np.complex128)
    for b in range(3):
        hi = [slice(1, n[a] + 2) for a in range(3)]
        lo = list(hi)
        lo[b] = slice(0, n[b] + 1)
        div += (A[b][tuple(hi)] - A[b][tuple(lo)]) / h
    out = np.zeros((3,) + n, dtype=np.complex128)
    for a in range(3):
        c0 = [slice(0, n[q]) for q in range(3)]
        c1 = list(c0)
        c1[a] = slice(1, n[a] + 1)
        out[a] = (div[tuple(c1)] - div[tuple(c0)]) / h
    return out


def kernel_apply_direct(n, h, k0, w):
    """K w = k^2 A + d div A on the faces of every cell, by direct sums."""
    A = _potential_direct(n, h, k0, w)
    nn = tuple(n)
    inner = A[:, 1:nn[0] + 1, 1:nn[1] + 1, 1:nn[2] + 1]
    return k0 * k0 * inner + _grad_div(A, h)


def apply_direct(n, h, k0, chi_f, w):
    """y = w - chi_f (K w) by direct sums (small grids)."""
    return w - chi_f * kernel_apply_direct(n, h, k0, w)


class FFTOperator:
    """The same operator with A from zero-padded FFT convolutions (one scalar
    convolution per component) on a padded grid P >= 2n + 1, so that A is
    exact on cells -1..n; the differences are then taken in real space."""

    def __init__(self, n, h, k0, chi, workers=None):
        self.n = tuple(int(v) for v in n)
        self.h, self.k0 = float(h), float(k0)
        self.P = tuple(_vie.smooth_size(2 * v + 1) for v in self.n)
        self.chi_f = face_contrast(chi)
        self.workers = workers
        rng = [np.fft.fftfreq(self.P[a], 1.0 / self.P[a]).astype(np.int64) for a in range(3)]
        M = np.stack(np.meshgrid(*rng, indexing="ij"), -1)
        self.Ghat = self._fft(scalar_kernel(M, self.h, self.k0))

    def _fft(self, a):
        import scipy.fft as sf
        return sf.fftn(a, workers=self.workers)

    def _ifft(self, a):
        import scipy.fft as sf
        return sf.ifftn(a, workers=self.workers)

    def kernel_apply(self, w):
        n, P = self.n, self.P
        A = np.zeros((3,) + tuple(v + 2 for v in n), dtype=np.complex128)
        for a in range(3):
            pad = np.zeros(P, dtype=np.complex128)
            pad[:n[0], :n[1], :n[2]] = w[a]
            full = self._ifft(self.Ghat * self._fft(pad))
            idx = [np.arange(-1, n[q] + 1) % P[q] for q in range(3)]
            A[a] = full[np.ix_(*idx)]
        inner = A[:, 1:n[0] + 1, 1:n[1] + 1, 1:n[2] + 1]
        return self.k0 * self.k0 * inner + _grad_div(A, self.h)

    def __call__(self, w):
        w = np.asarray(w).reshape((3,) + self.n)
        return w - self.chi_f * self.kernel_apply(w)


def rhs(chi, n, h, k0, khat, pol, origin=(0.0, 0.0, 0.0)):
    """b_a(c) = chi_a(c) pol_a exp(i k0 khat . r_face,a(c)), shape (3, n0, n1, n2)."""
    chi_f = face_contrast(chi)
    b = np.zeros((3,) + tuple(n), dtype=np.complex128)
    pol = np.asarray(pol, dtype=np.complex128)
    for a in range(3):
        r = face_positions(n, h, a, origin)
        b[a] = chi_f[a] * pol[a] * np.exp(1j * k0 * (r @ np.asarray(khat, float)))
    return b


def farfield(w, n, h, k0, dirs, origin=(0.0, 0.0, 0.0)):
    """F(rhat) of the face sources, shape (D, 3)."""
    dirs = np.asarray(dirs, float).reshape(-1, 3)
    kap = _vie.mean_value_factor(k0 * _vie.equivalent_radius(h))
    C = kap * k0 * k0 * h ** 3 / (4.0 * math.pi)
    S = np.zeros((len(dirs), 3), dtype=np.complex128)
    for a in range(3):
        r = face_positions(n, h, a, origin).reshape(-1, 3)
        wa = np.asarray(w[a]).reshape(-1)
        nz = wa != 0
        if np.any(nz):
            S[:, a] = np.exp(-1j * k0 * (dirs @ r[nz].T)) @ wa[nz]
    F = C * (S - dirs * np.sum(dirs * S, axis=1, keepdims=True))
    return F


def solve(n, h, k0, eps_r, channels, tol=1e-10, restart=80, maxiter=20000):
    """Currents of every channel with the oracle's GMRES; returns (W, infos)."""
    chi = _vie.contrast(eps_r)
    op = FFTOperator(n, h, k0, chi, workers=-1)
    W, infos = [], []
    for khat, pol in channels:
        b = rhs(chi, n, h, k0, khat, pol)
        x, info = _vie.gmres(lambda v: op(v).reshape(-1), b.reshape(-1), tol=tol, restart=restart,
                             maxiter=maxiter)
        W.append(x.reshape((3,) + tuple(n)))
        infos.append(info)
    return np.stack(W), infos
