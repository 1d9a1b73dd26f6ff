"""FP64 CPU oracle of the FFT-VIE hot path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module; the library never does.  It shares no
code with the CUDA path.  Everything is plain NumPy in float64/complex128,
written step by step from the paper:

* polarisation current and scattered field, Sec. II-C, Eqs. (Js_def),
  (Esca_from_J), the VIE (Eq. 24) and the dyadic Green's function (dyadicG);
* uniform-voxel discretisation with a convolution (Toeplitz) structure, so the
  matrix-vector product is a zero-padded FFT convolution (Sec. II-C, after
  Eq. Js_expand);
* far-field radiation integral (Eq. 25) and detector projection (Eq. Eproj),
  circular components (Eq. 30).

Unknown and discretisation (the paper fixes neither the integration rules of
its rooftop scheme nor C_inf).  With J = -i omega eps0 chi E_tot (Eq. Js_def)
the unknown is the contrast current w = chi * E_tot and Eq. 24 becomes, on
every voxel n,

    w_n - chi_n * sum_m K(n - m) w_m = chi_n * E_inc(r_n).

Each source voxel is replaced by the sphere of equal volume V = h^3 (radius
a = h (3/4pi)^{1/3}) and the equation is tested at voxel centres:

    K(m != 0) = kappa k0^2 V G(r_m),  kappa = 3 (sin ka - ka cos ka)/(ka)^3
    K(0)      = [2/3 ((1 - i ka) e^{i ka} - 1) - 1/3] I

kappa is the mean-value factor of a Helmholtz solution over a ball (exact,
since a < h), K(0) is the ball integral of k0^2 G including the -I/3
depolarisation.  The far field, with E_sca ~ F exp(i k0 r)/r, is

    F(rhat) = kappa k0^2 V / (4 pi) (I - rhat rhat) sum_n w_n exp(-i k0 rhat.r_n).

With these choices Im K equals kappa k0^2 V Im G entrywise, so the discrete
model satisfies the optical theorem and reciprocity exactly (pinned in tests).

Tensor components are stored in the order (xx, xy, xz, yy, yz, zz).
Vectors over the grid have shape ``(3, n0, n1, n2)`` (C order, z fastest).
"""
from __future__ import annotations

import math

import numpy as np

COMP = ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))
# index of component (i, j) in the 6-vector
CIDX = [[0, 1, 2], [1, 3, 4], [2, 4, 5]]


# --------------------------------------------------------------------------- #
# geometry
# --------------------------------------------------------------------------- #
def voxel_axes(n, h, origin=(0.0, 0.0, 0.0)):
    """Voxel-centre coordinates along x, y, z (grid centre at ``origin``)."""
    return tuple(origin[a] + (np.arange(n[a]) - 0.5 * (n[a] - 1)) * h for a in range(3))


def voxel_positions(n, h, origin=(0.0, 0.0, 0.0)):
    """All voxel centres, shape (n0, n1, n2, 3)."""
    x, y, z = voxel_axes(n, h, origin)
    X, Y, Z = np.meshgrid(x, y, z, indexing="ij")
    return np.stack([X, Y, Z], axis=-1)


def contrast(eps_r):
    """chi = eps_r - 1 (Eq. Js_def with eps/eps0 = eps_r, lossless => real)."""
    return np.asarray(eps_r, dtype=np.float64) - 1.0


# --------------------------------------------------------------------------- #
# Green's tensor and the discrete kernel K(m)
# --------------------------------------------------------------------------- #
def equivalent_radius(h):
    """Radius of the sphere with the voxel's volume h^3."""
    return h * (3.0 / (4.0 * math.pi)) ** (1.0 / 3.0)


def mean_value_factor(ka):
    """kappa(ka) = 3 (sin ka - ka cos ka)/(ka)^3: the average over a ball of
    radius a of any solution of (nabla^2 + k^2) u = 0, divided by u(centre)."""
    ka = float(ka)
    if ka < 1e-3:
        x2 = ka * ka
        return 1.0 - x2 / 10.0 + x2 * x2 / 280.0
    return 3.0 * (math.sin(ka) - ka * math.cos(ka)) / ka ** 3


def self_term(k0, h):
    """K(0)/I: k0^2 times the integral of the dyadic Green's function over the
    equal-volume ball centred on the observation point (principal-volume part
    plus the -1/3 depolarisation dyad)."""
    ka = k0 * equivalent_radius(h)
    return (2.0 / 3.0) * ((1.0 - 1j * ka) * np.exp(1j * ka) - 1.0) - 1.0 / 3.0


def green_dyadic(R, k0):
    """Free-space dyadic Green's function (Eq. dyadicG) for separations R != 0.

    (I + grad grad / k^2) e^{ikR}/(4 pi R) in closed form:
        g [ (1 + i/(kR) - 1/(kR)^2) I + (-1 - 3i/(kR) + 3/(kR)^2) Rhat Rhat ],
    g = e^{ikR}/(4 pi R).  ``R`` has shape (..., 3); returns (..., 6)."""
    R = np.asarray(R, dtype=np.float64)
    r = np.sqrt(np.sum(R * R, axis=-1))
    kr = k0 * r
    g = np.exp(1j * kr) / (4.0 * math.pi * r)
    a = 1.0 + 1j / kr - 1.0 / kr ** 2
    b = -1.0 - 3j / kr + 3.0 / kr ** 2
    u = R / r[..., None]
    out = np.empty(R.shape[:-1] + (6,), dtype=np.complex128)
    for c, (i, j) in enumerate(COMP):
        out[..., c] = g * (b * u[..., i] * u[..., j] + (a if i == j else 0.0))
    return out


def kernel_at(m, h, k0):
    """Discrete kernel K(m) for integer offsets ``m`` (shape (..., 3)) -> (..., 6)."""
    m = np.asarray(m, dtype=np.int64)
    a = equivalent_radius(h)
    kap = mean_value_factor(k0 * a)
    V = h ** 3
    zero = np.all(m == 0, axis=-1)
    R = m.astype(np.float64) * h
    Rs = np.where(zero[..., None], 1.0, R)  # placeholder for the self term
    out = kap * k0 * k0 * V * green_dyadic(Rs, k0)
    s = self_term(k0, h)
    if np.any(zero):
        out[zero] = np.array([s, 0, 0, s, 0, s], dtype=np.complex128)
    return out


def kernel_table(n, h, k0):
    """K on every offset m in (-(n-1) .. n-1)^3, shape (6, 2n0-1, 2n1-1, 2n2-1);
    entry [c, m0+n0-1, m1+n1-1, m2+n2-1] holds component c of K(m)."""
    rng = [np.arange(-(n[a] - 1), n[a]) for a in range(3)]
    M = np.stack(np.meshgrid(*rng, indexing="ij"), axis=-1)
    return np.moveaxis(kernel_at(M, h, k0), -1, 0).copy()


# --------------------------------------------------------------------------- #
# operator A w = w - chi (K * w): dense, direct sum and FFT
# --------------------------------------------------------------------------- #
def dense_operator(n, h, k0, chi):
    """Assemble A = I - diag(chi) K as a dense (3N x 3N) matrix, component-major
    (row index = i*N + voxel).  Each entry calls ``kernel_at`` for its own
    offset.  For small grids only."""
    N = int(np.prod(n))
    idx = np.stack(np.unravel_index(np.arange(N), n), axis=-1)
    diff = idx[:, None, :] - idx[None, :, :]
    K = kernel_at(diff, h, k0)  # (N, N, 6)
    A = np.zeros((3 * N, 3 * N), dtype=np.complex128)
    c = np.asarray(chi, float).reshape(-1)
    for i in range(3):
        for j in range(3):
            A[i * N:(i + 1) * N, j * N:(j + 1) * N] = -c[:, None] * K[:, :, CIDX[i][j]]
    A += np.eye(3 * N)
    return A


def convolve_direct(Ktab, n, w, targets=None):
    """(K * w)(t) = sum_s K(t - s) w(s) by direct summation over all sources.

    ``Ktab`` from ``kernel_table``; ``w`` shape (3, n0, n1, n2).  ``targets``:
    optional (T, 3) integer voxel indices; returns (3, T) for them, else the
    full (3, n0, n1, n2) field."""
    n = tuple(n)
    if targets is None:
        targets = np.stack(np.unravel_index(np.arange(int(np.prod(n))), n), axis=-1)
        full = True
    else:
        targets = np.asarray(targets)
        full = False
    out = np.zeros((3, len(targets)), dtype=np.complex128)
    for t, (t0, t1, t2) in enumerate(targets):
        # offsets t - s for s = 0..n-1 along each axis -> table index t - s + n - 1
        sub = Ktab[:, t0:t0 + n[0], t1:t1 + n[1], t2:t2 + n[2]][:, ::-1, ::-1, ::-1]
        for i in range(3):
            acc = 0.0 + 0.0j
            for j in range(3):
                acc += np.sum(sub[CIDX[i][j]] * w[j])
            out[i, t] = acc
    if full:
        return out.reshape((3,) + n)
    return out


def convolve_direct_points(n, h, k0, w, targets):
    """Like ``convolve_direct`` at a few targets, evaluating K on the fly (no
    (2n-1)^3 table): for large grids."""
    n = tuple(n)
    src = np.stack(np.unravel_index(np.arange(int(np.prod(n))), n), axis=-1)
    wf = w.reshape(3, -1)
    out = np.zeros((3, len(targets)), dtype=np.complex128)
    for t, tv in enumerate(np.asarray(targets)):
        K = kernel_at(tv[None, :] - src, h, k0)  # (N, 6)
        for i in range(3):
            out[i, t] = sum(np.dot(K[:, CIDX[i][j]], wf[j]) for j in range(3))
    return out


def convolve_direct_points_multi(n, h, k0, W, targets):
    """``convolve_direct_points`` for a stack of fields W (R, 3, n0, n1, n2),
    evaluating K once per target.  Returns (R, 3, T)."""
    n = tuple(n)
    src = np.stack(np.unravel_index(np.arange(int(np.prod(n))), n), axis=-1)
    Wf = np.asarray(W).reshape(len(W), 3, -1)
    out = np.zeros((len(W), 3, len(targets)), dtype=np.complex128)
    for t, tv in enumerate(np.asarray(targets)):
        K = kernel_at(tv[None, :] - src, h, k0)  # (N, 6)
        for i in range(3):
            out[:, i, t] = sum(Wf[:, j] @ K[:, CIDX[i][j]] for j in range(3))
    return out


def convolve_points_sparse(src, Wsrc, h, k0, targets, chunk=1 << 20):
    """(K * w)(t) = sum_s K(t - s) w(s) over an explicit source list, for grids
    too large to hold as dense fields: ``src`` (S, 3) integer voxel indices,
    ``Wsrc`` (R, 3, S) their currents, ``targets`` (T, 3).  Returns (R, 3, T).
    Sources are taken in chunks of ``chunk`` (memory only; same sum)."""
    src = np.asarray(src, dtype=np.int64)
    Wsrc = np.asarray(Wsrc)
    out = np.zeros((Wsrc.shape[0], 3, len(targets)), dtype=np.complex128)
    for t, tv in enumerate(np.asarray(targets, dtype=np.int64)):
        for c0 in range(0, len(src), chunk):
            K = kernel_at(tv[None, :] - src[c0:c0 + chunk], h, k0)  # (S', 6)
            Wc = Wsrc[:, :, c0:c0 + chunk]
            for i in range(3):
                out[:, i, t] += sum(Wc[:, j] @ K[:, CIDX[i][j]] for j in range(3))
    return out


def apply_direct(Ktab, n, chi, w):
    """y = w - chi (K * w) with the direct-sum convolution."""
    return w - chi[None] * convolve_direct(Ktab, n, w)


def smooth_size(m, radices=(2, 3, 5, 7)):
    """Smallest integer >= m whose prime factors are all in ``radices``."""
    v = max(1, int(m))
    while True:
        r = v
        for p in radices:
            while r % p == 0:
                r //= p
        if r == 1:
            return v
        v += 1


def circulant_kernel(n, h, k0, P):
    """Embed K(m), |m_a| <= n_a - 1, into a periodic array of size P (each
    P_a >= 2 n_a - 1): index p holds K(p) for p <= n-1, K(p - P) for
    p >= P - n + 1, zero in between.  Shape (6, P0, P1, P2)."""
    for a in range(3):
        if P[a] < 2 * n[a] - 1:
            raise ValueError("padded size too small")
    offs = []
    for a in range(3):
        p = np.arange(P[a])
        o = np.where(p <= n[a] - 1, p, p - P[a])
        valid = (p <= n[a] - 1) | (p >= P[a] - n[a] + 1)
        offs.append((o, valid))
    M = np.stack(np.meshgrid(offs[0][0], offs[1][0], offs[2][0], indexing="ij"), axis=-1)
    V = (offs[0][1][:, None, None] & offs[1][1][None, :, None] & offs[2][1][None, None, :])
    K = np.moveaxis(kernel_at(M, h, k0), -1, 0)
    K[:, ~V] = 0.0
    return K


class FFTOperator:
    """A w = w - chi (K * w) with the convolution done as a zero-padded
    circular convolution through 3-D FFTs (O(N log N), Sec. II-C)."""

    def __init__(self, n, h, k0, chi, P=None, workers=None):
        self.n = tuple(int(v) for v in n)
        self.P = tuple(P) if P is not None else tuple(smooth_size(2 * v - 1) for v in self.n)
        self.chi = np.asarray(chi, dtype=np.float64)
        self.workers = workers
        Kc = circulant_kernel(self.n, h, k0, self.P)
        self.Khat = self._fft(Kc, axes=(1, 2, 3))

    def _fft(self, a, axes):
        import scipy.fft as sf
        return sf.fftn(a, axes=axes, workers=self.workers)

    def _ifft(self, a, axes):
        import scipy.fft as sf
        return sf.ifftn(a, axes=axes, workers=self.workers)

    def convolve(self, w):
        n, P = self.n, self.P
        pad = np.zeros((3,) + P, dtype=np.complex128)
        pad[:, :n[0], :n[1], :n[2]] = w
        W = self._fft(pad, axes=(1, 2, 3))
        U = np.empty_like(W)
        for i in range(3):
            U[i] = sum(self.Khat[CIDX[i][j]] * W[j] for j in range(3))
        u = self._ifft(U, axes=(1, 2, 3))
        return u[:, :n[0], :n[1], :n[2]]

    def __call__(self, w):
        w = np.asarray(w).reshape((3,) + self.n)
        return w - self.chi[None] * self.convolve(w)


# --------------------------------------------------------------------------- #
# incident field, right-hand side
# --------------------------------------------------------------------------- #
def incident_field(n, h, k0, khat, pol, origin=(0.0, 0.0, 0.0)):
    """E_inc(r_n) = pol exp(i k0 khat . r_n) at voxel centres, shape (3, n0, n1, n2)."""
    r = voxel_positions(n, h, origin)
    ph = np.exp(1j * k0 * (r @ np.asarray(khat, float)))
    return np.asarray(pol, dtype=np.complex128)[:, None, None, None] * ph[None]


def rhs(chi, Einc):
    """b = chi E_inc (the VIE right-hand side in the w unknown)."""
    return chi[None] * Einc


# --------------------------------------------------------------------------- #
# GMRES (restarted, Givens rotations), Saad's formulation
# --------------------------------------------------------------------------- #
def gmres(apply, b, tol=1e-12, restart=60, maxiter=5000, x0=None):
    """Solve A x = b to ||b - A x||_2 <= tol ||b||_2.  Arnoldi with modified
    Gram-Schmidt, Givens rotations for the least-squares problem, restart
    from the true residual.  Returns (x, info) with info = dict(iters,
    relres, converged)."""
    shape = b.shape
    bv = b.reshape(-1).astype(np.complex128)
    x = np.zeros_like(bv) if x0 is None else x0.reshape(-1).astype(np.complex128).copy()
    bnorm = np.linalg.norm(bv)
    if bnorm == 0.0:
        return x.reshape(shape), dict(iters=0, relres=0.0, converged=True)
    A = lambda v: np.asarray(apply(v.reshape(shape))).reshape(-1)
    it = 0
    r = bv - A(x) if x0 is not None else bv.copy()
    beta = np.linalg.norm(r)
    while it < maxiter:
        if beta <= tol * bnorm:
            return x.reshape(shape), dict(iters=it, relres=beta / bnorm, converged=True)
        m = restart
        V = np.zeros((m + 1, bv.size), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m, dtype=np.complex128)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        V[0] = r / beta
        g[0] = beta
        k = 0
        for j in range(m):
            wv = A(V[j])
            it += 1
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], wv)
                wv = wv - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(wv)
            if H[j + 1, j] != 0:
                V[j + 1] = wv / H[j + 1, j]
            # apply previous rotations to column j
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + np.conj(cs[i]) * H[i + 1, j]
                H[i, j] = t
            # new rotation annihilating H[j+1, j]
            a, bb = H[j, j], H[j + 1, j]
            den = math.sqrt(abs(a) ** 2 + abs(bb) ** 2)
            if den == 0.0:
                cs[j], sn[j] = 1.0, 0.0
            elif a == 0:
                cs[j], sn[j] = 0.0, 1.0
            else:
                cs[j] = abs(a) / den
                sn[j] = (a / abs(a)) * np.conj(bb) / den
            H[j, j] = cs[j] * a + sn[j] * bb
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            if abs(g[j + 1]) <= tol * bnorm or it >= maxiter:
                break
        y = np.zeros(k, dtype=np.complex128)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - np.dot(H[i, i + 1:k], y[i + 1:k])) / H[i, i]
        x = x + V[:k].T @ y
        r = bv - A(x)
        beta = np.linalg.norm(r)
    return x.reshape(shape), dict(iters=it, relres=beta / bnorm, converged=beta <= tol * bnorm)


def cocr(op, b, tol=1e-12, maxiter=100000):
    """Solve A w = b (A = I - diag(chi) K, ``op`` an FFTOperator) by the
    conjugate orthogonal conjugate residual method (Sogabe and Zhang, J.
    Comput. Appl. Math. 199, 2007), a short recurrence for complex symmetric
    systems.  K is complex symmetric (reciprocity), so on the body voxels
    S = diag(chi)^-1 A = diag(1/chi) - K is too, and COCR runs on S w = b / chi
    with the unconjugated product u^T v.  The residual of A follows as
    b - A w = chi (b/chi - S w).  Stops when ||b - A w||_2 <= tol ||b||_2, checked
    at the end against the operator itself.  Returns (w, info)."""
    chi = op.chi
    body = chi > 0
    inv = np.zeros_like(chi)
    inv[body] = 1.0 / chi[body]
    mask = body[None].astype(float)

    def S(v):
        return (inv[None] * v - op.convolve(v)) * mask

    bv = np.asarray(b, dtype=np.complex128).reshape((3,) + op.n)
    bnorm = np.linalg.norm(bv)
    x = np.zeros_like(bv)
    if bnorm == 0.0:
        return x, dict(iters=0, relres=0.0, converged=True)
    r = inv[None] * bv
    Sr = S(r)
    p = r.copy()
    Sp = Sr.copy()
    rho = np.sum(r * Sr)
    it = 0
    while it < maxiter:
        alpha = rho / np.sum(Sp * Sp)
        x += alpha * p
        r -= alpha * Sp
        it += 1
        if np.linalg.norm(chi[None] * r) <= tol * bnorm:
            true = np.linalg.norm(bv - op(x)) / bnorm
            if true <= tol:
                return x, dict(iters=it, relres=true, converged=True)
            r = inv[None] * (bv - op(x))  # restart the recurrence from the true residual
            Sr = S(r)
            p = r.copy()
            Sp = Sr.copy()
            rho = np.sum(r * Sr)
            continue
        Sr = S(r)
        rho_new = np.sum(r * Sr)
        beta = rho_new / rho
        rho = rho_new
        p = r + beta * p
        Sp = Sr + beta * Sp
    true = np.linalg.norm(bv - op(x)) / bnorm
    return x, dict(iters=it, relres=true, converged=true <= tol)


# --------------------------------------------------------------------------- #
# far field and detector projection
# --------------------------------------------------------------------------- #
def farfield_constant(h, k0):
    """C_inf of Eq. 25 in this normalisation: kappa k0^2 V / (4 pi)."""
    return mean_value_factor(k0 * equivalent_radius(h)) * k0 * k0 * h ** 3 / (4.0 * math.pi)


def farfield(w, n, h, k0, dirs, origin=(0.0, 0.0, 0.0), chunk=256):
    """F(rhat) for each unit vector in ``dirs`` (D, 3), by direct summation of
    Eq. 25 over all voxels.  ``w`` shape (3, n0, n1, n2).  Returns (D, 3)."""
    dirs = np.asarray(dirs, dtype=np.float64).reshape(-1, 3)
    r = voxel_positions(n, h, origin).reshape(-1, 3)
    wf = np.asarray(w).reshape(3, -1)
    C = farfield_constant(h, k0)
    out = np.zeros((len(dirs), 3), dtype=np.complex128)
    for s in range(0, len(dirs), chunk):
        d = dirs[s:s + chunk]
        E = np.exp(-1j * k0 * (d @ r.T))  # (c, N)
        S = E @ wf.T  # (c, 3)
        rs = np.sum(d * S, axis=1)
        out[s:s + chunk] = C * (S - d * rs[:, None])
    return out


def na_rule(center, theta_na, sigma, nt, nphi):
    """Quadrature of a detector with a finite numerical aperture (Eq. NAfield):
    directions rhat = cos(t) c + sin(t) (cos(p) u + sin(p) v) around the unit
    axis c, t in [0, theta_na] on ``nt`` Gauss-Legendre nodes (a library rule),
    p = 2 pi j / nphi, with weights W(t) sin(t) dt dp, W(t) = exp(-t^2 / (2
    sigma^2)), normalised to sum 1.  Frame: u = (a x c)/|a x c| with a = z, or
    a = x when |c_z| >= 0.9; v = c x u.  Returns (dirs (Q, 3), weights (Q,))."""
    c = np.asarray(center, float)
    c = c / np.linalg.norm(c)
    a = np.array([0.0, 0.0, 1.0]) if abs(c[2]) < 0.9 else np.array([1.0, 0.0, 0.0])
    u = np.cross(a, c)
    u /= np.linalg.norm(u)
    v = np.cross(c, u)
    x, gw = np.polynomial.legendre.leggauss(nt)
    t = 0.5 * theta_na * (x + 1.0)
    wt = 0.5 * theta_na * gw * np.exp(-t * t / (2.0 * sigma * sigma)) * np.sin(t)
    p = 2.0 * math.pi * np.arange(nphi) / nphi
    T, Pp = np.meshgrid(t, p, indexing="ij")
    W = np.broadcast_to(wt[:, None], T.shape) * (2.0 * math.pi / nphi)
    dirs = (np.cos(T)[..., None] * c + np.sin(T)[..., None] * (np.cos(Pp)[..., None] * u + np.sin(Pp)[..., None] * v))
    W = W.reshape(-1)
    return dirs.reshape(-1, 3), W / W.sum()


def farfield_na(w, n, h, k0, centers, pols, theta_na, sigma, nt, nphi):
    """Aperture-collected detector amplitudes E_NA[d] = sum_q W_q pol_d . F(rhat_q)
    (bilinear projection as Eq. Eproj) of one current ``w``; shape (D,)."""
    out = np.zeros(len(centers), dtype=np.complex128)
    for d, (c, p) in enumerate(zip(centers, pols)):
        dirs, W = na_rule(c, theta_na, sigma, nt, nphi)
        F = farfield(w, n, h, k0, dirs)
        out[d] = np.sum(W * (F @ np.asarray(p, dtype=np.complex128)))
    return out


def spherical_unit_vectors(dirs):
    """(e_theta, e_phi) for unit vectors ``dirs`` (D, 3); theta = acos(z),
    phi = atan2(y, x)."""
    d = np.asarray(dirs, float)
    th = np.arccos(np.clip(d[:, 2], -1.0, 1.0))
    ph = np.arctan2(d[:, 1], d[:, 0])
    eth = np.stack([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), -np.sin(th)], -1)
    eph = np.stack([-np.sin(ph), np.cos(ph), np.zeros_like(ph)], -1)
    return eth, eph


def project(F, dirs, basis):
    """Detector projection (Eq. Eproj).  basis 0: (Fx, Fy, Fz); basis 1:
    (F_theta, F_phi, F_r); basis 2: (F_L, F_R, F_r) with
    F_{L,R} = (F_theta +/- i F_phi)/sqrt(2) (Eq. 30).  The incident plane wave
    contributes nothing off its own direction, so E_tot,inf = F there."""
    F = np.asarray(F)
    if basis == 0:
        return F.copy()
    d = np.asarray(dirs, float)
    eth, eph = spherical_unit_vectors(d)
    Ft = np.sum(eth * F, axis=1)
    Fp = np.sum(eph * F, axis=1)
    Fr = np.sum(d * F, axis=1)
    if basis == 1:
        return np.stack([Ft, Fp, Fr], -1)
    s = 1.0 / math.sqrt(2.0)
    return np.stack([s * (Ft + 1j * Fp), s * (Ft - 1j * Fp), Fr], -1)


def sphere_quadrature(L):
    """Gauss-Legendre in cos(theta) (L nodes) x uniform phi (2L nodes):
    integrates band-limited functions of degree < 2L on the unit sphere
    exactly.  Returns (dirs (M, 3), weights (M,))."""
    x, wt = np.polynomial.legendre.leggauss(L)
    M = 2 * L
    ph = 2.0 * math.pi * np.arange(M) / M
    th = np.arccos(x)
    T, Pp = np.meshgrid(th, ph, indexing="ij")
    W = np.repeat(wt[:, None] * (2.0 * math.pi / M), M, axis=1)
    dirs = np.stack([np.sin(T) * np.cos(Pp), np.sin(T) * np.sin(Pp), np.cos(T)], -1)
    return dirs.reshape(-1, 3), W.reshape(-1)


# --------------------------------------------------------------------------- #
# end-to-end helpers
# --------------------------------------------------------------------------- #
def solve_channels(n, h, k0, eps_r, channels, tol=1e-12, restart=80, maxiter=20000,
                   method="fft", origin=(0.0, 0.0, 0.0), workers=None):
    """Solve the VIE for each channel (khat, pol).  ``method`` is 'fft'
    (GMRES with the FFT operator), 'cocr' (COCR with the FFT operator),
    'direct' (GMRES with the direct sum) or 'lu' (dense LU).  Returns
    (w[R,3,n0,n1,n2], infos)."""
    chi = contrast(eps_r)
    out, infos = [], []
    if method == "lu":
        A = dense_operator(n, h, k0, chi)
    elif method == "direct":
        Ktab = kernel_table(n, h, k0)
        op = lambda v: apply_direct(Ktab, n, chi, v)
    else:
        op = FFTOperator(n, h, k0, chi, workers=workers)
    for khat, pol in channels:
        b = rhs(chi, incident_field(n, h, k0, khat, pol, origin))
        if method == "lu":
            x = np.linalg.solve(A, b.reshape(-1)).reshape(b.shape)
            info = dict(iters=0, relres=np.linalg.norm(A @ x.reshape(-1) - b.reshape(-1)) /
                        np.linalg.norm(b), converged=True)
        elif method == "cocr":
            x, info = cocr(op, b, tol=tol, maxiter=maxiter)
        else:
            x, info = gmres(op, b, tol=tol, restart=restart, maxiter=maxiter)
        out.append(x)
        infos.append(info)
    return np.stack(out), infos
