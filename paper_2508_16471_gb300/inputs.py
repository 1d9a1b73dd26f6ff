"""Seeded synthetic inputs shared by the CUDA path, the oracle tests and the bench.

This module holds geometry voxelisers, incident-channel definitions and
direction grids only: it contains none of the method's arithmetic (no Green's
tensor, no convolution, no far-field sum).  Everything is NumPy FP64 and
deterministic for a given seed (PCG64).

Lengths are in units of the free-space wavelength (k0 = 2*pi) unless stated.

Workloads (sizes follow the paper's examples, Sec. III):
  * ``sphere16_workload``  -- 16^3, h = 1/20, R = 0.4, eps_r = 2.25, two channels.
  * ``sphere64_workload``  -- 64^3, h = 1/32, R = 1.0, eps_r = 4.0, 8 channels.
  * ``metasurface``     -- 256x256x32 PB-phase nanofin array (Sec. III-B, Eq. 32).
  * ``metasurface_paper`` -- the same design at the paper's scale, 40 x 12 x 2
    wavelengths at 62 cells per wavelength (2480 x 744 x 124 cells).
  * ``random_body``     -- random unions of ellipsoids / cuboids, eps_r in [1.5, 6].
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

TWO_PI = 2.0 * math.pi


# --------------------------------------------------------------------------- #
# grids and voxelisation
# --------------------------------------------------------------------------- #
@dataclass
class Grid:
    """Uniform voxel grid: ``n`` cells per axis (x, y, z), spacing ``h``.

    Voxel (i, j, k) has its centre at ``origin + (idx - (n-1)/2) * h`` on each
    axis, so the grid centre sits at ``origin``.  Arrays over the grid are
    C-ordered ``[i][j][k]`` (z fastest).
    """

    n: tuple
    h: float
    origin: tuple = (0.0, 0.0, 0.0)

    def axes(self):
        return [self.origin[a] + (np.arange(self.n[a]) - 0.5 * (self.n[a] - 1)) * self.h
                for a in range(3)]

    def mesh(self):
        x, y, z = self.axes()
        return np.meshgrid(x, y, z, indexing="ij")

    @property
    def size(self):
        return int(self.n[0] * self.n[1] * self.n[2])


def sphere(grid: Grid, radius: float, eps_r: float, centre=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Relative permittivity of a homogeneous sphere: a voxel belongs to the body
    when its centre lies inside or on the sphere (centre-in rule)."""
    X, Y, Z = grid.mesh()
    d2 = (X - centre[0]) ** 2 + (Y - centre[1]) ** 2 + (Z - centre[2]) ** 2
    eps = np.ones(grid.n, dtype=np.float64)
    eps[d2 <= radius * radius] = eps_r
    return eps


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniformly distributed rotation matrix (QR of a Gaussian matrix, sign-fixed)."""
    a = rng.standard_normal((3, 3))
    q, r = np.linalg.qr(a)
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def random_body(seed: int, n_min: int = 32, n_max: int = 96, h: float = 1.0 / 20.0,
                n_axis: int | None = None):
    """Random lossless body: 1-3 primitives (ellipsoid or cuboid), each with
    semi-axes U[0.15, 0.45] x extent, a uniform random rotation, a centre in the
    inner 60 % of the box and eps_r ~ U[1.5, 6]; later primitives overwrite
    earlier ones.  The cubic grid size is drawn from U{n_min..n_max} unless
    ``n_axis`` is given.  Returns ``(Grid, eps_r)``."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(n_min, n_max + 1)) if n_axis is None else int(n_axis)
    grid = Grid((n, n, n), h)
    X, Y, Z = grid.mesh()
    P = np.stack([X, Y, Z], axis=-1)
    extent = n * h
    eps = np.ones(grid.n, dtype=np.float64)
    n_prim = int(rng.integers(1, 4))
    for _ in range(n_prim):
        kind = int(rng.integers(0, 2))  # 0 ellipsoid, 1 cuboid
        semi = rng.uniform(0.15, 0.45, size=3) * extent
        rot = _random_rotation(rng)
        c = (rng.uniform(-0.3, 0.3, size=3)) * extent
        er = float(rng.uniform(1.5, 6.0))
        loc = (P - c) @ rot  # coordinates in the primitive's frame
        if kind == 0:
            inside = np.sum((loc / semi) ** 2, axis=-1) <= 1.0
        else:
            inside = np.all(np.abs(loc) <= semi, axis=-1)
        eps[inside] = er
    if not np.any(eps > 1.0):  # guarantee a non-empty body
        eps[n // 2, n // 2, n // 2] = 2.0
    return grid, eps


# PB-phase metasurface (Sec. III-B).  Pitch p = 667 nm at lambda = 1550 nm.
META_PITCH = 667.0 / 1550.0
META_THETA_T_DEG = 10.0


def pb_rotation_increment_deg(pitch: float = META_PITCH, theta_t_deg: float = META_THETA_T_DEG,
                              k0: float = TWO_PI) -> float:
    """In-plane rotation step between adjacent cells of the PB design rule
    (Eq. 32): half of k0 * sin(theta_t) * p, in degrees."""
    return math.degrees(0.5 * k0 * math.sin(math.radians(theta_t_deg)) * pitch)


def metasurface(seed: int = 0, n=(256, 256, 32), fins=(8, 8), eps_r: float = 5.8,
                fin_size=(0.3, 0.1, 0.4)):
    """Glass-free PB-phase nanofin array on a ``n`` grid with h = p/32.

    Fin (m, q) sits at the centre of its p x p cell and is rotated in-plane by
    theta_{m,q} = theta0 + 0.5 k0 sin(10 deg) m p (Eq. 32; gradient along x);
    theta0 ~ U[0, pi) from ``seed``.  Returns ``(Grid, eps_r, angles)``."""
    rng = np.random.default_rng(seed)
    h = META_PITCH / 32.0
    grid = Grid(tuple(n), h)
    X, Y, Z = grid.mesh()
    eps = np.ones(grid.n, dtype=np.float64)
    theta0 = float(rng.uniform(0.0, math.pi))
    step = math.radians(pb_rotation_increment_deg())
    lx, ly, lz = (0.5 * s for s in fin_size)
    angles = np.zeros(fins)
    x0 = -0.5 * fins[0] * META_PITCH
    y0 = -0.5 * fins[1] * META_PITCH
    for m in range(fins[0]):
        for q in range(fins[1]):
            th = theta0 + step * m
            angles[m, q] = th
            cx = x0 + (m + 0.5) * META_PITCH
            cy = y0 + (q + 0.5) * META_PITCH
            dx, dy = X - cx, Y - cy
            u = math.cos(th) * dx + math.sin(th) * dy
            v = -math.sin(th) * dx + math.cos(th) * dy
            inside = (np.abs(u) <= lx) & (np.abs(v) <= ly) & (np.abs(Z) <= lz)
            eps[inside] = eps_r
    return grid, eps, angles


# The paper-scale PB metasurface (Sec. III-B): unit cells of pitch 667 nm with
# silicon nanofins (n = 3.44) of 486 x 219 x 830 nm at 1550 nm, simulated in a
# 40 x 12 x 2 wavelength box at 62 cells per wavelength.
META_FIN_PAPER = (486.0 / 1550.0, 219.0 / 1550.0, 830.0 / 1550.0)
META_EPS_SI = 3.44 ** 2

# Axis order of the paper-scale grid: grid axis a holds paper axis
# PAPER_AXES[a] (height first, the 40-wavelength axis last).  Swapping x and z
# is its own inverse; vectors map with ``to_grid_frame`` both ways.
PAPER_AXES = (2, 1, 0)


def to_grid_frame(v):
    """Map vectors (..., 3) between the paper frame and the paper-scale grid frame."""
    v = np.asarray(v)
    return v[..., list(PAPER_AXES)]


def metasurface_paper(cells_per_lambda: int = 62, box=(40.0, 12.0, 2.0), eps_r: float = META_EPS_SI,
                      theta0: float = 0.0):
    """Free-standing PB-phase silicon nanofin array filling a ``box`` (paper
    x, y, z in wavelengths) at ``cells_per_lambda``.

    Column m of fins (along the paper x axis) is rotated in-plane by
    theta0 + 0.5 k0 sin(10 deg) m p (Eq. 32); fins are centred in their p x p
    cells and in the box height; a voxel belongs to a fin when its centre does.
    The array is returned in the grid frame (axes ordered by ``PAPER_AXES``:
    shape (n_z, n_y, n_x)).  Returns ``(Grid, eps_r, info)`` with the fin
    counts and angles in ``info``."""
    h = 1.0 / cells_per_lambda
    n_p = tuple(int(round(b * cells_per_lambda)) for b in box)  # paper x, y, z
    n_g = tuple(n_p[a] for a in PAPER_AXES)
    eps = np.ones(n_g, dtype=np.float64)
    p = META_PITCH
    mx, my = int(box[0] // p), int(box[1] // p)
    l, d, hf = META_FIN_PAPER
    step = math.radians(pb_rotation_increment_deg())
    ax = [(np.arange(n_p[a]) - 0.5 * (n_p[a] - 1)) * h for a in range(3)]
    zsel = np.flatnonzero(np.abs(ax[2]) <= 0.5 * hf)
    z0, z1 = int(zsel[0]), int(zsel[-1]) + 1
    reach = 0.5 * math.hypot(l, d) + h
    angles = np.zeros((mx, my))
    for m in range(mx):
        th = theta0 + step * m
        c, s = math.cos(th), math.sin(th)
        cx = (m + 0.5 - 0.5 * mx) * p
        for q in range(my):
            angles[m, q] = th
            cy = (q + 0.5 - 0.5 * my) * p
            i0 = max(0, int(math.floor((cx - reach) / h + 0.5 * (n_p[0] - 1))))
            i1 = min(n_p[0], int(math.ceil((cx + reach) / h + 0.5 * (n_p[0] - 1))) + 1)
            j0 = max(0, int(math.floor((cy - reach) / h + 0.5 * (n_p[1] - 1))))
            j1 = min(n_p[1], int(math.ceil((cy + reach) / h + 0.5 * (n_p[1] - 1))) + 1)
            dx = ax[0][i0:i1, None] - cx
            dy = ax[1][None, j0:j1] - cy
            u = c * dx + s * dy
            v = -s * dx + c * dy
            inside = (np.abs(u) <= 0.5 * l) & (np.abs(v) <= 0.5 * d)  # [x][y]
            sub = eps[z0:z1, j0:j1, i0:i1]  # grid frame: [z][y][x]
            sub[:, inside.T] = eps_r
    # unit-cell boundaries as interior cut positions (first cell past each boundary), grid frame
    cuts_p = []
    for a, m in ((0, mx), (1, my)):
        cuts_p.append([int(math.floor((k - 0.5 * m) * p / h + 0.5 * (n_p[a] - 1))) + 1 for k in range(1, m)])
    cuts_p.append([])
    info = {"fins": (mx, my), "angles": angles, "n_paper": n_p, "z_cells": z1 - z0,
            "cell_cuts": [cuts_p[a] for a in PAPER_AXES]}
    return Grid(n_g, h), eps, info


def even_cuts(n: int, parts: int):
    """Interior cut positions splitting ``n`` cells into ``parts`` near-equal blocks."""
    return [int(round(k * n / parts)) for k in range(1, parts)]


# --------------------------------------------------------------------------- #
# incident channels and directions
# --------------------------------------------------------------------------- #
@dataclass
class Channel:
    """Incident plane wave E = pol * exp(i k0 khat . r) (e^{-i omega t})."""

    khat: np.ndarray
    pol: np.ndarray  # complex 3-vector, transverse to khat

    def as_array(self):
        """[khat(3) real, pol(3) complex interleaved] -> 9 doubles."""
        p = np.asarray(self.pol, dtype=np.complex128)
        return np.concatenate([np.asarray(self.khat, float),
                               np.stack([p.real, p.imag], axis=-1).ravel()])


def spherical_basis(theta: float, phi: float):
    """(rhat, e_theta, e_phi) for polar angle theta and azimuth phi (radians)."""
    st, ct, sp, cp = math.sin(theta), math.cos(theta), math.sin(phi), math.cos(phi)
    rhat = np.array([st * cp, st * sp, ct])
    eth = np.array([ct * cp, ct * sp, -st])
    eph = np.array([-sp, cp, 0.0])
    return rhat, eth, eph


def channels_two_plane_waves():
    """Two channels: x-polarised along +z, z-polarised along +x."""
    return [Channel(np.array([0.0, 0.0, 1.0]), np.array([1.0, 0.0, 0.0], complex)),
            Channel(np.array([1.0, 0.0, 0.0]), np.array([0.0, 0.0, 1.0], complex))]


def channels_paper_sphere():
    """The paper's sphere channels (Sec. III-A): y-polarised along +x,
    x-polarised along +y."""
    return [Channel(np.array([1.0, 0.0, 0.0]), np.array([0.0, 1.0, 0.0], complex)),
            Channel(np.array([0.0, 1.0, 0.0]), np.array([1.0, 0.0, 0.0], complex))]


def channels_four_angles_two_pol():
    """8 channels: khat at theta in {0,45,90,135} deg in the xz-plane,
    polarisation e_theta then e_phi for each."""
    out = []
    for th in (0.0, 45.0, 90.0, 135.0):
        k, et, ep = spherical_basis(math.radians(th), 0.0)
        out.append(Channel(k, et.astype(complex)))
        out.append(Channel(k, ep.astype(complex)))
    return out


def channels_metasurface(thetas_deg=None):
    """Incidence angles theta_s (signed, xz-plane, propagating +z); for each,
    L then R circular polarisation p = (e_theta +/- i e_phi)/sqrt(2) (Eq. 28)."""
    if thetas_deg is None:
        thetas_deg = np.arange(-31.0, 31.0 + 1e-9, 2.0)
    out = []
    for ts in thetas_deg:
        t = math.radians(ts)
        k = np.array([math.sin(t), 0.0, math.cos(t)])
        et = np.array([math.cos(t), 0.0, -math.sin(t)])
        ep = np.array([0.0, 1.0, 0.0])
        out.append(Channel(k, (et + 1j * ep) / math.sqrt(2.0)))
        out.append(Channel(k, (et - 1j * ep) / math.sqrt(2.0)))
    return out


def fibonacci_directions(count: int):
    """``count`` quasi-uniform unit vectors on the sphere (Fibonacci lattice)."""
    golden = math.pi * (3.0 - math.sqrt(5.0))
    out = []
    for i in range(count):
        z = 1.0 - 2.0 * (i + 0.5) / count
        r = math.sqrt(max(0.0, 1.0 - z * z))
        ph = golden * i
        out.append(np.array([r * math.cos(ph), r * math.sin(ph), z]))
    return out


def channels_fibonacci(count: int):
    """For each of ``count`` Fibonacci directions: e_theta then e_phi."""
    out = []
    for k in fibonacci_directions(count):
        th = math.acos(max(-1.0, min(1.0, k[2])))
        ph = math.atan2(k[1], k[0])
        _, et, ep = spherical_basis(th, ph)
        out.append(Channel(k, et.astype(complex)))
        out.append(Channel(k, ep.astype(complex)))
    return out


def channels_array(chs) -> np.ndarray:
    """Pack channels as an ``[n][9]`` float64 array (khat, pol re/im interleaved)."""
    return np.stack([c.as_array() for c in chs]).astype(np.float64)


def angle_grid(theta_deg, phi_deg):
    """Product direction grid in radians: (theta[nt], phi[np])."""
    return np.radians(np.asarray(theta_deg, float)), np.radians(np.asarray(phi_deg, float))


def directions_from_angles(theta, phi):
    """Unit vectors for every (theta, phi) pair, theta-major: ``[nt*np][3]``."""
    T, P = np.meshgrid(theta, phi, indexing="ij")
    return np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], -1).reshape(-1, 3)


def random_field(grid: Grid, n_rhs: int, seed: int, mask=None) -> np.ndarray:
    """Seeded complex test vector ``[n_rhs][3][n0][n1][n2]`` (unit normal parts),
    zero outside ``mask`` when one is given."""
    rng = np.random.default_rng(seed)
    shp = (n_rhs, 3) + tuple(grid.n)
    w = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    if mask is not None:
        w = w * mask[None, None]
    return w


# Named workloads ----------------------------------------------------------------
@dataclass
class Workload:
    name: str
    grid: Grid
    eps: np.ndarray
    channels: list
    k0: float = TWO_PI
    extra: dict = field(default_factory=dict)


def sphere16_workload() -> Workload:
    g = Grid((16, 16, 16), 1.0 / 20.0)
    return Workload("sphere16_R0.4_eps2.25", g, sphere(g, 0.4, 2.25), channels_two_plane_waves(),
                    extra=dict(theta_deg=np.arange(0.0, 180.0 + 1e-9, 5.0),
                               phi_deg=np.arange(0.0, 355.0 + 1e-9, 5.0),
                               detectors_deg=((60.0, 0.0), (60.0, 180.0)),
                               sigma=1.2, dtau=np.arange(-5.0, 5.0 + 1e-9, 0.01)))


def sphere64_workload() -> Workload:
    g = Grid((64, 64, 64), 1.0 / 32.0)
    return Workload("sphere64_R1.0_eps4", g, sphere(g, 1.0, 4.0), channels_four_angles_two_pol(),
                    extra=dict(theta_deg=np.arange(0.0, 180.0 + 1e-9, 1.0),
                               phi_deg=np.arange(0.0, 359.0 + 1e-9, 1.0)))


def random_body_workload(seed: int, n_axis: int | None = None, n_dirs: int = 8,
                         h: float = 1.0 / 20.0) -> Workload:
    g, eps = random_body(seed, n_axis=n_axis, h=h)
    return Workload(f"random_body_s{seed}_n{g.n[0]}", g, eps, channels_fibonacci(n_dirs))
