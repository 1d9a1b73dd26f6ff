"""Pins of the oracle's discrete operator A w = w - chi (K * w) and its solver:
dense assembly vs direct sum vs FFT convolution (Sec. II-C: the voxel grid
makes the MoM matrix a convolution, applied by zero-padded FFTs), FFT size
independence, and GMRES vs dense LU."""
import math

import numpy as np

from oracle import vie

K0 = 2.0 * math.pi


def _case(n, seed):
    rng = np.random.default_rng(seed)
    chi = rng.uniform(0.0, 2.0, n)
    w = rng.standard_normal((3,) + n) + 1j * rng.standard_normal((3,) + n)
    return chi, w


def test_dense_direct_fft_agree_nonsquare():
    n = (5, 6, 4)
    h = 0.08
    chi, w = _case(n, 1)
    A = vie.dense_operator(n, h, K0, chi)
    yd = (A @ w.reshape(-1)).reshape(w.shape)
    ys = vie.apply_direct(vie.kernel_table(n, h, K0), n, chi, w)
    yf = vie.FFTOperator(n, h, K0, chi)(w)
    s = np.abs(yd).max()
    assert np.abs(yd - ys).max() <= 1e-12 * s
    assert np.abs(yd - yf).max() <= 1e-12 * s


def test_dense_8cubed_direct_sum():
    n = (8, 8, 8)
    h = 1.0 / 20.0
    chi, w = _case(n, 2)
    A = vie.dense_operator(n, h, K0, chi)
    yd = (A @ w.reshape(-1)).reshape(w.shape)
    ys = vie.apply_direct(vie.kernel_table(n, h, K0), n, chi, w)
    assert np.abs(yd - ys).max() <= 1e-12 * np.abs(yd).max()


def test_fft_padded_size_independence():
    n = (7, 5, 6)
    h = 0.1
    chi, w = _case(n, 3)
    y1 = vie.FFTOperator(n, h, K0, chi)(w)
    y2 = vie.FFTOperator(n, h, K0, chi, P=(18, 15, 11))(w)
    y3 = vie.FFTOperator(n, h, K0, chi, P=(13, 9, 12))(w)  # minimal 2n-1
    s = np.abs(y1).max()
    assert np.abs(y1 - y2).max() <= 1e-12 * s
    assert np.abs(y1 - y3).max() <= 1e-12 * s


def test_sampled_direct_points_match_table_sum():
    n = (9, 7, 8)
    h = 0.06
    _, w = _case(n, 4)
    T = vie.kernel_table(n, h, K0)
    full = vie.convolve_direct(T, n, w)
    pts = np.array([[0, 0, 0], [8, 6, 7], [4, 3, 2], [1, 5, 6]])
    s = vie.convolve_direct_points(n, h, K0, w, pts)
    ref = np.stack([full[:, a, b, c] for a, b, c in pts], axis=1)
    assert np.abs(s - ref).max() <= 1e-12 * np.abs(ref).max()


def test_gmres_matches_lu_8cubed():
    n = (8, 8, 8)
    h = 1.0 / 20.0
    rng = np.random.default_rng(5)
    eps = 1.0 + rng.uniform(0.0, 3.0, n) * (rng.uniform(size=n) < 0.6)
    chi = vie.contrast(eps)
    b = vie.rhs(chi, vie.incident_field(n, h, K0, [0, 0, 1.0], [1.0, 0, 0]))
    A = vie.dense_operator(n, h, K0, chi)
    x_lu = np.linalg.solve(A, b.reshape(-1)).reshape(b.shape)
    op = vie.FFTOperator(n, h, K0, chi)
    x_g, info = vie.gmres(op, b, tol=1e-12, restart=30)
    assert info["converged"]
    assert np.abs(x_g - x_lu).max() <= 1e-10 * np.abs(x_lu).max()
    # unknowns outside the body stay exactly zero
    assert np.abs(x_lu[:, chi == 0]).max() < 1e-13 * np.abs(x_lu).max()


def test_smooth_size():
    assert vie.smooth_size(255) == 256
    assert vie.smooth_size(73) == 75
    assert vie.smooth_size(121) == 125
    assert vie.smooth_size(191) == 192


def test_multi_point_direct_sum_matches_single():
    n = (6, 5, 4)
    h = 0.08
    rng = np.random.default_rng(8)
    W = rng.standard_normal((2, 3) + n) + 1j * rng.standard_normal((2, 3) + n)
    pts = np.array([[0, 0, 0], [5, 4, 3], [2, 1, 2]])
    multi = vie.convolve_direct_points_multi(n, h, K0, W, pts)
    for r in range(2):
        single = vie.convolve_direct_points(n, h, K0, W[r], pts)
        assert np.abs(multi[r] - single).max() <= 1e-13 * np.abs(single).max()


def test_sparse_source_direct_sum_matches_table_sum():
    """The source-list direct sum (used where dense fields do not fit in host
    memory) equals the table convolution over the dense field with zeros off
    the list, whatever the chunking."""
    n = (5, 7, 6)
    h = 0.06
    rng = np.random.default_rng(21)
    mask = rng.uniform(size=n) < 0.4
    W = (rng.standard_normal((2, 3) + n) + 1j * rng.standard_normal((2, 3) + n)) * mask
    src = np.argwhere(mask)
    Wsrc = np.stack([W[:, :, a, b, c] for (a, b, c) in src], -1)
    pts = np.array([[0, 0, 0], [4, 6, 5], [2, 3, 1], [1, 5, 4]])
    T = vie.kernel_table(n, h, K0)
    for chunk in (7, 1 << 20):
        got = vie.convolve_points_sparse(src, Wsrc, h, K0, pts, chunk=chunk)
        for r in range(2):
            ref = vie.convolve_direct(T, n, W[r], targets=pts)
            assert np.abs(got[r] - ref).max() <= 1e-13 * np.abs(ref).max()


def test_operator_is_symmetric_in_the_contrast_weighted_bilinear_form():
    """Reciprocity of the discrete kernel (K_ab(m) = K_ba(-m)) makes
    A = I - diag(chi) K symmetric in [x, y] = sum x_i y_i / chi_i: diag(1/chi) A
    equals its transpose (not its conjugate transpose).  This is the structure
    the COCR solver relies on; a dropped transpose or a conjugated kernel
    breaks it."""
    n = (4, 3, 5)
    h = 0.07
    rng = np.random.default_rng(12)
    chi = rng.uniform(0.3, 9.0, n)
    A = vie.dense_operator(n, h, K0, chi)
    mu = np.tile(1.0 / chi.reshape(-1), 3)
    MA = mu[:, None] * A
    s = np.abs(MA).max()
    assert np.abs(MA - MA.T).max() <= 1e-14 * s
    assert np.abs(MA - MA.conj().T).max() > 1e-3 * s  # complex symmetric, not Hermitian


def test_d2_operator_is_symmetric_in_the_face_contrast_weighted_form():
    """The same for the rooftop / pulse operator: y = w - chi_f (K2 w) with the
    face contrast chi_f; K2 (scalar kernel plus staggered grad-div) is
    symmetric, so diag(1/chi_f) A is, on the faces with chi_f > 0."""
    from oracle import d2
    n = (3, 3, 3)
    h = 0.08
    rng = np.random.default_rng(13)
    eps = 1.0 + rng.uniform(0.5, 5.0, n)
    eps[0] = 1.0
    chi = vie.contrast(eps)
    chi_f = d2.face_contrast(chi)
    keep = np.flatnonzero(chi_f.reshape(-1) > 0)
    cols = []
    for j in keep:
        e = np.zeros(chi_f.size, dtype=np.complex128)
        e[j] = 1.0
        cols.append(d2.apply_direct(n, h, K0, chi_f, e.reshape((3,) + n)).reshape(-1)[keep])
    A = np.stack(cols, 1)
    MA = A / chi_f.reshape(-1)[keep][:, None]
    s = np.abs(MA).max()
    assert np.abs(MA - MA.T).max() <= 1e-13 * s


def test_oracle_cocr_matches_dense_lu_and_gmres():
    """The oracle's COCR (short recurrence on the complex symmetric
    diag(1/chi) A) reaches the dense-LU solution on a small random body with a
    varying contrast and the GMRES solution of the 16^3 sphere, each to 1e-9 of
    the solution's size; its reported residual is the operator's own."""
    import math
    from oracle import vie as ovie
    from paper_2508_16471_gb300 import inputs
    k0 = 2.0 * math.pi
    rng = np.random.default_rng(21)
    n = (6, 5, 4)
    eps = 1.0 + rng.uniform(0.5, 4.0, n) * (rng.uniform(size=n) < 0.6)
    chs = [((0.0, 0.0, 1.0), (1.0, 0.0, 0.0)), ((0.6, 0.0, 0.8), (0.0, 1.0, 0.0))]
    w_lu, _ = ovie.solve_channels(n, 0.07, k0, eps, chs, method="lu")
    w_co, inf = ovie.solve_channels(n, 0.07, k0, eps, chs, method="cocr", tol=1e-12)
    assert all(i["converged"] and i["relres"] <= 1e-12 for i in inf)
    assert np.abs(w_co - w_lu).max() <= 1e-9 * np.abs(w_lu).max()
    wl = inputs.sphere16_workload()
    g = wl.grid
    chs1 = [(c.khat, c.pol) for c in wl.channels]
    w_g, _ = ovie.solve_channels(g.n, g.h, wl.k0, wl.eps, chs1, tol=1e-12)
    w_c, inf = ovie.solve_channels(g.n, g.h, wl.k0, wl.eps, chs1, method="cocr", tol=1e-12)
    assert all(i["converged"] for i in inf)
    assert np.abs(w_c - w_g).max() <= 1e-9 * np.abs(w_g).max()
