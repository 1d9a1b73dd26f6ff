"""GPU parity of the FFT engine and the FFT-VIE operator against the oracle.

The operator y = w - chi (K * w) (Sec. II-C, Eq. 24 in the w unknown) from the
CUDA path is compared element by element with the oracle's direct-sum
convolution on the same seeded inputs.  FP64 path: 1e-11 relative to max|y|
(FFT round-off over ~log2(P^3) stages); FP32 path: 2e-5 (single-precision
FFT round-off, ~10 eps32 * log2 P per pass).
"""
import math

import numpy as np
import pytest

from oracle import vie as ovie
from paper_2508_16471_gb300 import inputs
from sample_points import pick_voxels

pytestmark = pytest.mark.gpu
K0 = 2.0 * math.pi
TOL64 = 1e-11
TOL32 = 2e-5


@pytest.mark.parametrize("L", [1, 2, 3, 7, 16, 32, 75, 96, 125, 128, 192, 256, 343, 512, 1024, 1500, 4096, 5000,
                               6561, 8192])
def test_fft_lines_vs_numpy(vielib, L):
    rng = np.random.default_rng(L)
    x = rng.standard_normal((5, L)) + 1j * rng.standard_normal((5, L))
    ref = np.fft.fft(x, axis=1)
    refi = np.fft.ifft(x, axis=1) * L
    s = np.abs(ref).max()
    assert np.abs(vielib.fft_lines(x, precision=vielib.PREC_MIXED) - ref).max() <= 2e-6 * s * max(1, math.log2(L))
    if L > 6400:
        # two FP64 line buffers of L points exceed the shared memory of one CTA
        with pytest.raises(vielib.VieError):
            vielib.fft_lines(x, precision=vielib.PREC_FP64)
        return
    assert np.abs(vielib.fft_lines(x, precision=vielib.PREC_FP64) - ref).max() <= 1e-13 * s * max(1, math.log2(L))
    assert np.abs(vielib.fft_lines(x, inverse=True, precision=vielib.PREC_FP64) - refi).max() <= 1e-13 * s * max(1, math.log2(L))


def _case_random(n, seed, fill=0.6):
    rng = np.random.default_rng(seed)
    eps = 1.0 + rng.uniform(0.2, 4.0, n) * (rng.uniform(size=n) < fill)
    if not np.any(eps > 1):
        eps.flat[0] = 2.0
    return eps


def _check_apply(vielib, n, h, eps, R=2, seed=0):
    mask = eps > 1.0
    g = inputs.Grid(n, h)
    w = inputs.random_field(g, R, seed, mask)
    chi = ovie.contrast(eps)
    T = ovie.kernel_table(n, h, K0)
    ref = np.stack([ovie.apply_direct(T, n, chi, w[r]) for r in range(R)])
    with vielib.Handle(n, h, eps, K0) as hd:
        y64 = hd.apply(w, precision=vielib.PREC_FP64)
        y32 = hd.apply(w, precision=vielib.PREC_MIXED)
        ydf = hd.apply(w, precision=vielib.PREC_F32X2)
    s = np.abs(ref).max()
    e64 = np.abs(y64 - ref).max() / s
    e32 = np.abs(y32 - ref).max() / s
    edf = np.abs(ydf - ref).max() / s
    assert e64 <= TOL64, e64
    assert e32 <= TOL32, e32
    assert edf <= TOL64, edf  # double-float arithmetic meets the FP64 tolerance


@pytest.mark.parametrize("n", [(1, 1, 1), (2, 3, 1), (5, 6, 4), (7, 5, 9), (12, 10, 7)])
def test_apply_small_ragged_grids(vielib, n):
    _check_apply(vielib, n, 0.07, _case_random(n, sum(n)))


def test_apply_sphere16(vielib):
    wl = inputs.sphere16_workload()
    _check_apply(vielib, wl.grid.n, wl.grid.h, wl.eps, R=3)


def test_apply_full_body_and_single_voxel_body(vielib):
    n = (6, 6, 6)
    _check_apply(vielib, n, 0.05, np.full(n, 3.0))
    eps = np.ones(n)
    eps[2, 3, 4] = 2.5
    _check_apply(vielib, n, 0.05, eps)


def test_apply_nonsmooth_sizes(vielib):
    # 2n-1 = 73 -> P = 75 (radix 3, 5), 2n-1 = 21 -> P = 21
    n = (37, 11, 6)
    eps = _case_random(n, 5, fill=0.3)
    mask = eps > 1.0
    g = inputs.Grid(n, 0.04)
    w = inputs.random_field(g, 1, 3, mask)
    chi = ovie.contrast(eps)
    ref = ovie.apply_direct(ovie.kernel_table(n, 0.04, K0), n, chi, w[0])[None]
    with vielib.Handle(n, 0.04, eps, K0) as hd:
        assert hd.info()["P"] == (75, 21, 12)
        y64 = hd.apply(w, precision=vielib.PREC_FP64)
    assert np.abs(y64 - ref).max() <= TOL64 * np.abs(ref).max()


def _sampled_parity(vielib, n, h, eps, R, seed, nsamp, prec_list):
    g = inputs.Grid(n, h)
    mask = eps > 1.0
    w = inputs.random_field(g, R, seed, mask)
    body = np.argwhere(mask)
    rng = np.random.default_rng(seed + 1)
    pts = body[rng.choice(len(body), size=min(nsamp, len(body)), replace=False)]
    chi = ovie.contrast(eps)
    out = {}
    with vielib.Handle(n, h, eps, K0) as hd:
        for p in prec_list:
            out[p] = hd.apply(w, precision=p)
    convs = ovie.convolve_direct_points_multi(n, h, K0, w, pts)
    for r in range(R):
        conv = convs[r]
        ref = np.stack([w[r][:, a, b, c] - chi[a, b, c] * conv[:, i] for i, (a, b, c) in enumerate(pts)], 1)
        s = np.abs(ref).max()
        for p, tol in ((vielib.PREC_FP64, TOL64), (vielib.PREC_MIXED, TOL32), (vielib.PREC_F32X2, TOL64)):
            if p not in out:
                continue
            got = np.stack([out[p][r][:, a, b, c] for (a, b, c) in pts], 1)
            assert np.abs(got - ref).max() <= tol * s, (p, np.abs(got - ref).max() / s)


def test_apply_sphere64_sampled(vielib):
    wl = inputs.sphere64_workload()
    _sampled_parity(vielib, wl.grid.n, wl.grid.h, wl.eps, 2, 11, 24,
                    (vielib.PREC_FP64, vielib.PREC_MIXED, vielib.PREC_F32X2))


def test_apply_bench_size_sampled(vielib):
    """The 128^3 random-body workload the bench times, 4 RHS, sampled voxels;
    the double-float operator is the one the bench's residuals use."""
    wl = inputs.random_body_workload(20000, n_axis=128, h=1.0 / 128.0)
    _sampled_parity(vielib, wl.grid.n, wl.grid.h, wl.eps, 4, 12, 6,
                    (vielib.PREC_MIXED, vielib.PREC_FP64, vielib.PREC_F32X2))


@pytest.mark.parametrize("n", [(16, 16, 16), (32, 24, 20), (64, 64, 64)])
def test_fast_and_generic_fft_paths_agree(vielib, n):
    """Register four-step kernels (power-of-two padded axes) vs the generic
    shared-memory Stockham kernels, FP32, on the same vectors."""
    rng = np.random.default_rng(7)
    eps = 1.0 + rng.uniform(0.3, 3.0, n) * (rng.uniform(size=n) < 0.5)
    g = inputs.Grid(n, 0.03)
    w = inputs.random_field(g, 3, 9, eps > 1.0)
    with vielib.Handle(n, 0.03, eps, K0) as hd:
        y_fast = hd.apply(w, precision=vielib.PREC_MIXED)
        hd.set_fft_path(1)
        y_gen = hd.apply(w, precision=vielib.PREC_MIXED)
        y64 = hd.apply(w, precision=vielib.PREC_FP64)
    s = np.abs(y64).max()
    assert np.abs(y_fast - y64).max() <= TOL32 * s
    assert np.abs(y_gen - y64).max() <= TOL32 * s


def test_autotune_keeps_the_operator(vielib):
    """The autotuner times the candidate padded lengths (80 on the mixed-radix
    engine, 128 on the register or generic power-of-two kernels for a 40^3
    grid) and keeps the fastest; the operator's values must not change beyond
    rounding (FP64 1e-11, FP32 2e-5 of max |y|)."""
    wl = inputs.random_body_workload(11, n_dirs=1)
    g = wl.grid
    assert g.n[0] == 40
    w = inputs.random_field(g, 2, 3, wl.eps > 1.0)  # [2][3][n0][n1][n2], zero outside the body
    with vielib.Handle(g.n, g.h, wl.eps, wl.k0) as hd:
        y64 = hd.apply(w, precision=vielib.PREC_FP64)
        P, ms = hd.autotune(n_rhs=4, reps=2)
        assert P[0] == P[1] == P[2] and P[0] in (80, 128) and ms > 0
        assert tuple(hd.info()["P"]) == P
        z64 = hd.apply(w, precision=vielib.PREC_FP64)
        z32 = hd.apply(w, precision=vielib.PREC_MIXED)
    s = np.abs(y64).max()
    assert np.abs(z64 - y64).max() <= 1e-11 * s
    assert np.abs(z32 - y64).max() <= 2e-5 * s


@pytest.mark.parametrize("n", [(3, 4, 2500), (3, 700, 4), (2, 620, 30)])
def test_apply_long_padded_axes(vielib, n):
    """Padded lengths beyond 1024 (5000 on z, 1400 and 1250 on y): one line or
    four columns per CTA with the twiddles read from global memory, against the
    oracle's FFT operator (itself pinned to the direct sum)."""
    rng = np.random.default_rng(sum(n))
    eps = 1.0 + rng.uniform(0.3, 3.0, n) * (rng.uniform(size=n) < 0.5)
    h = 0.02
    g = inputs.Grid(n, h)
    w = inputs.random_field(g, 2, 4, eps > 1.0)
    op = ovie.FFTOperator(n, h, K0, ovie.contrast(eps), workers=-1)
    ref = np.stack([op(w[r]) for r in range(2)])
    with vielib.Handle(n, h, eps, K0) as hd:
        assert max(hd.info()["P"]) > 1024
        y64 = hd.apply(w, precision=vielib.PREC_FP64)
        y32 = hd.apply(w, precision=vielib.PREC_MIXED)
    s = np.abs(ref).max()
    assert np.abs(y64 - ref).max() <= TOL64 * s
    assert np.abs(y32 - ref).max() <= TOL32 * s


def test_first_axis_too_long_is_rejected(vielib):
    """The fused x pass keeps three components of a column in shared memory,
    which bounds the first padded length (about 3200 at FP64): set-up refuses
    a longer first axis before any kernel runs."""
    n = (2000, 2, 2)
    eps = np.full(n, 2.0)
    with pytest.raises(vielib.VieError) as e:
        vielib.Handle(n, 0.02, eps, K0)
    assert "first axis" in str(e.value)


def _apply_sampled(vielib, g, eps, R, seed, rr, count):
    """One FP32 application of R random vectors through the device layout;
    ``count`` picked voxels of the RHS ``rr`` against the oracle's direct sum
    over all source voxels."""
    import torch
    mask = eps > 1.0
    vox = np.flatnonzero(mask)
    Nb = len(vox)
    rng = np.random.default_rng(seed)
    w = (rng.standard_normal((R, 3, Nb)) + 1j * rng.standard_normal((R, 3, Nb))).astype(np.complex64)
    with vielib.Handle(g.n, g.h, eps, K0) as hd:
        wd = torch.from_numpy(w).cuda().contiguous()
        yd = torch.full_like(wd, complex(float("nan"), 0.0))
        torch.cuda.synchronize()  # the library runs on its own stream
        hd.apply_device(wd.data_ptr(), yd.data_ptr(), R, vielib.PREC_MIXED)
        torch.cuda.synchronize()
        y = yd.cpu().numpy().astype(np.complex128)
    assert np.isfinite(y).all()
    pts = pick_voxels(mask, count, seed)
    lin = np.ravel_multi_index(tuple(pts.T), g.n)
    picks = np.searchsorted(vox, lin)
    assert np.array_equal(vox[picks], lin)
    src = np.stack(np.unravel_index(vox, g.n), -1)
    conv = ovie.convolve_points_sparse(src, w[rr].astype(np.complex128), g.h, K0, pts)  # (len(rr), 3, T)
    chi = eps.reshape(-1)[lin] - 1.0
    for q, r in enumerate(rr):
        ref = w[r][:, picks] - chi[None, :] * conv[q]
        assert np.abs(y[r][:, picks] - ref).max() <= TOL32 * np.abs(ref).max(), r


def test_apply_bench_launch_configuration_sampled(vielib):
    """The bench's launch configuration: the 128^3 body, 32 RHS in one FP32
    operator application (32 slots per fused-x launch, next-slot prefetch)
    through the device layout; 32 voxels (the body's extreme ones along each
    axis, the ones nearest the grid corners, surface and random ones) of the
    first, a middle and the last RHS against the oracle's direct sum over all
    sources."""
    wl = inputs.random_body_workload(20000, n_axis=128, h=1.0 / 128.0)
    _apply_sampled(vielib, wl.grid, wl.eps, 32, 77, [0, 17, 31], 32)


def test_apply_128_body_filling_the_grid_sampled(vielib):
    """A 128^3 random medium that fills the grid (40 % of the voxels, all eight
    corners included), 4 RHS: the voxels where zero padding and cropping act
    (grid corners and faces) against the oracle's direct sum."""
    n = (128, 128, 128)
    rng = np.random.default_rng(128)
    eps = 1.0 + rng.uniform(0.5, 3.0, n) * (rng.uniform(size=n) < 0.4)
    for c in np.stack(np.meshgrid([0, 127], [0, 127], [0, 127], indexing="ij"), -1).reshape(-1, 3):
        eps[tuple(c)] = 2.5
    g = inputs.Grid(n, 1.0 / 128.0)
    _apply_sampled(vielib, g, eps, 4, 78, [0, 3], 32)
