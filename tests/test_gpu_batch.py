"""Multi-body batches (vie_batch_*): bodies of uneven grids whose FP32
operator runs in one launch per pass and padded size, each row with its own
grid, voxel map, contrast and kernel spectrum.

Bodies come from the random-body generator with the 1-lambda-box reading
(h = 1/n per body, so every body has its own kernel); their padded sizes are
64 and 128, so a batch exercises both the several-bodies-per-launch path and
the per-size grouping.  Checked against each body's own single-body operator
and solve, and against the oracle's direct sum."""
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
SIZES = (20, 27, 33, 45)  # padded 64, 64, 128, 128


def _bodies(sizes=SIZES, seed0=300):
    out = []
    for i, n in enumerate(sizes):
        g, eps = inputs.random_body(seed0 + i, n_axis=n, h=1.0 / n)
        out.append((g.n, g.h, eps))
    return out


def test_batch_operator_matches_single_bodies_and_oracle(vielib):
    import torch
    bodies = _bodies()
    R = 3
    with vielib.Batch(bodies, K0) as bt:
        S = bt.stride
        Ps = [bt.info(b)["P"][0] for b in range(len(bodies))]
        assert Ps == [64, 64, 128, 128]
        Nbs = [bt.info(b)["n_body"] for b in range(len(bodies))]
        assert S == max(Nbs)
        rng = np.random.default_rng(5)
        W = np.zeros((len(bodies) * R, 3, S), dtype=np.complex128)
        for b, nb in enumerate(Nbs):
            W[b * R:(b + 1) * R, :, :nb] = rng.standard_normal((R, 3, nb)) + 1j * rng.standard_normal((R, 3, nb))
        outs = {}
        for prec, dt in ((vielib.PREC_MIXED, np.complex64), (vielib.PREC_FP64, np.complex128),
                         (vielib.PREC_F32X2, np.complex128)):
            w_h = np.ascontiguousarray(W, dtype=dt)
            wd = torch.from_numpy(w_h).cuda()
            yd = torch.zeros_like(wd)
            torch.cuda.synchronize()  # the library runs on its own stream
            bt.apply_device(wd.data_ptr(), yd.data_ptr(), R, prec)
            torch.cuda.synchronize()
            outs[prec] = yd.cpu().numpy().astype(np.complex128)
    for b, (n, h, eps) in enumerate(bodies):
        nb = Nbs[b]
        wb = W[b * R:(b + 1) * R, :, :nb]
        # the body's own single-body operator (its own padded size) on the same vectors
        mask = eps > 1.0
        vox = np.flatnonzero(mask)
        full = np.zeros((R, 3) + tuple(n), dtype=np.complex128)
        full.reshape(R, 3, -1)[:, :, vox] = wb
        with vielib.Handle(n, h, eps, K0) as hd:
            y1 = hd.apply(full, precision=vielib.PREC_FP64).reshape(R, 3, -1)[:, :, vox]
        s = np.abs(y1).max()
        assert np.abs(outs[vielib.PREC_MIXED][b * R:(b + 1) * R, :, :nb] - y1).max() <= TOL32 * s, b
        assert np.abs(outs[vielib.PREC_FP64][b * R:(b + 1) * R, :, :nb] - y1).max() <= TOL64 * s, b
        assert np.abs(outs[vielib.PREC_F32X2][b * R:(b + 1) * R, :, :nb] - y1).max() <= TOL64 * s, b
        # entries beyond the body's own size are not written
        assert not np.any(outs[vielib.PREC_MIXED][b * R:(b + 1) * R, :, nb:])
        # the oracle's direct sum at 32 picked voxels of the first RHS
        pts = pick_voxels(mask, 32, b)
        src = np.stack(np.unravel_index(vox, n), -1)
        conv = ovie.convolve_points_sparse(src, wb[:1], h, K0, pts)[0]  # (3, T)
        lin = np.ravel_multi_index(tuple(pts.T), n)
        picks = np.searchsorted(vox, lin)
        chi = eps.reshape(-1)[lin] - 1.0
        ref = wb[0][:, picks] - chi[None, :] * conv
        got = outs[vielib.PREC_MIXED][b * R, :, picks].T
        assert np.abs(got - ref).max() <= TOL32 * np.abs(ref).max(), b
        got64 = outs[vielib.PREC_F32X2][b * R, :, picks].T
        assert np.abs(got64 - ref).max() <= TOL64 * np.abs(ref).max(), b


def test_batch_solve_matches_single_body_solves(vielib):
    """Three bodies of uneven grids, 4 channels each, solved together (one
    GMRES over the 12 rows, the FP32 operator in one launch per pass and
    padded size) to an FP64 residual of 1e-10: currents and far fields equal
    those of each body's own solve."""
    bodies = _bodies((24, 33, 40), seed0=310)
    chs = [(c.khat, c.pol) for c in inputs.channels_fibonacci(2)]
    dirs = inputs.directions_from_angles(np.radians([20.0, 75.0, 130.0]), np.radians([0.0, 110.0, 250.0]))
    with vielib.Batch(bodies, K0) as bt:
        st = bt.solve(chs, tol=1e-10, restart=60)
        assert st["converged"] == 3 * len(chs) and st["relres_max"] <= 1e-10
        Wb = [np.stack([bt.get_current(b, r) for r in range(len(chs))]) for b in range(3)]
        Fb = [bt.farfield_dirs(b, dirs) for b in range(3)]
    for b, (n, h, eps) in enumerate(bodies):
        with vielib.Handle(n, h, eps, K0) as hd:
            s1 = hd.solve(chs, tol=1e-10, restart=60)
            assert s1["converged"] == len(chs)
            W1 = np.stack([hd.get_current(r) for r in range(len(chs))])
            F1 = hd.farfield_dirs(dirs)
        assert np.abs(Wb[b] - W1).max() <= 1e-8 * np.abs(W1).max(), b
        assert np.abs(Fb[b] - F1).max() <= 1e-8 * np.abs(F1).max(), b


def test_batch_rejects_bad_input(vielib):
    n = (8, 8, 8)
    eps = np.full(n, 2.0)
    with pytest.raises(vielib.VieError):
        vielib.Batch([(n, 0.1, eps), ((200, 2, 2), 0.1, np.full((200, 2, 2), 2.0))], K0)
    with pytest.raises(vielib.VieError):
        vielib.Batch([(n, 0.1, np.ones(n))], K0)
    with vielib.Batch([(n, 0.1, eps)], K0) as bt:
        with pytest.raises(vielib.VieError):
            bt.solve([((0, 0, 1.0), (1.0, 0, 0))], solver=vielib.SOLVER_BICGSTAB)
        with pytest.raises(vielib.VieError):
            bt.get_current(0, 0)  # no solution yet
