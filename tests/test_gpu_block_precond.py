"""Block-Jacobi preconditioner (the block preconditioner of Sec. III-B; FGMRES
with opts.precond = 2).

The block operator A_bd = I - diag(chi) K_bd (K_bd keeps the interactions
between voxels of the same block) runs as one batched FFT operator with a
voxel map per block; it is checked against the oracle's FFT operator applied
to each block's part of the vector on its own.  The preconditioned solve must
reach the same discrete solution as plain GMRES."""
import math

import numpy as np
import pytest

from oracle import vie as ovie
from paper_2508_16471_gb300 import inputs

pytestmark = pytest.mark.gpu
K0 = 2.0 * math.pi


def _block_ref(g, eps, w, cuts):
    """Oracle: y = w - chi (K * w_t) on the voxels of block t, for every block."""
    chi = ovie.contrast(eps)
    vox = np.flatnonzero(chi > 0)
    ijk = np.stack(np.unravel_index(vox, g.n), -1)
    tid = np.zeros(len(vox), dtype=np.int64)
    for a in range(3):
        tid = tid * (len(cuts[a]) + 1) + np.searchsorted(np.asarray(cuts[a], int), ijk[:, a], side="right")
    op = ovie.FFTOperator(g.n, g.h, K0, chi, workers=-1)
    chiv = chi.reshape(-1)[vox]
    ref = np.zeros_like(w)
    for t in np.unique(tid):
        sel = tid == t
        full = np.zeros((3,) + tuple(g.n), dtype=np.complex128)
        for c in range(3):
            full[c].reshape(-1)[vox[sel]] = w[c, sel]
        conv = op.convolve(full)
        for c in range(3):
            ref[c, sel] = w[c, sel] - chiv[sel] * conv[c].reshape(-1)[vox[sel]]
    return ref, len(np.unique(tid))


def _gpu_block_apply(vielib, g, eps, w, cuts):
    import torch
    with vielib.Handle(g.n, g.h, eps, K0) as hd:
        hd.set_block_precond(cuts, inner=4)
        w_h = np.ascontiguousarray(w, dtype=np.complex64)  # kept alive until the copy is done
        wd = torch.from_numpy(w_h).cuda().contiguous()
        yd = torch.full_like(wd, complex(float("nan"), 0.0))
        torch.cuda.synchronize()  # the library runs on its own stream
        hd.block_apply_device(wd.data_ptr(), yd.data_ptr())
        torch.cuda.synchronize()
        return yd.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("case", ["fins", "random"])
def test_block_operator_matches_oracle(vielib, case):
    if case == "fins":  # 2 x 2 fins, one per block (cuts between the unit cells)
        g, eps, _ = inputs.metasurface(seed=0, n=(64, 64, 32), fins=(2, 2))
        cuts = ([32], [32], [])
    else:  # a random body cut through on every axis: 18 blocks, some partly filled
        g, eps = inputs.random_body(3, n_min=30, n_max=30)
        cuts = ([10, 20], [16], [5, 27])
    Nb = int((eps > 1.0).sum())
    rng = np.random.default_rng(5)
    w = rng.standard_normal((3, Nb)) + 1j * rng.standard_normal((3, Nb))
    ref, T = _block_ref(g, eps, w, cuts)
    y = _gpu_block_apply(vielib, g, eps, w, cuts)
    s = np.abs(ref).max()
    assert np.isfinite(y).all()
    assert np.abs(y - ref).max() <= 2e-5 * s
    if case == "random":
        assert T > 4
        # the cross-block interactions are really gone: the full operator differs
        chi = ovie.contrast(eps)
        vox = np.flatnonzero(chi > 0)
        full = np.zeros((3,) + tuple(g.n), dtype=np.complex128)
        for c in range(3):
            full[c].reshape(-1)[vox] = w[c]
        yf = ovie.FFTOperator(g.n, g.h, K0, chi, workers=-1)(full).reshape(3, -1)[:, vox]
        assert np.abs(yf - ref).max() > 1e-2 * s


def test_block_preconditioned_solve_matches_plain(vielib):
    """Reduced PB metasurface (2 x 2 fins), L/R/H/V channels: FGMRES with the
    fin-cell block-Jacobi preconditioner reaches the plain GMRES currents in
    fewer outer iterations."""
    g, eps, _ = inputs.metasurface(seed=0, n=(64, 64, 32), fins=(2, 2))
    LR = inputs.channels_metasurface([0.0])
    chs = [(c.khat, c.pol) for c in LR] + [(np.array([0, 0, 1.0]), np.array([1.0, 0, 0], complex)),
                                           (np.array([0, 0, 1.0]), np.array([0, 1.0, 0], complex))]
    with vielib.Handle(g.n, g.h, eps, K0) as hd:
        st0 = hd.solve(chs, tol=1e-8, restart=64, max_iter=20000)
        W0 = np.stack([hd.get_current(r) for r in range(4)])
        hd.set_block_precond(([32], [32], []), inner=8)
        st1 = hd.solve(chs, tol=1e-8, restart=64, max_iter=20000, precond=2)
        W1 = np.stack([hd.get_current(r) for r in range(4)])
    assert st0["converged"] == 4 and st1["converged"] == 4 and st1["relres_max"] <= 1e-8
    assert np.abs(W1 - W0).max() <= 1e-6 * np.abs(W0).max()
    assert st1["iters"].max() < st0["iters"].max()


def test_block_precond_options(vielib):
    g, eps, _ = inputs.metasurface(seed=0, n=(64, 64, 32), fins=(2, 2))
    chs = [(c.khat, c.pol) for c in inputs.channels_metasurface([0.0])]
    with vielib.Handle(g.n, g.h, eps, K0) as hd:
        with pytest.raises(vielib.VieError):  # not set up
            hd.solve(chs, precond=2)
        with pytest.raises(vielib.VieError):  # cut outside the grid
            hd.set_block_precond(([64], [], []))
        with pytest.raises(vielib.VieError):  # cuts not increasing
            hd.set_block_precond(([20, 10], [], []))
        hd.set_block_precond(([32], [32], []), inner=2)
        with pytest.raises(vielib.VieError):  # FP64 basis
            hd.solve(chs, precond=2, precision=vielib.PREC_FP64)
        with pytest.raises(vielib.VieError):  # BiCGStab
            hd.solve(chs, precond=2, solver=vielib.SOLVER_BICGSTAB)
        hd.set_eps(eps)  # a new body drops the blocks
        with pytest.raises(vielib.VieError):
            hd.solve(chs, precond=2)
    n = (18, 18, 18)
    e2 = np.ones(n)
    e2[4:14, 4:14, 4:14] = 2.0
    with vielib.Handle(n, 0.05, e2, K0, disc=vielib.DISC_D2) as hd:
        with pytest.raises(vielib.VieError):
            hd.set_block_precond(([9], [], []))
