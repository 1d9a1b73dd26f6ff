"""The PB metasurface at the paper's scale (Sec. III-B: a 40 x 12 x 2 wavelength
box at 62 cells per wavelength, 2480 x 744 x 124 cells; 92 x 27 silicon
nanofins, 14.4 million fin voxels, 43 million unknowns).

The FP64 and FP32 operators of the CUDA path are applied to a seeded random
current on the fin voxels and compared, at sampled fin voxels, with the
oracle's direct sum over every source.  The grid puts the box height first and
the 40-wavelength axis last (padded 256 x 1500 x 5000): the long axes run on
the one-line / four-column generic FFT kernels, and one FP32 work array holds
2.8e9 complex values, beyond 32-bit indexing.  About 140 GB of device memory."""
import math

import numpy as np
import pytest

from oracle import vie as ovie
from paper_2508_16471_gb300 import inputs

pytestmark = pytest.mark.gpu
K0 = 2.0 * math.pi


def test_paper_scale_operator_sampled(vielib):
    import torch
    g, eps, info = inputs.metasurface_paper()
    assert g.n == (124, 744, 2480) and info["fins"] == (92, 27)
    vox = np.flatnonzero(eps > 1.0)
    Nb = len(vox)
    rng = np.random.default_rng(2508)
    w = rng.standard_normal((3, Nb)) + 1j * rng.standard_normal((3, Nb))
    picks = np.array([0, Nb - 1, int(rng.integers(Nb)), int(rng.integers(Nb))])
    with vielib.Handle(g.n, g.h, eps, K0) as hd:
        inf = hd.info()
        assert inf["n_body"] == Nb and inf["P"] == (256, 1500, 5000)
        out = {}
        for prec, dt in ((vielib.PREC_FP64, torch.complex128), (vielib.PREC_MIXED, torch.complex64)):
            w_h = np.ascontiguousarray(w, dtype=np.complex128)  # kept alive until the copy is done
            wd = torch.from_numpy(w_h).to(dt).cuda().reshape(1, 3, Nb).contiguous()
            yd = torch.full_like(wd, complex(float("nan"), 0.0))
            torch.cuda.synchronize()  # the library runs on its own stream
            hd.apply_device(wd.data_ptr(), yd.data_ptr(), 1, prec)
            torch.cuda.synchronize()
            y = yd[0].cpu().numpy().astype(np.complex128)
            assert np.isfinite(y).all()
            out[prec] = y[:, picks]
            del wd, yd
    src = np.stack(np.unravel_index(vox, g.n), -1)
    conv = ovie.convolve_points_sparse(src, w[None], g.h, K0, src[picks])[0]  # (3, T)
    chi = eps.reshape(-1)[vox[picks]] - 1.0
    ref = w[:, picks] - chi[None, :] * conv
    s = np.abs(ref).max()
    e64 = np.abs(out[vielib.PREC_FP64] - ref).max() / s
    e32 = np.abs(out[vielib.PREC_MIXED] - ref).max() / s
    assert e64 <= 1e-11, e64
    assert e32 <= 2e-5, e32
