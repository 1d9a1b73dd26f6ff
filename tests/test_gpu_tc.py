"""Tensor-core (tcgen05, 3xTF32) complex GEMM of the far-field contraction vs
an FP64 NumPy product, and the two far-field engines against each other and
the oracle.  Tolerance 2e-5 relative (3xTF32 keeps ~FP32 accuracy; the sums
here have <= 256 terms)."""
import math

import numpy as np
import pytest

from oracle import vie as ovie
from paper_2508_16471_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K", [(128, 32, 16), (200, 37, 23), (1, 1, 1), (300, 181, 64), (1500, 360, 64),
                                   (129, 33, 17)])
@pytest.mark.parametrize("engine", [0, 1])
def test_cgemm_engines(vielib, M, N, K, engine):
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))
    B = rng.standard_normal((K, N)) + 1j * rng.standard_normal((K, N))
    C = vielib.cgemm(A, B, engine=engine)
    ref = A @ B
    err = np.abs(C - ref).max() / np.abs(ref).max()
    assert err < 2e-5, err


def test_farfield_engines_agree_with_oracle(vielib):
    wl = inputs.sphere16_workload()
    g = wl.grid
    chs = [(c.khat, c.pol) for c in wl.channels]
    th, ph = inputs.angle_grid(wl.extra["theta_deg"], wl.extra["phi_deg"])
    dirs = inputs.directions_from_angles(th, ph)
    with vielib.Handle(g.n, g.h, wl.eps, wl.k0) as hd:
        hd.solve(chs, tol=1e-10, restart=40)
        w = np.stack([hd.get_current(r) for r in range(2)])
        hd.set_farfield_engine(0)
        F_tc = hd.farfield(th, ph).reshape(2, -1, 3)
        hd.set_farfield_engine(1)
        F_cc = hd.farfield(th, ph).reshape(2, -1, 3)
    F_or = np.stack([ovie.farfield(w[j], g.n, g.h, wl.k0, dirs) for j in range(2)])
    for F in (F_tc, F_cc):
        assert np.linalg.norm(F - F_or) / np.linalg.norm(F_or) < 1e-5
        assert np.abs(F - F_or).max() / np.abs(F_or).max() < 1e-5
