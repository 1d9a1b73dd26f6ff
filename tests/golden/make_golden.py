"""Write the stored oracle results that the GPU parity tests compare against.

Calls only ``oracle/`` and the seeded input generators (which hold no
arithmetic of the method).  Every file records the workload, the channels, the
oracle's solver tolerance, iteration counts and the residuals it reached.

    python tests/golden/make_golden.py sphere64   # 64^3 sphere, R = 1 lambda, eps_r = 4, 8 channels
    python tests/golden/make_golden.py body64     # random body at 64^3 (1-lambda box), 16 channels

Each channel is solved in its own process (the oracle's FP64 GMRES, or its
COCR for the resonant sphere, both with the oracle's FFT operator, itself
pinned to the direct sum) to a relative residual of 1e-10;
the far field (Eq. 25) of each solution is evaluated by the oracle's direct
sum on the configuration's product grid of directions and stored as its
(theta, phi) components in complex64 (the r component vanishes identically;
complex64 keeps 6e-8 relative precision, far below the 1e-5 tolerance), and in
each channel's own (forward) direction in complex128, for the optical theorem.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

TOL = 1e-10


def _workload(name):
    """(workload, theta, phi, oracle solver, GMRES restart)"""
    from paper_2508_16471_gb300 import inputs
    if name == "sphere64":
        # the resonant sphere: restarted GMRES needs about 2e4 iterations to 1e-10 (restart 150), the
        # short-recurrence COCR about 1e3
        wl = inputs.sphere64_workload()
        th, ph = inputs.angle_grid(wl.extra["theta_deg"], wl.extra["phi_deg"])  # 181 x 360
        return wl, th, ph, "cocr", 0
    if name == "body64":
        wl = inputs.random_body_workload(BODY64_SEED, n_axis=64, h=1.0 / 64.0, n_dirs=8)
        th, ph = inputs.angle_grid(np.arange(0.0, 180.0 + 1e-9, 5.0), np.arange(0.0, 355.0 + 1e-9, 5.0))
        return wl, th, ph, "fft", 100
    raise ValueError(name)


BODY64_SEED = 3


def _one_channel(args):
    name, j = args
    from oracle import vie as ovie
    from paper_2508_16471_gb300 import inputs
    wl, th, ph, method, restart = _workload(name)
    g = wl.grid
    c = wl.channels[j]
    t0 = time.time()
    w, infos = ovie.solve_channels(g.n, g.h, wl.k0, wl.eps, [(c.khat, c.pol)], tol=TOL, restart=restart,
                                   maxiter=200000, workers=1, method=method)
    t_solve = time.time() - t0
    dirs = inputs.directions_from_angles(th, ph)
    F = ovie.farfield(w[0], g.n, g.h, wl.k0, dirs)
    Fs = ovie.project(F, dirs, 1)[:, :2].reshape(len(th), len(ph), 2)
    Ffwd = ovie.farfield(w[0], g.n, g.h, wl.k0, np.asarray(c.khat, float)[None])[0]  # forward, Cartesian
    print(f"{name} channel {j}: {infos[0]['iters']} iterations, relres {infos[0]['relres']:.2e}, "
          f"solve {t_solve:.0f} s, far field {time.time() - t0 - t_solve:.0f} s", flush=True)
    return j, Fs.astype(np.complex64), infos[0]["iters"], infos[0]["relres"], t_solve, Ffwd


def make(name, procs=None):
    # one solve per process, each single-threaded
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    wl, th, ph, method, restart = _workload(name)
    R = len(wl.channels)
    ctx = mp.get_context("spawn")
    t0 = time.time()
    with ctx.Pool(processes=procs or min(R, os.cpu_count() or 1)) as pool:
        res = sorted(pool.map(_one_channel, [(name, j) for j in range(R)]))
    F = np.stack([r[1] for r in res])  # [R][nt][np][2] (F_theta, F_phi)
    iters = np.array([r[2] for r in res])
    relres = np.array([r[3] for r in res])
    F_fwd = np.stack([r[5] for r in res])  # [R][3] complex128, far field in each channel's own direction
    assert np.all(relres <= TOL), relres
    out = os.path.join(HERE, f"{name}_farfield.npz")
    np.savez_compressed(out, F_theta_phi=F, F_forward=F_fwd, theta=th, phi=ph, tol=TOL, solver=method,
                        restart=restart, iters=iters,
                        relres=relres, seconds=time.time() - t0, workload=wl.name,
                        khat=np.stack([c.khat for c in wl.channels]), pol=np.stack([c.pol for c in wl.channels]))
    print(out, iters.tolist(), relres.max(), f"{time.time() - t0:.0f} s")


if __name__ == "__main__":
    for which in (sys.argv[1:] or ["sphere64", "body64"]):
        make(which)
