"""Write stored oracle results used by the GPU parity tests.

Calls only ``oracle/`` (and the seeded input generators).  Each output file
records the workload, the channels, the oracle solver tolerance and the
residual reached.

    python tests/golden/make_golden.py sphere64   # 64^3 sphere, R = 1, eps_r = 4
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import vie as ovie  # noqa: E402
from paper_2508_16471_gb300 import inputs  # noqa: E402


def sphere64(channels=(0, 5), tol=1e-9, restart=200):
    wl = inputs.sphere_config2()
    g = wl.grid
    chs = [(wl.channels[i].khat, wl.channels[i].pol) for i in channels]
    th = np.radians(np.arange(0.0, 181.0, 15.0))
    ph = np.radians(np.arange(0.0, 360.0, 30.0))
    dirs = inputs.directions_from_angles(th, ph)
    t = time.time()
    w, infos = ovie.solve_channels(g.n, g.h, wl.k0, wl.eps, chs, tol=tol, restart=restart,
                                   maxiter=200000, workers=-1)
    F = np.stack([ovie.farfield(w[j], g.n, g.h, wl.k0, dirs) for j in range(len(chs))])
    out = os.path.join(HERE, "sphere64_farfield.npz")
    np.savez_compressed(out, F=F, theta=th, phi=ph, channels=np.array(channels),
                        tol=tol, iters=np.array([i["iters"] for i in infos]),
                        relres=np.array([i["relres"] for i in infos]), seconds=time.time() - t,
                        workload=wl.name)
    print(out, [i["iters"] for i in infos], [i["relres"] for i in infos], time.time() - t)


if __name__ == "__main__":
    which = sys.argv[1] if len(sys.argv) > 1 else "sphere64"
    {"sphere64": sphere64}[which]()
