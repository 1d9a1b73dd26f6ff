"""Training pipelines of the learned initial guess and the learned
preconditioner (solver-generated data).

The library solves seeded random bodies, extracts (features, targets, mask)
on the coarse grid with vie_net_features / vie_precond_pairs and trains the
networks with vie_net_train_step; all arithmetic runs in the library's
kernels, PyTorch only holds the device buffers.
"""
from __future__ import annotations

import numpy as np

from . import inputs
from . import vie as V


def generate(n_axis, h, seeds, n_dirs, factor, restart=64, tol=1e-6, max_iter=20000):
    """Solve one body per seed (all on one grid) and return device tensors
    X [S][10][D^3], T [S][6][D^3], M [S][D^3] (float32) with S = 2 n_dirs per body,
    plus the solver iteration counts."""
    import torch
    D = n_axis // factor
    Vc = D ** 3
    Xs, Ts, Ms, iters = [], [], [], []
    hd = None
    try:
        for seed in seeds:
            wl = inputs.random_body_workload(seed, n_axis=n_axis, h=h, n_dirs=n_dirs)
            if hd is None:
                hd = V.Handle(wl.grid.n, wl.grid.h, wl.eps, wl.k0)
            else:
                hd.set_eps(wl.eps)
            chs = [(c.khat, c.pol) for c in wl.channels]
            st = hd.solve(chs, tol=tol, restart=restart, max_iter=max_iter, allow_noconv=True)
            R = len(chs)
            x = torch.empty(R, 10, Vc, device="cuda")
            t = torch.empty(R, 6, Vc, device="cuda")
            m = torch.empty(R, Vc, device="cuda")
            torch.cuda.synchronize()  # the library runs on the handle's own stream
            hd.net_features(factor, x.data_ptr(), t.data_ptr(), m.data_ptr())
            torch.cuda.synchronize()
            Xs.append(x)
            Ts.append(t)
            Ms.append(m)
            iters.append(st["iters"])
    finally:
        if hd is not None:
            hd.close()
    return torch.cat(Xs), torch.cat(Ts), torch.cat(Ms), np.concatenate(iters)


def train(net, X, T, M, D, epochs=20, batch=8, lr=2e-3, seed=0, lr_decay=0.9):
    """Minibatch Adam over the samples; returns the mean loss per epoch."""
    import torch
    S = X.shape[0]
    rng = np.random.default_rng(seed)
    hist = []
    for ep in range(epochs):
        perm = rng.permutation(S)
        tot, nb = 0.0, 0
        for b0 in range(0, S - batch + 1, batch):
            idx = torch.as_tensor(perm[b0:b0 + batch], device=X.device)
            xb = X.index_select(0, idx).contiguous()
            tb = T.index_select(0, idx).contiguous()
            mb = M.index_select(0, idx).contiguous()
            torch.cuda.synchronize()  # the network runs on its own stream
            tot += net.train_step(xb.data_ptr(), tb.data_ptr(), mb.data_ptr(), batch, D, lr)
            nb += 1
        hist.append(tot / max(nb, 1))
        lr *= lr_decay
    return hist


def generate_precond(n_axis, h, seeds, n_dirs, factor, powers=3, restart=64, tol=1e-6, max_iter=20000):
    """Training pairs of the learned preconditioner: for each body, the solved
    currents w and their images A w, A^2 w, ... (the early Krylov directions
    of the solves) are the vectors v; vie_precond_pairs forms u = A v and the
    coarse-grid features of u with the targets (v - u).  Returns device
    tensors X [S][7][D^3], T [S][6][D^3], M [S][D^3]."""
    import torch
    D = n_axis // factor
    Vc = D ** 3
    Xs, Ts, Ms = [], [], []
    hd = None
    try:
        for seed in seeds:
            wl = inputs.random_body_workload(seed, n_axis=n_axis, h=h, n_dirs=n_dirs)
            if hd is None:
                hd = V.Handle(wl.grid.n, wl.grid.h, wl.eps, wl.k0)
            else:
                hd.set_eps(wl.eps)
            chs = [(c.khat, c.pol) for c in wl.channels]
            hd.solve(chs, tol=tol, restart=restart, max_iter=max_iter, allow_noconv=True)
            R = len(chs)
            body = np.asarray(wl.eps).reshape(-1) != 1.0
            W = np.stack([hd.get_current(r).reshape(3, -1)[:, body] for r in range(R)]).astype(np.complex64)
            v = torch.from_numpy(W).cuda().contiguous()
            for k in range(powers + 1):
                x = torch.empty(R, 7, Vc, device="cuda")
                t = torch.empty(R, 6, Vc, device="cuda")
                m = torch.empty(R, Vc, device="cuda")
                torch.cuda.synchronize()  # the library runs on the handle's own stream
                hd.precond_pairs(factor, v.data_ptr(), R, x.data_ptr(), t.data_ptr(), m.data_ptr())
                Xs.append(x)
                Ts.append(t)
                Ms.append(m)
                if k < powers:
                    u = torch.empty_like(v)
                    hd.apply_device(v.data_ptr(), u.data_ptr(), R, V.PREC_MIXED)
                    v = u
                torch.cuda.synchronize()
    finally:
        if hd is not None:
            hd.close()
    return torch.cat(Xs), torch.cat(Ts), torch.cat(Ms)
