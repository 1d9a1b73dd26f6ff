"""FP64 NumPy reference of the learned initial-guess network (test
infrastructure only; only ``tests/`` may import it).

A 4-level 3-D U-Net on a cubic grid of D^3 voxels (D divisible by 8):

  enc0: conv(cin->c0) relu conv(c0->c0) relu          -> s0   (D^3)
  pool: 2x2x2 average
  enc1: conv(c0->c1) relu conv(c1->c1) relu           -> s1   ((D/2)^3)
  enc2: conv(c1->c2) relu conv(c2->c2) relu           -> s2   ((D/4)^3)
  bott: conv(c2->c3) relu conv(c3->c3) relu                   ((D/8)^3)
  dec2: up2(nearest) ++ s2 -> conv(c3+c2->c2) relu conv(c2->c2) relu
  dec1: up2 ++ s1          -> conv(c2+c1->c1) relu conv(c1->c1) relu
  dec0: up2 ++ s0          -> conv(c1+c0->c0) relu conv(c0->c0) relu
  head: 1x1x1 conv(c0->6)

Every 3x3x3 convolution is zero-padded ("same") and has a bias.  Arrays are
[batch][channel][x][y][z].  The loss is a masked mean squared error.  The
backward pass is written out layer by layer (chain rule), pinned by central
finite differences in tests/test_oracle_net.py.
"""
from __future__ import annotations

import numpy as np

OFFS = [(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)]


def layer_specs(c=(16, 32, 64, 128), cin=10, cout=6):
    """List of (name, Cin, Cout, ksize) in the order the network applies them."""
    c0, c1, c2, c3 = c
    return [("e0a", cin, c0, 3), ("e0b", c0, c0, 3), ("e1a", c0, c1, 3), ("e1b", c1, c1, 3),
            ("e2a", c1, c2, 3), ("e2b", c2, c2, 3), ("b_a", c2, c3, 3), ("b_b", c3, c3, 3),
            ("d2a", c3 + c2, c2, 3), ("d2b", c2, c2, 3), ("d1a", c2 + c1, c1, 3), ("d1b", c1, c1, 3),
            ("d0a", c1 + c0, c0, 3), ("d0b", c0, c0, 3), ("head", c0, cout, 1)]


def init_params(specs, seed=0):
    """He-normal weights [Cout][Cin][k^3], zero biases."""
    rng = np.random.default_rng(seed)
    P = {}
    for name, ci, co, k in specs:
        fan_in = ci * k ** 3
        P[name + ".w"] = rng.standard_normal((co, ci, k ** 3)) * np.sqrt(2.0 / fan_in)
        P[name + ".b"] = np.zeros(co)
    return P


def _shift(x, o):
    """y[..., i, j, k] = x[..., i+o0, j+o1, k+o2] with zeros outside."""
    y = np.zeros_like(x)
    D = x.shape[-3:]
    src = tuple(slice(max(0, oo), D[a] + min(0, oo)) for a, oo in enumerate(o))
    dst = tuple(slice(max(0, -oo), D[a] - max(0, oo)) for a, oo in enumerate(o))
    y[(Ellipsis,) + dst] = x[(Ellipsis,) + src]
    return y


def conv3(x, w, b):
    """'same' 3x3x3 convolution (cross-correlation): out[n,co,v] =
    b[co] + sum_{ci,k} w[co,ci,k] x[n,ci,v+off_k]."""
    if w.shape[2] == 1:
        return np.einsum("oc,nc...->no...", w[:, :, 0], x) + b[None, :, None, None, None]
    out = np.zeros((x.shape[0], w.shape[0]) + x.shape[2:])
    for k, o in enumerate(OFFS):
        out += np.einsum("oc,nc...->no...", w[:, :, k], _shift(x, o))
    return out + b[None, :, None, None, None]


def _outer(gy, x):
    """sum over batch and voxels of gy[n,o,v] x[n,c,v] -> [o][c]."""
    n, o = gy.shape[:2]
    c = x.shape[1]
    return np.einsum("nov,ncv->oc", gy.reshape(n, o, -1), x.reshape(n, c, -1))


def conv3_backward(x, w, gy):
    """Gradients of conv3 w.r.t. x, w, b given dL/dy."""
    gb = gy.sum(axis=(0, 2, 3, 4))
    if w.shape[2] == 1:
        gw = _outer(gy, x)[:, :, None]
        gx = np.einsum("oc,no...->nc...", w[:, :, 0], gy)
        return gx, gw, gb
    gw = np.zeros_like(w)
    gx = np.zeros_like(x)
    for k, o in enumerate(OFFS):
        xs = _shift(x, o)
        gw[:, :, k] = _outer(gy, xs)
        # y[v] gets x[v+o]  =>  dx[u] += w^T gy[u-o]
        gx += _shift(np.einsum("oc,no...->nc...", w[:, :, k], gy), tuple(-oo for oo in o))
    return gx, gw, gb


def pool2(x):
    n, c, a, b, d = x.shape
    return x.reshape(n, c, a // 2, 2, b // 2, 2, d // 2, 2).mean(axis=(3, 5, 7))


def pool2_backward(g):
    return np.repeat(np.repeat(np.repeat(g, 2, 2), 2, 3), 2, 4) / 8.0


def up2(x):
    return np.repeat(np.repeat(np.repeat(x, 2, 2), 2, 3), 2, 4)


def up2_backward(g):
    n, c, a, b, d = g.shape
    return g.reshape(n, c, a // 2, 2, b // 2, 2, d // 2, 2).sum(axis=(3, 5, 7))


def forward(P, x, specs, keep=False):
    """Network output (and, with keep=True, the cache for backward)."""
    cache = {}

    def cr(name, h):
        z = conv3(h, P[name + ".w"], P[name + ".b"])
        a = np.maximum(z, 0.0)
        if keep:
            cache[name] = (h, z)
        return a

    s0 = cr("e0b", cr("e0a", x))
    s1 = cr("e1b", cr("e1a", pool2(s0)))
    s2 = cr("e2b", cr("e2a", pool2(s1)))
    bt = cr("b_b", cr("b_a", pool2(s2)))
    d2 = cr("d2b", cr("d2a", np.concatenate([up2(bt), s2], axis=1)))
    d1 = cr("d1b", cr("d1a", np.concatenate([up2(d2), s1], axis=1)))
    d0 = cr("d0b", cr("d0a", np.concatenate([up2(d1), s0], axis=1)))
    y = conv3(d0, P["head.w"], P["head.b"])
    if keep:
        cache["head"] = (d0, None)
        cache["dims"] = dict(c0=s0.shape[1], c1=s1.shape[1], c2=s2.shape[1], c3=bt.shape[1])
    return (y, cache) if keep else y


def loss(y, t, m):
    """Masked MSE: sum m (y - t)^2 / (sum over the mask's support x channels)."""
    d = (y - t) * m
    den = max(float(np.sum(m)) * y.shape[1] / m.shape[1], 1.0)
    return float(np.sum(d * d) / den), 2.0 * d * m / den


def backward(P, cache, gy):
    """dL/dP for every parameter (and dL/dx under the key "input"), given
    dL/d(output)."""
    G = {}
    d0, _ = cache["head"]
    gx, G["head.w"], G["head.b"] = conv3_backward(d0, P["head.w"], gy)
    dims = cache["dims"]

    def crb(name, g):
        h, z = cache[name]
        g = g * (z > 0)
        gh, G[name + ".w"], G[name + ".b"] = conv3_backward(h, P[name + ".w"], g)
        return gh

    g = crb("d0a", crb("d0b", gx))
    g_up, g_s0 = g[:, :dims["c1"]], g[:, dims["c1"]:]
    g = crb("d1a", crb("d1b", up2_backward(g_up)))
    g_up, g_s1 = g[:, :dims["c2"]], g[:, dims["c2"]:]
    g = crb("d2a", crb("d2b", up2_backward(g_up)))
    g_up, g_s2 = g[:, :dims["c3"]], g[:, dims["c3"]:]
    g = crb("b_a", crb("b_b", up2_backward(g_up)))
    g_s2 = g_s2 + pool2_backward(g)
    g = crb("e2a", crb("e2b", g_s2))
    g_s1 = g_s1 + pool2_backward(g)
    g = crb("e1a", crb("e1b", g_s1))
    g_s0 = g_s0 + pool2_backward(g)
    G["input"] = crb("e0a", crb("e0b", g_s0))
    return G


def adam_step(P, G, state, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba) of every parameter, in place."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in P:
        if k == "input":
            continue
        m = state.setdefault("m." + k, np.zeros_like(P[k]))
        v = state.setdefault("v." + k, np.zeros_like(P[k]))
        m[...] = b1 * m + (1 - b1) * G[k]
        v[...] = b2 * v + (1 - b2) * G[k] ** 2
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        P[k] = P[k] - lr * mh / (np.sqrt(vh) + eps)
    return P
