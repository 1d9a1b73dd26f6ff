"""Pins of the oracle's learned-initial-guess network: every analytic gradient
(convolutions, pooling, upsampling, skip concatenations, ReLU, masked MSE)
against central finite differences, the conv against a direct loop, and the
Adam update against its closed form for one step."""
import numpy as np
import pytest

from oracle import net

SPECS = net.layer_specs(c=(2, 3, 2, 4), cin=7, cout=6)


def _setup(seed=0, D=8):
    rng = np.random.default_rng(seed)
    P = net.init_params(SPECS, seed=seed)
    for k in P:
        if k.endswith(".b"):
            P[k] = rng.standard_normal(P[k].shape) * 0.1
    x = rng.standard_normal((2, 7, D, D, D))
    t = rng.standard_normal((2, 6, D, D, D))
    m = (rng.uniform(size=(2, 1, D, D, D)) < 0.6).astype(float)
    return P, x, t, m


def _L(P, x, t, m):
    return net.loss(net.forward(P, x, SPECS), t, m)[0]


def test_conv3_matches_direct_loop():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((1, 2, 4, 3, 5))
    w = rng.standard_normal((3, 2, 27))
    b = rng.standard_normal(3)
    y = net.conv3(x, w, b)
    ref = np.zeros_like(y)
    for o in range(3):
        for i in range(4):
            for j in range(3):
                for k in range(5):
                    acc = b[o]
                    for q, (a, bb, c) in enumerate(net.OFFS):
                        ii, jj, kk = i + a, j + bb, k + c
                        if 0 <= ii < 4 and 0 <= jj < 3 and 0 <= kk < 5:
                            acc += w[o, :, q] @ x[0, :, ii, jj, kk]
                    ref[0, o, i, j, k] = acc
    assert np.abs(y - ref).max() < 1e-12


def test_parameter_gradients_match_finite_differences():
    P, x, t, m = _setup()
    y, cache = net.forward(P, x, SPECS, keep=True)
    _, gy = net.loss(y, t, m)
    G = net.backward(P, cache, gy)
    rng = np.random.default_rng(2)
    h = 1e-6
    for name in P:
        flat = P[name].reshape(-1)
        for idx in rng.choice(flat.size, size=min(3, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = _L(P, x, t, m)
            flat[idx] = old - h
            lm = _L(P, x, t, m)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = G[name].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (name, idx, fd, an)


def test_input_gradient_through_the_whole_net():
    """d loss / d input by finite differences vs the chain of backward ops
    (covers the skip connections and pooling at every level)."""
    P, x, t, m = _setup(3)
    y, cache = net.forward(P, x, SPECS, keep=True)
    _, gy = net.loss(y, t, m)
    G = net.backward(P, cache, gy)
    rng = np.random.default_rng(4)
    h = 1e-6
    for _ in range(6):
        idx = tuple(int(rng.integers(0, s)) for s in x.shape)
        x2 = x.copy()
        x2[idx] += h
        lp = _L(P, x2, t, m)
        x2[idx] -= 2 * h
        lm = _L(P, x2, t, m)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - G["input"][idx]) <= 1e-6 * max(1.0, abs(fd))


def test_adam_first_step_closed_form():
    P = {"a": np.array([1.0, -2.0])}
    G = {"a": np.array([0.5, -4.0])}
    st = {}
    net.adam_step(P, G, st, lr=0.1)
    # first step: m/(1-b1) = g, v/(1-b2) = g^2 -> update = lr * g / (|g| + eps)
    assert np.allclose(P["a"], np.array([1.0 - 0.1, -2.0 + 0.1]), atol=1e-7)
