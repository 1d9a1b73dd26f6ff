"""The one-sweep Arnoldi recurrence that the GPU solver runs (opts.arnoldi = 1),
modelled step by step in NumPy with the basis rounded to complex64 after every
vector operation, as the FP32 basis is on the device, on the oracle's operator
of a small random body.

Per step j the model applies the operator to the pending (not yet
orthogonalised) vector y_j, forms v_j = (y_j - V lag) / beta_j, the next pending
vector B v_j = (B y_j - V_{j} (H_B lag)) / beta_j through the Arnoldi relation of
B = A - sigma I, and the Hessenberg column from the inner products of the
basis with B y_j (Pythagorean norm); A step whose orthogonal part is below
eta ||B v||^2 takes two explicit classical passes.  Checked: with sigma = 1 the
Arnoldi relation A V_m = V_{m+1} H holds to FP32 level and the basis stays
orthonormal as with classical Gram-Schmidt; unshifted (sigma = 0) the
recurrence amplifies its rounding errors until the basis is lost, which is why
the solver runs it on A - I (the scattering part -chi K of A = I - chi K)."""
import math

import numpy as np

from oracle import vie as ovie
from paper_2508_16471_gb300 import inputs

K0 = 2.0 * math.pi


def _operator(n_axis=12, seed=20003):
    g, eps = inputs.random_body(seed, n_axis=n_axis, h=1.0 / n_axis)
    chi = ovie.contrast(eps)
    op = ovie.FFTOperator(g.n, g.h, K0, chi)
    mask = chi > 0
    nb = int(mask.sum())

    def A(v):
        full = np.zeros((3,) + g.n, dtype=complex)
        full[:, mask] = v.reshape(3, nb)
        return op(full)[:, mask].reshape(-1)

    return A, 3 * nb


def _f32(x):
    return x.astype(np.complex64).astype(complex)


def _one_sweep(A, b, m, sigma, eta=0.1):
    n = b.size
    V = np.zeros((m + 1, n), complex)
    H = np.zeros((m + 1, m), complex)   # Hessenberg of A (what GMRES rotates)
    Hu = np.zeros((m + 1, m), complex)  # Hessenberg of B = A - sigma I
    lag = np.zeros(m + 1, complex)
    V[0] = _f32(b / np.linalg.norm(b))
    inv = 0.0
    flagged = 0
    for j in range(m):
        if j == 0:  # nothing lagged: the classical first step on A v_0
            V[1] = _f32(A(V[0]))
            coef = np.array([np.vdot(V[0], V[1]), np.vdot(V[1], V[1])])
            H[0, 0] = coef[0]
        else:
            u = V[j]
            z = _f32(A(u)) - sigma * u                    # B y_j
            c = Hu[:j + 1, :j] @ lag[:j]                   # B V_{j-1} lag in the basis
            V[j] = _f32((u - lag[:j] @ V[:j]) * inv)       # v_j
            V[j + 1] = _f32((z - c @ V[:j + 1]) * inv)     # pending B v_j
            g = V[:j + 1].conj() @ z
            coef = np.zeros(j + 2, complex)
            coef[:j + 1] = (g - c) * inv
            coef[j + 1] = np.vdot(V[j + 1], V[j + 1]).real
            H[:j + 1, j] = coef[:j + 1]
            H[j, j] += sigma
        yy = coef[j + 1].real
        lag[:j + 1] = coef[:j + 1]
        beta2 = yy - np.sum(np.abs(coef[:j + 1]) ** 2)
        if not beta2 >= eta * yy:  # two explicit classical passes
            flagged += 1
            V[j + 1] = _f32(V[j + 1] - coef[:j + 1] @ V[:j + 1])
            c2 = V[:j + 1].conj() @ V[j + 1]
            H[:j + 1, j] += c2
            V[j + 1] = _f32(V[j + 1] - c2 @ V[:j + 1])
            beta2 = np.vdot(V[j + 1], V[j + 1]).real
            lag[:j + 1] = 0
        H[j + 1, j] = math.sqrt(max(beta2, 0.0))
        Hu[:j + 2, j] = H[:j + 2, j]
        Hu[j, j] -= sigma
        inv = 1.0 / H[j + 1, j]
    V[m] = _f32((V[m] - lag[:m] @ V[:m]) * inv)  # the last pending vector, for the check
    return V, H, flagged


def _classical(A, b, m):
    n = b.size
    V = np.zeros((m + 1, n), complex)
    H = np.zeros((m + 1, m), complex)
    V[0] = _f32(b / np.linalg.norm(b))
    for j in range(m):
        w = _f32(A(V[j]))
        for _ in range(2):
            h = V[:j + 1].conj() @ w
            H[:j + 1, j] += h
            w = _f32(w - h @ V[:j + 1])
        H[j + 1, j] = np.linalg.norm(w)
        V[j + 1] = _f32(w / H[j + 1, j])
    return V, H


def _relation_and_orthogonality(A, V, H):
    m = H.shape[1]
    AV = np.stack([A(V[i]) for i in range(m)])
    rel = np.linalg.norm(AV - H.T @ V) / np.linalg.norm(AV)
    orth = np.abs(V.conj() @ V.T - np.eye(m + 1)).max()
    return rel, orth


def test_shifted_one_sweep_recurrence_keeps_the_arnoldi_relation():
    A, n = _operator()
    rng = np.random.default_rng(11)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    m = 56
    Vc, Hc = _classical(A, b, m)
    rel_c, orth_c = _relation_and_orthogonality(A, Vc, Hc)
    V1, H1, flagged = _one_sweep(A, b, m, sigma=1.0)
    rel_1, orth_1 = _relation_and_orthogonality(A, V1, H1)
    assert rel_c < 1e-6 and orth_c < 1e-5
    assert rel_1 < 2e-6 and orth_1 < 1e-4, (rel_1, orth_1)
    # same Krylov space, same Hessenberg (up to the FP32 rounding of the basis)
    assert np.abs(H1 - Hc).max() <= 1e-4 * np.abs(Hc).max()
    # unshifted, the same recurrence loses the basis (orthogonality O(1) after 56 steps)
    V0, H0, _ = _one_sweep(A, b, m, sigma=0.0, eta=0.0)
    _, orth_0 = _relation_and_orthogonality(A, V0, H0)
    assert orth_0 > 0.1 and orth_0 > 1e4 * orth_1, (orth_0, orth_1)
