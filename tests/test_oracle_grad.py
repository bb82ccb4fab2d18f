"""Pins of the FP64 gradient reference (oracle/grad_oracle.py) and of the
adjoint's closed forms, on the CPU.

The reference is checked against central finite differences of the numpy
oracle (independent code), against dlog det A/dA = A^{-T}, and against the
Pfaffian gradient of App. A.3 (Eq. pf_grad) evaluated with the Householder
Pfaffian.  The closed forms the GPU adjoint implements are then checked
against the reference.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import grad_oracle as GO  # noqa: E402
from oracle import lru_oracle as O  # noqa: E402


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def mat(g, shape, cplx):
    x = g.standard_normal(shape)
    return x + 1j * g.standard_normal(shape) if cplx else x


def logr_np(A, U, V):
    r = O.det_ratio_direct(A, U, V)
    return np.log(r) if np.iscomplexobj(r) else math.log(abs(r))


@pytest.mark.parametrize("cplx", [False, True])
def test_det_reference_matches_finite_differences(cplx):
    g = rng(1)
    n, k, h = 6, 2, 1e-6
    A = mat(g, (n, n), cplx) + 3 * np.eye(n)
    U, V = mat(g, (n, k), cplx) * 0.5, mat(g, (k, n), cplx) * 0.5
    gA, gU, gV = GO.vjp(GO.det_log_ratio, [torch.tensor(A), torch.tensor(U), torch.tensor(V)], 1.0)
    for X, G, which in ((A, gA, 0), (U, gU, 1), (V, gV, 2)):
        D = mat(g, X.shape, cplx)
        args = [A, U, V]
        args[which] = X + h * D
        fp = logr_np(*args)
        args[which] = X - h * D
        fm = logr_np(*args)
        fd = (fp - fm) / (2 * h)
        # torch returns conj(df/dx) for holomorphic f: the directional derivative is sum(conj(G) * D)
        an = np.sum(np.conj(G.numpy()) * D)
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (which, fd, an)


def test_logdet_closed_form():
    g = rng(2)
    for cplx in (False, True):
        A = mat(g, (7, 7), cplx)
        (gA,) = GO.vjp(GO.log_det, [torch.tensor(A)], 1.0)
        assert np.allclose(np.conj(gA.numpy()), O.inv(A).T, atol=1e-12)


def test_pf_gradient_formula_of_appendix():
    # App. A.3, Eq. pf_grad: d pf(A')/d A_ij = (1/2) pf(A') (A'^{-1})_ji, A' = (A - A^T)/2,
    # checked by finite differences of the Householder Pfaffian and against the reference
    g = rng(3)
    n, h = 8, 1e-6
    A = g.standard_normal((n, n))
    As = (A - A.T) / 2
    pfA = O.pf(As)
    formula = 0.5 * pfA * O.inv(As).T
    for (i, j) in [(0, 1), (2, 5), (6, 3), (4, 4)]:
        E = np.zeros((n, n)); E[i, j] = 1.0
        fd = (O.pf((A + h * E - (A + h * E).T) / 2) - O.pf((A - h * E - (A - h * E).T) / 2)) / (2 * h)
        assert abs(fd - formula[i, j]) <= 1e-6 * max(1.0, abs(pfA)), (i, j)
    (gA,) = GO.vjp(GO.log_pf, [torch.tensor(A)], 1.0)
    assert np.allclose(gA.numpy() * pfA, formula, atol=1e-10)


@pytest.mark.parametrize("cplx", [False, True])
def test_pf_reference_matches_finite_differences(cplx):
    g = rng(4)
    n, k, h = 8, 1, 1e-6
    A = mat(g, (n, n), cplx)
    B = mat(g, (n, 2 * k), cplx) * 0.4
    C = mat(g, (2 * k, 2 * k), cplx)

    def f(A_, B_, C_):
        As, Cs = O.skew_part(A_), O.skew_part(C_)
        r = O.pf_ratio_direct(As, B_, Cs)
        return np.log(r) if np.iscomplexobj(r) else math.log(abs(r))

    gA, gB, gC = GO.vjp(GO.pf_log_ratio, [torch.tensor(A), torch.tensor(B), torch.tensor(C)], 1.0)
    for X, G, which in ((A, gA, 0), (B, gB, 1), (C, gC, 2)):
        D = mat(g, X.shape, cplx)
        args = [A, B, C]
        args[which] = X + h * D
        fp = f(*args)
        args[which] = X - h * D
        fm = f(*args)
        an = np.sum(np.conj(G.numpy()) * D)
        assert abs((fp - fm) / (2 * h) - an) <= 1e-6 * max(1.0, abs(an)), which


@pytest.mark.parametrize("cplx", [False, True])
def test_det_adjoint_closed_forms(cplx):
    # the forms of the GPU adjoint: dU = (R^{-1} Y)^T, dV = (X R^{-1})^T, dA = -(X R^{-1} Y)^T
    g = rng(5)
    n, k = 9, 3
    A = mat(g, (n, n), cplx) + 3 * np.eye(n)
    U, V = mat(g, (n, k), cplx) * 0.4, mat(g, (k, n), cplx) * 0.4
    Ai = O.inv(A)
    X, Y = Ai @ U, V @ Ai
    Ri = O.inv(np.eye(k) + V @ X)
    gA, gU, gV = (x.numpy() for x in GO.vjp(GO.det_log_ratio, [torch.tensor(A), torch.tensor(U), torch.tensor(V)], 1.0))
    assert np.allclose(np.conj(gU), (Ri @ Y).T, atol=1e-12)
    assert np.allclose(np.conj(gV), (X @ Ri).T, atol=1e-12)
    assert np.allclose(np.conj(gA), -(X @ Ri @ Y).T, atol=1e-12)


@pytest.mark.parametrize("cplx", [False, True])
def test_pf_adjoint_closed_forms(cplx):
    # gB = X M^{-1}, gA_ij = (X M^{-1} X^T)_ji / 2, gC = skew part of -[C^{-1}(M^{-1} - C)C^{-1}]^T / 2
    g = rng(6)
    n, k = 10, 2
    A = O.skew_part(mat(g, (n, n), cplx))
    B = mat(g, (n, 2 * k), cplx) * 0.4
    C = O.skew_part(mat(g, (2 * k, 2 * k), cplx))
    Ai, Ci = O.inv(A), O.inv(C)
    X = Ai @ B
    M = Ci + B.T @ Ai @ B
    Mi = O.inv(M)
    gA, gB, gC = (x.numpy() for x in GO.vjp(GO.pf_log_ratio, [torch.tensor(A), torch.tensor(B), torch.tensor(C)], 1.0))
    assert np.allclose(np.conj(gB), X @ Mi, atol=1e-11)
    assert np.allclose(np.conj(gA), 0.5 * (X @ Mi @ X.T).T, atol=1e-11)
    G = -0.5 * (Ci @ (Mi - C) @ Ci).T
    assert np.allclose(np.conj(gC), (G - G.T) / 2, atol=1e-11)
