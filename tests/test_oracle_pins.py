"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: brute-force
sums, worked examples printed in the paper, identities of App. A.2, exact
integer arithmetic, or an independent library routine.  A dropped term, a
wrong sign or a transposed operand in the oracle fails at least one of them.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

from oracle import lru_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def rand_mat(g, n, cplx=False):
    A = g.standard_normal((n, n))
    if cplx:
        A = A + 1j * g.standard_normal((n, n))
    return A


def rand_skew(g, n, cplx=False):
    A = rand_mat(g, n, cplx)
    return A - A.T


# --------------------------------------------------------------------------
# determinant / inverse
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 5, 6])
@pytest.mark.parametrize("cplx", [False, True])
def test_det_matches_leibniz(n, cplx):
    g = rng(100 + n)
    A = rand_mat(g, n, cplx)
    assert np.isclose(O.det(A), O.det_leibniz(A), rtol=1e-12, atol=1e-12)


def test_det_needs_pivoting():
    # zero leading entry: elimination without row exchange would divide by 0
    A = np.array([[0.0, 2.0, 1.0], [3.0, 1.0, 0.0], [1.0, 1.0, 1.0]])
    assert O.det(A) == pytest.approx(O.det_leibniz(A), abs=1e-14)
    assert O.det(A) == pytest.approx(-4.0, abs=1e-14)  # cofactor expansion: 0 - 2*3 + 1*2


def test_slogdet_matches_numpy_and_singular():
    g = rng(7)
    for cplx in (False, True):
        A = rand_mat(g, 40, cplx)
        s, l = O.slogdet(A)
        s2, l2 = np.linalg.slogdet(A)
        assert l == pytest.approx(l2, rel=1e-12)
        assert abs(s - s2) < 1e-12
    S = np.ones((4, 4))
    assert O.slogdet(S) == (0.0, -math.inf)


def test_inverse_exact_on_unimodular_integers():
    # product of unit triangular integer matrices: det = 1, inverse integral
    g = rng(3)
    n = 6
    L = np.tril(g.integers(-2, 3, (n, n)), -1) + np.eye(n)
    U = np.triu(g.integers(-2, 3, (n, n)), 1) + np.eye(n)
    P = np.eye(n)[g.permutation(n)]
    A = P @ L @ U
    X = O.inv(A)
    # the exact inverse is integral; pivots other than +-1 may round in between
    assert np.allclose(X, np.round(X), rtol=0, atol=1e-11)
    assert np.array_equal(A @ np.round(X), np.eye(n))
    assert abs(O.det(A)) == pytest.approx(1.0, abs=1e-12)


@pytest.mark.parametrize("cplx", [False, True])
def test_inverse_property(cplx):
    g = rng(11)
    A = rand_mat(g, 30, cplx)
    X = O.inv(A)
    assert np.allclose(A @ X, np.eye(30), atol=1e-11)
    assert np.allclose(X @ A, np.eye(30), atol=1e-11)


# --------------------------------------------------------------------------
# Pfaffian
# --------------------------------------------------------------------------

def test_pf_worked_examples():
    d = json.load(open(os.path.join(GOLDEN, "pf_worked_examples.json")))
    for case in d["cases"]:
        A = np.array(case["matrix"], dtype=float)
        assert O.pf(A) == pytest.approx(case["pf"], abs=1e-12), case["name"]
        assert O.pf_pairings(A) == case["pf"], case["name"]


@pytest.mark.parametrize("n", [2, 4, 6, 8])
@pytest.mark.parametrize("cplx", [False, True])
def test_pf_matches_pairing_sum(n, cplx):
    g = rng(200 + n)
    A = rand_skew(g, n, cplx)
    assert np.isclose(O.pf(A), O.pf_pairings(A), rtol=1e-11, atol=1e-12)


def test_pf_pairing_count_and_odd():
    assert sum(1 for _ in O._pairings(list(range(10)))) == 945   # (2m-1)!!
    assert O.pf_pairings(np.zeros((3, 3))) == 0.0
    assert O.slogpf(rand_skew(rng(1), 5))[1] == -math.inf


@pytest.mark.parametrize("cplx", [False, True])
def test_pf_squared_is_det(cplx):
    # App. A.2, Eq. pf2=det
    g = rng(31)
    for n in (10, 24):
        A = rand_skew(g, n, cplx)
        s, l = O.slogpf(A)
        sd, ld = O.slogdet(A)
        assert 2 * l == pytest.approx(ld, rel=1e-11)
        assert abs(s * s - sd) < 1e-10


@pytest.mark.parametrize("cplx", [False, True])
def test_pf_congruence(cplx):
    # App. A.2, Eq. pf->det_pf: pf(B A B^T) = det(B) pf(A)
    g = rng(41)
    A = rand_skew(g, 8, cplx)
    B = rand_mat(g, 8, cplx)
    assert np.isclose(O.pf(B @ A @ B.T), O.det(B) * O.pf(A), rtol=1e-10)


def test_pf_offdiagonal_and_skew_eye():
    # App. A.2, Eq. pf_offdiagonal: pf [[0, M], [-M^T, 0]] = (-1)^{m(m-1)/2} det M
    g = rng(51)
    for m in (1, 2, 3, 4, 5):
        M = rand_mat(g, m)
        Z = np.zeros((m, m))
        big = np.block([[Z, M], [-M.T, Z]])
        assert O.pf(big) == pytest.approx((-1) ** (m * (m - 1) // 2) * O.det(M), rel=1e-11)
        # Sec. 3.1: pf J = (-1)^{k(k-1)/2}
        assert O.pf(O.skew_eye(m)) == pytest.approx((-1) ** (m * (m - 1) // 2))
        assert O.pf_pairings(O.skew_eye(m)) == (-1) ** (m * (m - 1) // 2)
    J = O.skew_eye(3)
    assert np.array_equal(np.linalg.inv(J), -J)     # J^{-1} = -J (Sec. 3.1)


def test_pf_block_diagonal_and_block_schur():
    # App. A.2, Eqs. pf_diagonal and pf_block
    g = rng(61)
    A1, A2 = rand_skew(g, 4), rand_skew(g, 6)
    Z = np.zeros((4, 6))
    assert O.pf(np.block([[A1, Z], [Z.T, A2]])) == pytest.approx(O.pf(A1) * O.pf(A2), rel=1e-11)
    M, N, Q = rand_skew(g, 4), rand_skew(g, 6), rand_mat(g, 10)[:4, :6]
    big = np.block([[M, Q], [-Q.T, N]])
    lhs = O.pf(big)
    assert lhs == pytest.approx(O.pf(M) * O.pf(N + Q.T @ np.linalg.inv(M) @ Q), rel=1e-10)
    assert lhs == pytest.approx(O.pf(N) * O.pf(M + Q @ np.linalg.inv(N) @ Q.T), rel=1e-10)


@pytest.mark.parametrize("k", [1, 2])
def test_pf_low_rank_lemma_brute_force(k):
    # App. A.2, Eq. pf_low_rank, with every Pfaffian a pairing sum (n = 6)
    g = rng(71 + k)
    n = 6
    A = rand_skew(g, n)
    B = g.standard_normal((n, 2 * k))
    C = rand_skew(g, 2 * k)
    Cinv = np.linalg.inv(C)
    lhs = O.pf_pairings(A + B @ C @ B.T) / O.pf_pairings(A)
    rhs = O.pf_pairings(Cinv + B.T @ np.linalg.inv(A) @ B) / O.pf_pairings(Cinv)
    assert lhs == pytest.approx(rhs, rel=1e-10)
    assert O.pf_lru(np.linalg.inv(A), B, C) == pytest.approx(lhs, rel=1e-10)


# --------------------------------------------------------------------------
# operand forms (Sec. 2.2, 3.2)
# --------------------------------------------------------------------------

def test_printed_update_matrices():
    d = json.load(open(os.path.join(GOLDEN, "update_matrices.json")))
    for case in d["det"]:
        v = np.array(case["v"], float)     # paper v  (= U here)
        u = np.array(case["u"], float)     # paper u  (V = u^T here)
        assert np.array_equal(v @ u.T, np.array(case["A1_minus_A0"], float)), case["name"]
    for case in d["pf"]:
        u = np.array(case["u"], float)     # paper u  (= B here), C = -J
        k = u.shape[1] // 2
        C = -O.skew_eye(k)
        assert np.array_equal(u @ C @ u.T, np.array(case["A1_minus_A0"], float)), case["name"]


def test_det_row_move_is_row_replacement():
    g = rng(81)
    Phi = g.standard_normal((12, 5))
    occ = np.array([0, 3, 4, 7, 9])
    U, V = O.det_row_move(Phi, occ, 2, 11)
    occ2 = occ.copy()
    occ2[2] = 11
    assert np.allclose(O.slater_matrix(Phi, occ) + U @ V, O.slater_matrix(Phi, occ2), atol=0)


def test_pf_row_col_move_is_position_change():
    g = rng(82)
    G = g.standard_normal((16, 16))
    F = G - G.T
    pos = np.array([1, 4, 5, 8, 10, 13])
    B, C = O.pf_row_col_move(F, pos, 3, 15)
    pos2 = pos.copy()
    pos2[3] = 15
    A, A2 = O.pairing_matrix(F, pos), O.pairing_matrix(F, pos2)
    assert np.allclose(A + B @ C @ B.T, A2, atol=1e-15)


@pytest.mark.parametrize("cplx", [False, True])
def test_pf_two_particle_move_is_position_change(cplx):
    # two particles moved at once: the 2-rows-2-columns form of Sec. 3.2,
    # A' - A = -u J u^T with u = [x, y, e_p, e_q]; its (p, q) entry is x_q - y_p
    g = rng(83 + cplx)
    G = g.standard_normal((18, 18)) + (1j * g.standard_normal((18, 18)) if cplx else 0)
    F = G - G.T
    pos = np.array([1, 4, 5, 8, 10, 13, 16])
    p, q, new_p, new_q = 1, 4, 17, 2
    B, C = O.pf_two_particle_move(F, pos, p, q, new_p, new_q)
    pos2 = pos.copy()
    pos2[p], pos2[q] = new_p, new_q
    A, A2 = O.pairing_matrix(F, pos), O.pairing_matrix(F, pos2)
    assert np.allclose(A + B @ C @ B.T, A2, rtol=0, atol=1e-14)
    assert np.array_equal(C, -O.skew_eye(2))
    assert np.array_equal(B[:, 2], np.eye(len(pos))[p]) and np.array_equal(B[:, 3], np.eye(len(pos))[q])
    assert (A2 - A)[p, q] == pytest.approx(B[q, 0] - B[p, 1], abs=1e-14)


def test_pf_two_particle_ratio_brute_force():
    # pf(A') / pf(A) by the pairing sum (App. A.1) against the low-rank ratio of
    # the two-particle operands (App. A.2, k = 2)
    g = rng(85)
    G = g.standard_normal((14, 14))
    F = G - G.T
    pos = np.array([0, 2, 3, 6, 7, 9, 11, 12])
    B, C = O.pf_two_particle_move(F, pos, 2, 5, 13, 1)
    pos2 = pos.copy()
    pos2[2], pos2[5] = 13, 1
    A, A2 = O.pairing_matrix(F, pos), O.pairing_matrix(F, pos2)
    exact = O.pf_pairings(A2) / O.pf_pairings(A)
    r = O.pf_lru(O.skew_part(O.inv(A)), B, C)
    assert r == pytest.approx(exact, rel=1e-11)


# --------------------------------------------------------------------------
# plain LRU
# --------------------------------------------------------------------------

@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("k", [1, 3])
def test_det_lru_matches_direct_ratio(cplx, k):
    g = rng(91 + k)
    n = 9
    A = rand_mat(g, n, cplx)
    U = rand_mat(g, n, cplx)[:, :k]
    V = rand_mat(g, n, cplx)[:k, :]
    r, Ainv2 = O.det_lru(O.inv(A), U, V, return_update=True)
    assert r == pytest.approx(O.det_ratio_direct(A, U, V), rel=1e-11)
    assert np.allclose(Ainv2, O.inv(A + U @ V), rtol=1e-10, atol=1e-11)
    # ratio against brute force (Leibniz) on a 5x5 slice
    A5, U5, V5 = A[:5, :5], U[:5], V[:, :5]
    bf = O.det_leibniz(A5 + U5 @ V5) / O.det_leibniz(A5)
    assert O.det_lru(O.inv(A5), U5, V5) == pytest.approx(bf, rel=1e-10)


def test_sherman_morrison_exact_integers():
    # A unimodular integer matrix and an update chosen so R = 1 + V A^{-1} U = -1:
    # every quantity is an integer, so FP64 results must be exact.
    A = np.array([[2.0, 1.0, 0.0], [1.0, 1.0, 0.0], [0.0, 0.0, 1.0]])  # det 1
    Ainv = O.inv(A)
    assert np.array_equal(Ainv, np.array([[1, -1, 0], [-1, 2, 0], [0, 0, 1]], float))
    U = np.array([[0.0], [0.0], [1.0]])
    V = np.array([[0.0, 0.0, -2.0]])          # R = 1 + (-2)*1 = -1
    r, new = O.det_lru(Ainv, U, V, return_update=True)
    assert r == -1.0
    A2 = A + U @ V
    assert np.array_equal(new, O.inv(A2))
    assert np.array_equal(A2 @ new, np.eye(3))


def test_det_lru_two_step_chain():
    # analogue of the consecutive-update listing of Sec. 2.1 (n=4, two updates)
    g = rng(5)
    n = 4
    A = g.standard_normal((n, n))
    Ainv = O.inv(A)
    detA = O.det(A)
    u1, v1, u2, v2 = (g.standard_normal((n, 1)) for _ in range(4))
    r, Ainv = O.det_lru(Ainv, v1, u1.T, return_update=True)
    detA *= r
    r, Ainv = O.det_lru(Ainv, v2, u2.T, return_update=True)
    detA *= r
    exact = O.det_leibniz(A + v1 @ u1.T + v2 @ u2.T)
    assert detA == pytest.approx(exact, rel=1e-11)


@pytest.mark.parametrize("cplx", [False, True])
def test_pf_lru_k1_closed_form(cplx):
    # Sec. 3.1, k=1: A'^{-1} = A^{-1} + (1/r)(A^{-1}y)(A^{-1}x)^T - (1/r)(A^{-1}x)(A^{-1}y)^T
    g = rng(17)
    n = 8
    A = rand_skew(g, n, cplx)
    Ainv = O.inv(A)
    x = rand_mat(g, n, cplx)[:, 0]
    y = rand_mat(g, n, cplx)[:, 1]
    u = np.stack([x, y], axis=1)
    r, new = O.pf_lru(Ainv, u, None, return_update=True)
    # R = J + u^T A^{-1} u = [[0, r], [-r, 0]] with r = 1 + x^T A^{-1} y
    assert r == pytest.approx(1 + x @ Ainv @ y, rel=1e-12)
    Ax, Ay = Ainv @ x, Ainv @ y
    closed = Ainv + np.outer(Ay, Ax) / r - np.outer(Ax, Ay) / r
    assert np.allclose(new, closed, rtol=1e-11, atol=1e-12)
    J = O.skew_eye(1)
    assert np.allclose(new, O.inv(A - u @ J @ u.T), rtol=1e-9, atol=1e-10)
    assert r == pytest.approx(O.pf(A - u @ J @ u.T) / O.pf(A), rel=1e-10)


@pytest.mark.parametrize("cplx", [False, True])
def test_pf_lru_general_C_matches_direct(cplx):
    g = rng(23)
    n, k = 10, 2
    A = rand_skew(g, n, cplx)
    B = rand_mat(g, n, cplx)[:, :2 * k]
    C = rand_skew(g, 2 * k, cplx)
    r, new = O.pf_lru(O.inv(A), B, C, return_update=True)
    assert r == pytest.approx(O.pf_ratio_direct(A, B, C), rel=1e-10)
    assert np.allclose(new, O.inv(A + B @ C @ B.T), rtol=1e-9, atol=1e-10)
    # 2x2 check of pf(C^{-1}) = (-1)^k / pf(C): C = [[0,c],[-c,0]] -> -1/c
    c = 2.5
    C2 = np.array([[0, c], [-c, 0]])
    assert O.pf(np.linalg.inv(C2)) == pytest.approx(-1 / c)


def test_pf_lru_two_step_chain():
    # analogue of the consecutive Pfaffian listing of Sec. 3.1 (n=4, two updates)
    g = rng(29)
    n = 4
    A = g.standard_normal((n, n))
    A = (A - A.T) / 2
    Ainv = O.inv(A)
    pfA = O.pf(A)
    J = O.skew_eye(1)
    u1, u2 = g.standard_normal((n, 2)), g.standard_normal((n, 2))
    r, Ainv = O.pf_lru(Ainv, u1, None, return_update=True)
    pfA *= r
    r, Ainv = O.pf_lru(Ainv, u2, None, return_update=True)
    pfA *= r
    exact = O.pf_pairings(A - u1 @ J @ u1.T - u2 @ J @ u2.T)
    assert pfA == pytest.approx(exact, rel=1e-11)


# --------------------------------------------------------------------------
# delayed LRU
# --------------------------------------------------------------------------

@pytest.mark.parametrize("cplx", [False, True])
def test_det_delayed_listing_analogue(cplx):
    # Sec. 2.3 listing structure: n=10, T=4, 20 one-hot row updates, exact check each step
    g = rng(37)
    n, T = 10, 4
    A = rand_mat(g, n, cplx)
    carrier = O.init_det_carrier(A, T)
    Ainv_plain = O.inv(A)
    detA = O.det(A)
    for step in range(20):
        u = rand_mat(g, n, cplx)[0]
        row = int(g.integers(0, n))
        U = O.onehot_matrix(n, [row], dtype=A.dtype)
        V = u[None, :]
        r = O.det_lru_delayed(carrier, U, V)
        r_plain, Ainv_plain = O.det_lru(Ainv_plain, U, V, return_update=True)
        detA *= r
        A = A + U @ V
        assert r == pytest.approx(r_plain, rel=1e-10)
        assert detA == pytest.approx(O.det(A), rel=1e-9)
        assert carrier.tau == (step + 1) % T
        assert np.allclose(O.carrier_inverse(carrier), O.inv(A), rtol=1e-8, atol=1e-9)


def test_det_delayed_rank2_dense_and_reject():
    g = rng(43)
    n, T, k = 12, 3, 2
    A = rand_mat(g, n)
    carrier = O.init_det_carrier(A, T)
    for step in range(8):
        U = g.standard_normal((n, k)) * 0.3
        V = g.standard_normal((k, n)) * 0.3
        accept = step % 3 != 1
        r = O.det_lru_delayed(carrier, U, V, accept=accept)
        assert r == pytest.approx(O.det_ratio_direct(A, U, V), rel=1e-9)
        if accept:
            A = A + U @ V
        assert np.allclose(O.carrier_inverse(carrier), O.inv(A), rtol=1e-8, atol=1e-9)


@pytest.mark.parametrize("cplx", [False, True])
def test_pf_delayed_listing_analogue(cplx):
    # Sec. 3.3 listing structure: n=10, T=4, 20 row+column updates, exact check each step
    g = rng(47)
    n, T = 10, 4
    A = rand_mat(g, n, cplx)
    A = (A - A.T) / 2
    carrier = O.init_pf_carrier(A, T)
    pfA = O.pf(A)
    for step in range(20):
        x = rand_mat(g, n, cplx)[0]
        e = int(g.integers(0, n))
        B = np.zeros((n, 2), dtype=A.dtype)
        B[:, 0] = x
        B[e, 1] = 1
        r = O.pf_lru_delayed(carrier, B)          # C = -J
        pfA *= r
        A = A.copy()
        A[e, :] += x
        A[:, e] -= x
        assert pfA == pytest.approx(O.pf(A), rel=1e-9)
        assert carrier.tau == (step + 1) % T
        assert np.allclose(O.carrier_inverse(carrier), O.inv(A), rtol=1e-8, atol=1e-9)


def test_pf_delayed_general_C_k2():
    g = rng(53)
    n, T, k = 12, 3, 2
    A = rand_skew(g, n)
    carrier = O.init_pf_carrier(A, T)
    for step in range(7):
        B = g.standard_normal((n, 2 * k)) * 0.3
        C = rand_skew(g, 2 * k)
        r = O.pf_lru_delayed(carrier, B, C)
        assert r == pytest.approx(O.pf_ratio_direct(A, B, C), rel=1e-9)
        A = A + B @ C @ B.T
        assert np.allclose(O.carrier_inverse(carrier), O.inv(A), rtol=1e-8, atol=1e-9)


@pytest.mark.parametrize("delayed", [False, True])
def test_pf_chain_stays_accurate_over_many_steps(delayed):
    # 80 row+column moves on a pairing matrix: the tracked inverse and the
    # accumulated log|pf| must stay at rounding level against from-scratch values
    g = rng(59)
    m, n = 40, 16
    G = g.standard_normal((m, m)) / math.sqrt(n)
    F = G - G.T
    pos = g.permutation(m)[:n]
    A = O.pairing_matrix(F, pos)
    Ainv = O.skew_part(O.inv(A))
    carrier = O.init_pf_carrier(A, 5)
    s0, logpf = O.slogpf(A)
    for step in range(80):
        i = int(g.integers(0, n))
        free = np.setdiff1d(np.arange(m), pos)
        new = int(free[g.integers(0, len(free))])
        B, C = O.pf_row_col_move(F, pos, i, new)
        if delayed:
            r = O.pf_lru_delayed(carrier, B, C)
        else:
            r, Ainv = O.pf_lru(Ainv, B, C, return_update=True)
        logpf += math.log(abs(r))
        pos[i] = new
    A = O.pairing_matrix(F, pos)
    ref = O.inv(A)
    got = O.carrier_inverse(carrier) if delayed else Ainv
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-11
    assert logpf == pytest.approx(O.slogpf(A)[1], abs=1e-10)
