"""Plain, slow CPU oracle for low-rank updates (LRU) of determinants and Pfaffians.

TEST INFRASTRUCTURE ONLY.  This module exists to check the CUDA path.  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import it.  The product path (``paper_2602_05255_gb300``) never
imports it and shares no code with it.

Everything here runs in float64 / complex128 with numpy.  Each function follows
one passage of the paper (arXiv 2602.05255, "lrux: Fast low-rank updates of
determinants and Pfaffians in JAX") and says which.  The notation bridge used
throughout:

* Determinant update (Sec. 2.1): the paper writes ``A_t = A_{t-1} + v u^T``
  with ``u, v`` of shape n x k.  Here ``A' = A + U V`` with ``U`` (n x k) the
  paper's ``v`` and ``V`` (k x n) the paper's ``u^T``.  The core is
  ``R = I_k + V A^{-1} U`` (Eq. det_R) and the ratio is ``det R`` (Eq. det_ratio).
* Pfaffian update (Sec. 3.1): the paper writes ``A_t = A_{t-1} - u J u^T``.
  Here ``A' = A + B C B^T`` with ``B`` (n x 2k) the paper's ``u`` and
  ``C = -J``; the general identity is the low-rank lemma of App. A.2 (Eq.
  pf_low_rank), ``pf(A + B C B^T)/pf(A) = pf(C^{-1} + B^T A^{-1} B)/pf(C^{-1})``.

All transposes are plain transposes, also for complex numbers: the Pfaffian is
defined for complex skew-symmetric (not skew-Hermitian) matrices (App. A.1).

Functions whose result has a plain definition (det, inverse, ratio, Pfaffian)
are that definition written out; the LRU chains (plain and delayed) follow the
paper's equations in the paper's order.  Parity pins live in ``tests/``:
brute-force Leibniz determinants and pairing-sum Pfaffians, the worked
examples of App. A.1, the identities of App. A.2, exact integer Sherman-Morrison
cases and from-scratch recomputation.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "lu_factor", "slogdet", "det", "inv", "det_leibniz",
    "pf_pairings", "slogpf", "pf", "skew_part", "skew_eye",
    "onehot_matrix", "det_ratio_direct", "pf_ratio_direct",
    "det_lru", "DetCarrier", "init_det_carrier", "det_lru_delayed",
    "pf_lru", "PfCarrier", "init_pf_carrier", "pf_lru_delayed",
    "carrier_inverse", "det_row_move", "pf_row_col_move", "pf_two_particle_move",
    "slater_matrix", "pairing_matrix",
]


def _ftype(*arrays):
    """float64 or complex128, whichever holds every input."""
    return np.result_type(np.float64, *[np.asarray(a).dtype for a in arrays])


# ---------------------------------------------------------------------------
# Dense determinant and inverse (the paper's from-scratch reference values,
# jnp.linalg.det / jnp.linalg.inv in the listings of Sec. 2.1)
# ---------------------------------------------------------------------------

def lu_factor(A):
    """LU factorisation with partial (row) pivoting, P A = L U.

    Textbook Gaussian elimination (Golub & Van Loan, Alg. 3.4.1): at column k
    the entry of largest modulus on or below the diagonal becomes the pivot.
    Returns ``(LU, perm, nswaps, singular)``; L has a unit diagonal and is
    stored below the diagonal of ``LU``; ``perm[i]`` is the original row now
    at row i.
    """
    LU = np.array(A, dtype=_ftype(A), copy=True)
    n = LU.shape[0]
    perm = np.arange(n)
    nswaps = 0
    singular = False
    for k in range(n):
        p = k + int(np.argmax(np.abs(LU[k:, k])))
        if p != k:
            LU[[k, p]] = LU[[p, k]]
            perm[[k, p]] = perm[[p, k]]
            nswaps += 1
        piv = LU[k, k]
        if piv == 0:
            singular = True
            continue
        LU[k + 1:, k] /= piv
        LU[k + 1:, k + 1:] -= np.outer(LU[k + 1:, k], LU[k, k + 1:])
    return LU, perm, nswaps, singular


def slogdet(A):
    """(sign or unit phase, log|det A|) from the LU factors.

    det A = (-1)^{swaps} * prod_k U_kk.  For complex A the first value is the
    phase det/|det|.  A singular matrix gives (0, -inf).
    """
    A = np.asarray(A)
    if A.shape[0] == 0:
        return np.asarray(1.0, dtype=_ftype(A))[()], 0.0
    LU, _, nswaps, singular = lu_factor(A)
    d = np.diag(LU)
    if singular or np.any(d == 0):
        return np.zeros((), dtype=LU.dtype)[()], -math.inf
    logabs = float(np.sum(np.log(np.abs(d))))
    sign = (-1.0) ** nswaps * np.prod(d / np.abs(d))
    return sign, logabs


def det(A):
    """det A = sign * exp(logabs)."""
    s, l = slogdet(A)
    return s * math.exp(l) if l != -math.inf else s * 0.0


def inv(A):
    """A^{-1} by forward and back substitution on the LU factors (P A = L U)."""
    LU, perm, _, singular = lu_factor(A)
    if singular:
        raise np.linalg.LinAlgError("singular matrix")
    n = LU.shape[0]
    X = np.eye(n, dtype=LU.dtype)[perm]          # right-hand side P I
    for i in range(n):                            # L y = P I
        X[i] -= LU[i, :i] @ X[:i]
    for i in range(n - 1, -1, -1):                # U x = y
        X[i] = (X[i] - LU[i, i + 1:] @ X[i + 1:]) / LU[i, i]
    return X


def det_leibniz(A):
    """Brute-force determinant: sum over all permutations (Leibniz formula).

    For n <= 7 only (5040 terms).  Parity is counted by inversions.
    """
    A = np.asarray(A)
    n = A.shape[0]
    total = 0
    for p in itertools.permutations(range(n)):
        inversions = sum(1 for a in range(n) for b in range(a + 1, n) if p[a] > p[b])
        term = (-1) ** inversions
        for i in range(n):
            term = term * A[i, p[i]]
        total = total + term
    return total


# ---------------------------------------------------------------------------
# Pfaffian (App. A.1)
# ---------------------------------------------------------------------------

def _pairings(elems):
    """All partitions of ``elems`` (sorted) into pairs (i, j) with i < j, the
    pairs ordered by their first element (App. A.1, Eq. pf_def)."""
    if not elems:
        yield []
        return
    first = elems[0]
    for idx in range(1, len(elems)):
        partner = elems[idx]
        rest = elems[1:idx] + elems[idx + 1:]
        for tail in _pairings(rest):
            yield [(first, partner)] + tail


def pf_pairings(A):
    """Brute-force Pfaffian, Eq. pf_def of App. A.1, written out.

    pf A = sum over pairings alpha of sign(alpha) prod A[i_k, j_k], where
    sign(alpha) is the parity of the permutation (i_1, j_1, ..., i_m, j_m).
    (2m-1)!! terms: use for 2m <= 10.
    """
    A = np.asarray(A)
    n = A.shape[0]
    if n % 2:
        return 0.0
    total = 0
    for alpha in _pairings(list(range(n))):
        seq = [x for pair in alpha for x in pair]
        inversions = sum(1 for a in range(n) for b in range(a + 1, n) if seq[a] > seq[b])
        term = (-1) ** inversions
        for (i, j) in alpha:
            term = term * A[i, j]
        total = total + term
    return total


def slogpf(A):
    """(sign or unit phase, log|pf A|) by Householder tridiagonalisation.

    Published method: skew-symmetric Householder reduction (M. Wimmer, ACM
    TOMS 38, 30 (2012)), written here from its mathematics.  Step k maps the
    column x = A[k+1:, k] onto alpha e_1 with the unitary reflection
    H = I - 2 v v^H / (v^H v), v = x - alpha e_1, alpha = -e^{i arg x_0} |x|.
    The congruence A <- Q A Q^T with Q = diag(I_{k+1}, H) keeps A
    skew-symmetric and, by App. A.2 (Eq. pf->det_pf), multiplies the Pfaffian
    by det Q = det H = -1.  The tridiagonal result T has
    pf T = T_01 T_23 ... T_{n-2,n-1}.
    """
    A = np.array(A, dtype=_ftype(A), copy=True)
    n = A.shape[0]
    if n == 0:
        return np.asarray(1.0, dtype=A.dtype)[()], 0.0
    if n % 2:
        return np.zeros((), dtype=A.dtype)[()], -math.inf
    flips = 0
    for k in range(n - 2):
        x = A[k + 1:, k].copy()
        if np.linalg.norm(x[1:]) == 0:
            continue                              # already reduced: H = I
        xnorm = np.linalg.norm(x)
        phase = x[0] / abs(x[0]) if x[0] != 0 else 1.0
        alpha = -phase * xnorm
        v = x.copy()
        v[0] -= alpha
        vv = np.vdot(v, v).real
        # rows k+1.. : A <- H A ;  columns k+1.. : A <- A H^T
        A[k + 1:, :] -= (2.0 / vv) * np.outer(v, v.conj() @ A[k + 1:, :])
        A[:, k + 1:] -= (2.0 / vv) * np.outer(A[:, k + 1:] @ v.conj(), v)
        flips += 1
    t = np.array([A[2 * i, 2 * i + 1] for i in range(n // 2)])
    if np.any(t == 0):
        return np.zeros((), dtype=A.dtype)[()], -math.inf
    logabs = float(np.sum(np.log(np.abs(t))))
    sign = (-1.0) ** flips * np.prod(t / np.abs(t))
    return sign, logabs


def pf(A):
    """Pfaffian value sign * exp(logabs)."""
    s, l = slogpf(A)
    return s * math.exp(l) if l != -math.inf else s * 0.0


def skew_part(M):
    """(M - M^T)/2: the skew-symmetric part.

    The inverse of a skew-symmetric matrix is skew-symmetric, and the Pfaffian
    updates of Sec. 3 rely on it ((A^{-1})^T = -A^{-1} in Eq. pf_inv).  In
    floating point the update of Eq. pf_inv does not keep the stored inverse
    skew, and the symmetric part of its rounding error grows by a factor 2-3
    per step; restoring the skew part after every update (the projection App.
    A.3 applies to A before differentiating) keeps the chain at rounding level.
    """
    M = np.asarray(M)
    return (M - M.T) / 2


def skew_eye(k, dtype=np.float64):
    """J = [[0, I_k], [-I_k, 0]], the 2k x 2k skew identity of Sec. 3.1."""
    J = np.zeros((2 * k, 2 * k), dtype=dtype)
    J[:k, k:] = np.eye(k)
    J[k:, :k] = -np.eye(k)
    return J


# ---------------------------------------------------------------------------
# Operands (Sec. 2.2 and 3.2)
# ---------------------------------------------------------------------------

def onehot_matrix(n, idx, dtype=np.float64):
    """n x k matrix whose column a is e_{idx[a]} (the one-hot form, Sec. 2.2)."""
    idx = np.atleast_1d(np.asarray(idx))
    M = np.zeros((n, len(idx)), dtype=dtype)
    M[idx, np.arange(len(idx))] = 1
    return M


def det_ratio_direct(A, U, V):
    """Definition of the determinant ratio: det(A + U V) / det(A) (Eq. det_ratio)."""
    s1, l1 = slogdet(np.asarray(A) + np.asarray(U) @ np.asarray(V))
    s0, l0 = slogdet(A)
    return s1 / s0 * math.exp(l1 - l0) if l1 != -math.inf else 0.0 * s1


def pf_ratio_direct(A, B, C):
    """Definition of the Pfaffian ratio: pf(A + B C B^T) / pf(A)."""
    B = np.asarray(B)
    s1, l1 = slogpf(np.asarray(A) + B @ np.asarray(C) @ B.T)
    s0, l0 = slogpf(A)
    return s1 / s0 * math.exp(l1 - l0) if l1 != -math.inf else 0.0 * s1


# ---------------------------------------------------------------------------
# Plain determinant LRU (Sec. 2.1)
# ---------------------------------------------------------------------------

def det_lru(Ainv, U, V, return_update=False):
    """One determinant low-rank update.

    R = I_k + V A^{-1} U (Eq. det_R), r = det R (Eq. det_ratio) and, if asked,
    A'^{-1} = A^{-1} - (A^{-1} U) R^{-1} (V A^{-1}) (Sherman-Morrison-Woodbury,
    Eq. det_inv).  Returns ``r`` or ``(r, A'^{-1})``.
    """
    Ainv = np.asarray(Ainv)
    U = np.asarray(U)
    V = np.asarray(V)
    k = U.shape[1]
    R = np.eye(k, dtype=_ftype(Ainv, U, V)) + V @ Ainv @ U
    r = det(R)
    if not return_update:
        return r
    new = Ainv - (Ainv @ U) @ inv(R) @ (V @ Ainv)
    return r, new


# ---------------------------------------------------------------------------
# Delayed determinant LRU (Sec. 2.3)
# ---------------------------------------------------------------------------

@dataclass
class DetCarrier:
    """State of the delayed determinant update: A_0^{-1}, the stored a_t, b_t
    (t = 1..tau) and the delay bound T (Sec. 2.3)."""
    A0inv: np.ndarray
    max_delay: int
    a: list = field(default_factory=list)
    b: list = field(default_factory=list)

    @property
    def tau(self):
        return len(self.a)


def init_det_carrier(A, max_delay):
    """Carrier from a matrix: A_0^{-1} from scratch, no stored corrections."""
    return DetCarrier(inv(A), int(max_delay))


def carrier_inverse(carrier):
    """A_tau^{-1} rebuilt from the carrier (Eq. delayed_Ainv for the
    determinant, Eq. pf_delayed_Ainv for the Pfaffian)."""
    M = carrier.A0inv.copy()
    if isinstance(carrier, DetCarrier):
        for a, b in zip(carrier.a, carrier.b):
            M = M - a @ b.T
    else:
        for a, Rinv in zip(carrier.a, carrier.Rinv):
            M = M + a @ Rinv @ a.T
    return M


def det_lru_delayed(carrier, U, V, accept=True):
    """One delayed determinant update (Sec. 2.3).

    With tau the number of stored corrections before this step:
      R_tau = I + V A_0^{-1} U - sum_t (V a_t)(b_t^T U)         (R_tau equation)
      a_tau = A_0^{-1} U - sum_t a_t (b_t^T U)                   (a_tau equation)
      b_tau = [A_0^{-T} V^T - sum_t b_t (a_t^T V^T)] R_tau^{-T}  (b_tau equation)
    r = det R_tau.  On acceptance a_tau, b_tau are stored; when the store holds
    T = max_delay corrections, A_0^{-1} <- A_0^{-1} - sum_t a_t b_t^T
    (Eq. delayed_Ainv) and the store is emptied.  A rejected proposal leaves the
    carrier unchanged.  Returns r.
    """
    U = np.asarray(U)
    V = np.asarray(V)
    A0 = carrier.A0inv
    k = U.shape[1]
    R = np.eye(k, dtype=_ftype(A0, U, V)) + V @ A0 @ U
    for a_t, b_t in zip(carrier.a, carrier.b):
        R = R - (V @ a_t) @ (b_t.T @ U)
    r = det(R)
    if not accept:
        return r
    a_new = A0 @ U
    for a_t, b_t in zip(carrier.a, carrier.b):
        a_new = a_new - a_t @ (b_t.T @ U)
    b_new = A0.T @ V.T
    for a_t, b_t in zip(carrier.a, carrier.b):
        b_new = b_new - b_t @ (a_t.T @ V.T)
    b_new = b_new @ inv(R).T
    carrier.a.append(a_new)
    carrier.b.append(b_new)
    if carrier.tau == carrier.max_delay:
        carrier.A0inv = carrier_inverse(carrier)
        carrier.a.clear()
        carrier.b.clear()
    return r


# ---------------------------------------------------------------------------
# Plain Pfaffian LRU (Sec. 3.1, App. A.2)
# ---------------------------------------------------------------------------

def pf_lru(Ainv, B, C=None, return_update=False):
    """One Pfaffian low-rank update A' = A + B C B^T.

    M = C^{-1} + B^T A^{-1} B and r = pf M / pf(C^{-1}) (low-rank lemma, Eq.
    pf_low_rank; with C = -J this is Eqs. pf_ratio and pf_R, where C^{-1} = J
    and pf J = (-1)^{k(k-1)/2}).  The inverse follows Woodbury with
    (A^{-1})^T = -A^{-1}:  A'^{-1} = A^{-1} + X M^{-1} X^T, X = A^{-1} B
    (Eq. pf_inv).  ``C=None`` means C = -J.
    """
    Ainv = np.asarray(Ainv)
    B = np.asarray(B)
    m = B.shape[1]
    if m % 2:
        raise ValueError("B must have an even number of columns")
    if C is None:
        C = -skew_eye(m // 2)
    Cinv = skew_part(inv(C))
    M = skew_part(Cinv + B.T @ Ainv @ B)
    r = pf(M) / pf(Cinv)
    if not return_update:
        return r
    X = Ainv @ B
    return r, skew_part(Ainv + X @ skew_part(inv(M)) @ X.T)


@dataclass
class PfCarrier:
    """State of the delayed Pfaffian update: A_0^{-1}, the stored a_t and
    R_t^{-1} (Sec. 3.3)."""
    A0inv: np.ndarray
    max_delay: int
    a: list = field(default_factory=list)
    Rinv: list = field(default_factory=list)

    @property
    def tau(self):
        return len(self.a)


def init_pf_carrier(A, max_delay):
    return PfCarrier(skew_part(inv(A)), int(max_delay))


def pf_lru_delayed(carrier, B, C=None, accept=True):
    """One delayed Pfaffian update (Sec. 3.3), for a general skew C.

      R_tau = C^{-1} + B^T A_0^{-1} B + sum_t (B^T a_t) R_t^{-1} (B^T a_t)^T
      a_tau = A_0^{-1} B + sum_t a_t R_t^{-1} (B^T a_t)^T
    (the printed a_tau equation has u_t where u_tau is meant; this follows the
    derivation from Eqs. pf_a and pf_delayed_Ainv).  r = pf R_tau / pf(C^{-1}).
    On acceptance a_tau and R_tau^{-1} are stored and, once T are stored,
    A_0^{-1} <- A_0^{-1} + sum_t a_t R_t^{-1} a_t^T (Eq. pf_delayed_Ainv).
    """
    B = np.asarray(B)
    m = B.shape[1]
    if C is None:
        C = -skew_eye(m // 2)
    Cinv = skew_part(inv(C))
    A0 = carrier.A0inv
    R = Cinv + B.T @ A0 @ B
    for a_t, Ri in zip(carrier.a, carrier.Rinv):
        BtA = B.T @ a_t
        R = R + BtA @ Ri @ BtA.T
    R = skew_part(R)
    r = pf(R) / pf(Cinv)
    if not accept:
        return r
    a_new = A0 @ B
    for a_t, Ri in zip(carrier.a, carrier.Rinv):
        a_new = a_new + a_t @ Ri @ (B.T @ a_t).T
    carrier.a.append(a_new)
    carrier.Rinv.append(skew_part(inv(R)))
    if carrier.tau == carrier.max_delay:
        carrier.A0inv = skew_part(carrier_inverse(carrier))
        carrier.a.clear()
        carrier.Rinv.clear()
    return r


# ---------------------------------------------------------------------------
# Operand formation for the QMC moves of Sec. 2.2 / 3.2
# ---------------------------------------------------------------------------

def slater_matrix(Phi, occ):
    """Slater matrix A = Phi[occ] (row i holds the orbital row occupied by
    particle i)."""
    return np.asarray(Phi)[np.asarray(occ)]


def det_row_move(Phi, occ, i, new_row):
    """Rank-1 row replacement (Sec. 2.2, Eq. det_rank1_row): particle slot i
    moves from orbital row occ[i] to ``new_row``.  A' - A = e_i (Phi[new] -
    Phi[occ_i]), so U = e_i (one-hot) and V = Phi[new] - Phi[occ_i]."""
    Phi = np.asarray(Phi)
    n = len(occ)
    U = onehot_matrix(n, [i], dtype=Phi.dtype)
    V = (Phi[new_row] - Phi[occ[i]])[None, :]
    return U, V


def pairing_matrix(F, pos):
    """Pfaffian matrix A_ij = F(r_i, r_j) from a skew pairing matrix F."""
    pos = np.asarray(pos)
    return np.asarray(F)[np.ix_(pos, pos)]


def pf_row_col_move(F, pos, i, new_site):
    """Row-and-column replacement (Sec. 3.2, Eq. pf_rank2): particle i moves
    from site pos[i] to ``new_site``.  x_j = F(r', r_j) - F(r_i, r_j); the
    update is A' - A = e_i x^T - x e_i^T = B C B^T with B = [x, e_i] and
    C = -J (the i-th entry of x cancels on the diagonal)."""
    F = np.asarray(F)
    pos = np.asarray(pos)
    x = F[new_site, pos] - F[pos[i], pos]
    n = len(pos)
    B = np.zeros((n, 2), dtype=F.dtype)
    B[:, 0] = x
    B[i, 1] = 1
    return B, -skew_eye(1, dtype=F.dtype)


def pf_two_particle_move(F, pos, p, q, new_p, new_q):
    """Two particles moved at once: rows and columns p and q replaced (Sec.
    3.2, the update of 2 rows and 2 columns, A' - A = -u J u^T with
    u = [x, y, e_p, e_q]).  Entry (p, q) of the change is x_q - y_p, so
    x_j = F(r'_p, r'_j) - F(r_p, r_j) with the new sites of both particles
    (x_p = 0), y_j = F(r'_q, r_j) - F(r_q, r_j) at the old sites, y_p = 0
    (its diagonal entry y_q cancels).  Returns (B, C) with B = [x, y, e_p,
    e_q] and C = -J (2 x 2 blocks)."""
    F = np.asarray(F)
    pos = np.asarray(pos)
    new_pos = pos.copy()
    new_pos[p] = new_p
    new_pos[q] = new_q
    x = F[new_p, new_pos] - F[pos[p], pos]
    y = F[new_q, pos] - F[pos[q], pos]
    y[p] = 0
    n = len(pos)
    B = np.zeros((n, 4), dtype=F.dtype)
    B[:, 0] = x
    B[:, 1] = y
    B[p, 2] = 1
    B[q, 3] = 1
    return B, -skew_eye(2, dtype=F.dtype)
