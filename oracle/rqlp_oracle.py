"""FP64 CPU oracle for Rand-QLP (arXiv 2110.01011).

TEST INFRASTRUCTURE ONLY. This module is the parity reference for the CUDA path;
only tests, the smoke check and the benchmark's CPU-baseline leg may import it.
The product path never calls it and shares no code with it.

Everything is plain numpy in float64. Matrix products use numpy's ``@`` (a
library GEMM, used as one step); the QR factorisation is Householder
orthogonal triangularisation written out below (section 2 names Gram-Schmidt
and Householder as the two ways to compute the unpivoted QR).

Notation follows the paper: A is m x n, Omega the Gaussian test matrix,
Qbar = orth(A^T Omega) (called P~ for the truncated chain), Q = orth(A Qbar),
and A ~= Q L P^T with L lower triangular.

Three modes:

* ``rand_qlp``: the truncated chain of this library. Omega has d = k + p
  columns, q power passes refine P~ = qf((A^T A)^q A^T Omega), the projection
  A P~ is factored Q R, and the QR of R^T = P^ R^ gives L = R^^T and
  P = P~ P^. No third pass over A.
* ``rand_qlp_literal``: Algorithm 1 step 5 as printed, P R = (Q^T A)^T, one
  more product with A (section 3.1). With a square m x n Omega and q = 0 this
  is Algorithm 1 exactly (``rand_qlp_full``).
* Both modes give the same Q; they give the same L and P whenever
  d = n or rank(A) <= d (then A P~ P~^T = A).

QR sign convention (not fixed by the paper): every R is returned with a
non-negative diagonal (a zero diagonal is taken as +), so the thin QR of a
full-column-rank matrix is unique and factors compare entry by entry.
"""
from __future__ import annotations

import numpy as np

__all__ = ["householder_qr", "qf", "rand_qlp", "rand_qlp_literal", "rand_qlp_full",
           "residual_fro", "rank_r_error_fro", "rank_r_errors", "RQLPResult"]


def householder_qr(X):
    """Thin QR X = Q R by Householder reflections (section 2, unpivoted QR).

    X is m x d with m >= d. Returns Q (m x d, orthonormal columns) and R
    (d x d, upper triangular with non-negative diagonal), both float64.

    Step j reflects column j's trailing part x = R[j:, j] onto -s*||x|| e_1
    with s = sign(x_0), using the unit vector v = (x + s ||x|| e_1)/||.||;
    H_j = I - 2 v v^T is applied to the trailing columns. Q = H_0 ... H_{d-1}
    times the first d columns of the identity.
    """
    R = np.array(X, dtype=np.float64, copy=True)
    m, d = R.shape
    if m < d:
        raise ValueError("householder_qr needs m >= d")
    vs = []
    for j in range(d):
        x = R[j:, j]
        alpha = np.linalg.norm(x)
        if alpha == 0.0:
            vs.append(None)
            continue
        s = 1.0 if x[0] >= 0.0 else -1.0
        v = x.copy()
        v[0] += s * alpha
        v /= np.linalg.norm(v)
        R[j:, j:] -= 2.0 * np.outer(v, v @ R[j:, j:])
        vs.append(v)
    Rout = np.triu(R[:d, :d])
    Q = np.zeros((m, d))
    Q[:d, :d] = np.eye(d)
    for j in range(d - 1, -1, -1):
        v = vs[j]
        if v is None:
            continue
        Q[j:, :] -= 2.0 * np.outer(v, v @ Q[j:, :])
    sgn = np.where(np.diag(Rout) < 0.0, -1.0, 1.0)
    return Q * sgn, sgn[:, None] * Rout


def qf(X):
    """Q factor of the thin QR of X with R's diagonal made non-negative."""
    return householder_qr(X)[0]


class RQLPResult:
    """Factors of A ~= Q L P^T plus the orthonormal sketch basis P~."""

    def __init__(self, Q, L, P, Ptilde):
        self.Q, self.L, self.P, self.Ptilde = Q, L, P, Ptilde

    def __iter__(self):
        return iter((self.Q, self.L, self.P))


def _sketch_basis(A, Omega, q):
    """P~ = orth(A^T Omega) refined by q power passes (section 3.1, step 3).

    Each pass forms Z = qf(A P~) then P~ = qf(A^T Z): orthonormalising after
    every product leaves the spanned subspace (A^T A)^q A^T Omega unchanged.
    """
    Pt = qf(A.T @ Omega)
    for _ in range(int(q)):
        Z = qf(A @ Pt)
        Pt = qf(A.T @ Z)
    return Pt


def rand_qlp(A, Omega, q=0):
    """Truncated Rand-QLP chain (d = Omega's column count).

    1. Y = A^T Omega; P~ = qf(Y)                      (Alg. 1 step 3)
    2. q times: Z = qf(A P~); P~ = qf(A^T Z)          (power passes)
    3. B = A P~; (Q, R) = qr(B)                       (Alg. 1 step 4)
    4. (P^, R^) = qr(R^T); L = R^^T; P = P~ P^        (step 5 on the d x d R)

    Returns an RQLPResult with Q (m x d), L (d x d lower), P (n x d), P~.
    """
    A = np.asarray(A, dtype=np.float64)
    Omega = np.asarray(Omega, dtype=np.float64)
    Pt = _sketch_basis(A, Omega, q)
    Q, R = householder_qr(A @ Pt)
    Phat, Rhat = householder_qr(R.T)
    return RQLPResult(Q, Rhat.T, Pt @ Phat, Pt)


def rand_qlp_literal(A, Omega, q=0):
    """Algorithm 1 with step 5 as printed: P R' = (Q^T A)^T, L = R'^T.

    Q = orth(A P~) (step 4) and the QR of A^T Q (n x d) gives P and L
    directly; this costs a third product with A.
    """
    A = np.asarray(A, dtype=np.float64)
    Omega = np.asarray(Omega, dtype=np.float64)
    Pt = _sketch_basis(A, Omega, q)
    Q = qf(A @ Pt)
    P, Rp = householder_qr(A.T @ Q)
    return RQLPResult(Q, Rp.T, P, Pt)


def rand_qlp_full(A, Omega):
    """Algorithm 1 exactly: Omega is m x n (full size), no power passes."""
    A = np.asarray(A, dtype=np.float64)
    if Omega.shape != A.shape:
        raise ValueError("Algorithm 1 draws Omega with the shape of A")
    return rand_qlp_literal(A, Omega, 0)


def residual_fro(A, Q, L, P):
    """||A - Q L P^T||_F computed explicitly in float64."""
    A = np.asarray(A, dtype=np.float64)
    return float(np.linalg.norm(A - (Q @ L) @ P.T))


def rank_r_error_fro(A, Q, L, P, r):
    """||A - A_r||_F with A_r = Q L(:, 1:r) P(:, 1:r)^T (section 5.2).

    The printed formula indexes P by rows; with P n x d its first r columns
    are meant (the product is otherwise not conformal).
    """
    A = np.asarray(A, dtype=np.float64)
    Ar = (Q @ L[:, :r]) @ P[:, :r].T
    return float(np.linalg.norm(A - Ar))


def rank_r_errors(A, L):
    """||A - A_r||_F for r = 1..d from the identity of reading C9: for this
    chain A_r = Q L(:, 1:r) P(:, 1:r)^T = A P_r P_r^T (section 5.2), so
    ||A - A_r||_F^2 = ||A||_F^2 - ||L(:, 1:r)||_F^2."""
    A = np.asarray(A, dtype=np.float64)
    L = np.asarray(L, dtype=np.float64)
    nA2 = float((A * A).sum())
    col2 = (L * L).sum(axis=0)
    return np.sqrt(np.maximum(nA2 - np.cumsum(col2), 0.0))
