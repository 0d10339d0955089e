"""Right-hand sides of Theorems 1-3 and the measured quantities they bound.

TEST INFRASTRUCTURE ONLY. Inputs: the exact SVD factors of a synthetic A
(known by construction), the Gaussian Omega used by the factorisation, the
rank split k, and the factors Q, L, P produced by the oracle.

Notation (section 4.1, eq. 3): Omega_1 = first k columns of Omega,
Omega~ = U^T Omega_1 split into its first k rows Omega~_1 and the rest
Omega~_2; t = ||Omega~_2 Omega~_1^{-1}||_2; psi_i = sigma_{k+1} / sigma_i.
U must be square (m = n) for Omega~ to have the stated shape.

Readings of the printed statement:
* Theorem 1's lower bound is proved for sigma_i(L_11) (the proof bounds the
  eigenvalues of A^T Q_1 Q_1^T A = L_11 P_1^T P_1 L_11^T); ``theorem1`` returns
  the bound and the test compares it with sigma_i(L_11).
* Theorem 2's fourth line repeats "sin phi_Q"; it is the bound for sin phi_P.
  The printed numerators carry ||Omega~_2 Omega~_1^{-1}||^2, but the proof
  (x / (1 + x) increasing in x = sigma_1(G)^2) yields the first power:
  sin phi_Q <= psi_k^2 t / sqrt(1 + psi_k^4 t^2) and
  sin phi_P <= psi_k^3 t / sqrt(1 + psi_k^6 t^2).
"""
from __future__ import annotations

import numpy as np

__all__ = ["omega_ratio", "theorem1", "theorem2", "theorem3", "subspace_sin", "subspace_sines", "subspace_cosines"]


def omega_ratio(U, Omega, k):
    """t = ||Omega~_2 Omega~_1^{-1}||_2 with Omega~ = U^T Omega[:, :k]."""
    Ot = U.T @ np.asarray(Omega, dtype=np.float64)[:, :k]
    O1, O2 = Ot[:k, :], Ot[k:, :]
    return float(np.linalg.norm(O2 @ np.linalg.inv(O1), 2))


def theorem1(sigma, t, k):
    """(lower bounds on sigma_i(L_11), i = 1..k;  upper bound on ||L_22||_2)."""
    s = np.asarray(sigma, dtype=np.float64)
    psi = s[k] / s[:k]
    lower = s[:k] / np.sqrt(1.0 + psi ** 4 * t ** 2)
    l22 = (1.0 + psi[k - 1] ** 2 * t) * s[k]
    return lower, l22


def theorem2(sigma, t, k):
    """Upper bounds (sin theta_Q, sin theta_P, sin phi_Q, sin phi_P)."""
    s = np.asarray(sigma, dtype=np.float64)
    pk = s[k] / s[k - 1]
    return (pk ** 2 * t, pk ** 3 * t,
            pk ** 2 * t / np.sqrt(1.0 + pk ** 4 * t ** 2),
            pk ** 3 * t / np.sqrt(1.0 + pk ** 6 * t ** 2))


def theorem3(sigma, t, k, normA_rho, tail_rho):
    """Bounds on ||(I - Q_k Q_k^T) A||_rho and ||A (I - P_k P_k^T)||_rho."""
    s = np.asarray(sigma, dtype=np.float64)
    pk = s[k] / s[k - 1]
    return tail_rho + normA_rho * pk ** 2 * t, tail_rho + normA_rho * pk ** 3 * t


def subspace_sin(X, Y):
    """dist(R(X), R(Y)) for orthonormal X, Y of equal column count: the sine
    of the largest canonical angle, ||X_perp^T Y||_2 = ||(I - X X^T) Y||_2."""
    return float(np.linalg.norm(Y - X @ (X.T @ Y), 2))


def subspace_sines(X, Y):
    """Sines of the canonical angles between R(Y) and R(X) for orthonormal X
    (rows x a) and Y (rows x b), largest first: the singular values of
    (I - X X^T) Y (section 4.1, the distances of Theorem 2). The largest is
    ``subspace_sin`` when a = b."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    return np.linalg.svd(Y - X @ (X.T @ Y), compute_uv=False)


def subspace_cosines(X, Y):
    """Singular values of X^T Y, largest first (the cosines of the canonical
    angles; their largest is ||X^T Y||_2, the form of Theorem 2's sin phi
    bounds with Y the trailing columns of Q or P)."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    return np.linalg.svd(X.T @ Y, compute_uv=False)
