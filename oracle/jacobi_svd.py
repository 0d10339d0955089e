"""One-sided Jacobi SVD (Hestenes) for tiny matrices -- TEST INFRASTRUCTURE ONLY.

Brute-force singular values used to pin the oracle on inputs of a dozen rows
or so. Plane rotations are applied to column pairs (p, r) of a working copy W
of A (m x n, m >= n) until every pair is orthogonal to machine precision; the
singular values are then the column norms of W and the right singular vectors
the accumulated rotations (Golub & Van Loan, section 8.6.3 / Hestenes 1958).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["jacobi_svd"]


def jacobi_svd(A, tol=1e-15, max_sweeps=60):
    """Return (U, s, V) with A = U diag(s) V^T, s descending (float64)."""
    W = np.array(A, dtype=np.float64, copy=True)
    m, n = W.shape
    transposed = False
    if m < n:
        W = W.T.copy()
        m, n = n, m
        transposed = True
    V = np.eye(n)
    for _ in range(max_sweeps):
        off = 0.0
        for p in range(n - 1):
            for r in range(p + 1, n):
                a = float(W[:, p] @ W[:, p])
                b = float(W[:, r] @ W[:, r])
                c = float(W[:, p] @ W[:, r])
                if a == 0.0 or b == 0.0:
                    continue
                rel = abs(c) / math.sqrt(a * b)
                off = max(off, rel)
                if rel <= tol:
                    continue
                zeta = (b - a) / (2.0 * c)
                t = math.copysign(1.0, zeta) / (abs(zeta) + math.sqrt(1.0 + zeta * zeta))
                cs = 1.0 / math.sqrt(1.0 + t * t)
                sn = cs * t
                wp, wr = W[:, p].copy(), W[:, r].copy()
                W[:, p] = cs * wp - sn * wr
                W[:, r] = sn * wp + cs * wr
                vp, vr = V[:, p].copy(), V[:, r].copy()
                V[:, p] = cs * vp - sn * vr
                V[:, r] = sn * vp + cs * vr
        if off <= tol:
            break
    s = np.linalg.norm(W, axis=0)
    order = np.argsort(-s, kind="stable")
    s = s[order]
    V = V[:, order]
    W = W[:, order]
    U = np.zeros_like(W)
    nz = s > 0
    U[:, nz] = W[:, nz] / s[nz]
    if transposed:
        return V, s, U
    return U, s, V
