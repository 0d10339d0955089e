"""Pins for the FP64 oracle: results the paper and the mathematics fix.

Each check compares the oracle with something other than itself: a library
routine (LAPACK via numpy), a brute-force Jacobi SVD, a closed form, an exact
identity, or a theorem's bound. ``test_planted_mistakes_are_caught`` plants
plausible bugs in copies of the oracle and checks that the pins reject them.
"""
import numpy as np
import pytest

from oracle import rqlp_oracle as orc
from oracle.bounds import omega_ratio, subspace_sin, theorem1, theorem2, theorem3
from oracle.jacobi_svd import jacobi_svd
from paper_2110_01011_gb300 import inputs


def _lib_qr(X):
    """LAPACK thin QR with the sign of R's diagonal made non-negative."""
    Qh, Rh = np.linalg.qr(np.asarray(X, dtype=np.float64))
    s = np.where(np.diag(Rh) < 0, -1.0, 1.0)
    return Qh * s, s[:, None] * Rh


def _matrix(m, n, sigma, seed, noise=0.0):
    return inputs.low_rank_matrix(m, n, sigma, noise, seed, dtype=np.float64)


# ---------------------------------------------------------------- QR and SVD pins

@pytest.mark.parametrize("shape", [(50, 13), (200, 200), (37, 1), (9, 9)])
def test_householder_matches_lapack(shape):
    X = inputs.rng(7).standard_normal(shape)
    Q, R = orc.householder_qr(X)
    Ql, Rl = _lib_qr(X)
    assert np.allclose(Q, Ql, atol=1e-12, rtol=0)
    assert np.allclose(R, Rl, atol=1e-12 * np.abs(Rl).max(), rtol=0)
    assert np.allclose(np.tril(R, -1), 0)
    assert (np.diag(R) >= 0).all()
    assert np.linalg.norm(Q.T @ Q - np.eye(shape[1])) < 1e-13
    assert np.linalg.norm(Q @ R - X) < 1e-13 * np.linalg.norm(X)


def test_householder_zero_column():
    X = inputs.rng(3).standard_normal((10, 4))
    X[:, 2] = 0.0
    Q, R = orc.householder_qr(X)
    assert np.linalg.norm(Q @ R - X) < 1e-13 * np.linalg.norm(X)
    assert R[2, 2] == 0.0


def test_jacobi_closed_forms():
    # [[3, 0], [4, 5]]: A^T A = [[25, 20], [20, 25]] -> sigma^2 = 45, 5
    _, s, _ = jacobi_svd(np.array([[3.0, 0.0], [4.0, 5.0]]))
    assert np.allclose(s, [np.sqrt(45.0), np.sqrt(5.0)], rtol=1e-14)
    D = np.diag([0.5, 3.0, 2.0, 0.0])
    _, s, _ = jacobi_svd(D)
    assert np.allclose(s, [3.0, 2.0, 0.5, 0.0], atol=1e-15)


@pytest.mark.parametrize("shape", [(12, 9), (7, 11), (12, 12)])
def test_jacobi_matches_lapack(shape):
    A = inputs.rng(11).standard_normal(shape)
    U, s, V = jacobi_svd(A)
    assert np.allclose(s, np.linalg.svd(A, compute_uv=False), rtol=1e-12, atol=1e-14)
    assert np.linalg.norm((U * s) @ V.T - A) < 1e-12 * np.linalg.norm(A)


# ---------------------------------------------------------------- chain pins

def test_rank_one_closed_form():
    """A = sigma u v^T, d = 1: L = [sigma], Q = s u, P = s v, s = sign(u^T omega)."""
    g = inputs.rng(5)
    u = g.standard_normal(30); u /= np.linalg.norm(u)
    v = g.standard_normal(20); v /= np.linalg.norm(v)
    A = 2.5 * np.outer(u, v)
    for seed in (1, 2, 3):
        Om = inputs.omega(30, 1, seed).astype(np.float64)
        s = np.sign(u @ Om[:, 0])
        Q, L, P = orc.rand_qlp(A, Om, q=1)
        assert np.allclose(L, [[2.5]], rtol=1e-13)
        assert np.allclose(Q[:, 0], s * u, atol=1e-13)
        assert np.allclose(P[:, 0], s * v, atol=1e-13)


@pytest.mark.parametrize("m,n,r,d,q", [(60, 40, 6, 8, 0), (40, 60, 8, 8, 1), (80, 80, 5, 12, 2)])
def test_exact_when_rank_le_d(m, n, r, d, q):
    sig = np.linspace(3.0, 0.5, r)
    A = _matrix(m, n, sig, seed=m + n + r)
    Om = inputs.omega(m, d, 17).astype(np.float64)
    res = orc.rand_qlp(A, Om, q)
    Q, L, P = res
    assert orc.residual_fro(A, Q, L, P) <= 1e-13 * np.linalg.norm(A)
    # the paper-literal step 5 gives the same factorisation when rank <= d
    lit = orc.rand_qlp_literal(A, Om, q)
    assert np.allclose(lit.Q[:, :r], Q[:, :r], atol=1e-10)
    assert np.allclose(lit.L[:r, :r], L[:r, :r], atol=1e-10)
    assert np.allclose(lit.P[:, :r], P[:, :r], atol=1e-10)


def test_full_size_equals_algorithm1():
    """At d = n, q = 0 the truncated chain is Algorithm 1 (QR of R^T vs of A^T Q)."""
    m, n = 30, 18
    A = inputs.rng(21).standard_normal((m, n))
    Om = inputs.rng(22).standard_normal((m, n))
    a = orc.rand_qlp(A, Om, 0)
    b = orc.rand_qlp_full(A, Om)
    for x, y in zip(a, b):
        assert np.allclose(x, y, atol=1e-11)
    assert orc.residual_fro(A, *b) < 1e-12 * np.linalg.norm(A)


@pytest.mark.parametrize("q", [0, 1, 3])
def test_structure_and_residual_identity(q):
    m, n, d = 120, 90, 15
    A = _matrix(m, n, inputs.exp_spectrum(90, 8.0), seed=31, noise=1e-4)
    Om = inputs.omega(m, d, 32).astype(np.float64)
    Q, L, P = orc.rand_qlp(A, Om, q)
    assert np.linalg.norm(Q.T @ Q - np.eye(d)) < 1e-13
    assert np.linalg.norm(P.T @ P - np.eye(d)) < 1e-13
    assert np.all(np.triu(L, 1) == 0.0)
    assert (np.diag(L) > 0).all()
    # Q L P^T = A P~ P~^T is an orthogonal projection of A's rows, hence
    # ||A - Q L P^T||_F^2 = ||A||_F^2 - ||L||_F^2 and the same for prefixes.
    nA2 = np.linalg.norm(A) ** 2
    res = orc.residual_fro(A, Q, L, P)
    assert abs(res ** 2 - (nA2 - np.linalg.norm(L) ** 2)) < 1e-12 * nA2
    for r in (1, 5, d):
        er = orc.rank_r_error_fro(A, Q, L, P, r)
        assert abs(er ** 2 - (nA2 - np.linalg.norm(L[:, :r]) ** 2)) < 1e-12 * nA2


def test_power_pass_subspace_matches_library():
    """P~ = qf((A^T A)^q A^T Omega) (uniqueness of the positive-diagonal QR)."""
    m, n, d = 70, 50, 6
    A = _matrix(m, n, np.linspace(1.0, 0.3, 50), seed=41)
    Om = inputs.omega(m, d, 42).astype(np.float64)
    for q in (0, 1, 2):
        K = A.T @ Om
        for _ in range(q):
            K = A.T @ (A @ K)
        Pt_ref = _lib_qr(K)[0]
        Pt = orc.rand_qlp(A, Om, q).Ptilde
        assert np.allclose(Pt, Pt_ref, atol=1e-9)
        # Q = qf(A P~): checked against LAPACK too
        Q = orc.rand_qlp(A, Om, q).Q
        assert np.allclose(Q, _lib_qr(A @ Pt_ref)[0], atol=1e-9)


def test_orthogonal_covariance():
    """A' = U0 A V0^T, Omega' = U0 Omega  =>  Q' = U0 Q, L' = L, P' = V0 P."""
    m, n, d = 40, 30, 7
    A = _matrix(m, n, inputs.exp_spectrum(30, 5.0), seed=51, noise=1e-3)
    Om = inputs.omega(m, d, 52).astype(np.float64)
    g = inputs.rng(53)
    U0 = inputs.haar_columns(m, m, g)
    V0 = inputs.haar_columns(n, n, g)
    Q, L, P = orc.rand_qlp(A, Om, 1)
    Q2, L2, P2 = orc.rand_qlp(U0 @ A @ V0.T, U0 @ Om, 1)
    assert np.allclose(Q2, U0 @ Q, atol=1e-10)
    assert np.allclose(L2, L, atol=1e-12)
    assert np.allclose(P2, V0 @ P, atol=1e-10)


def test_diag_converges_to_singular_values():
    """Many power passes on a well-separated spectrum: |L_ii| -> sigma_i."""
    m, n, d = 50, 40, 6
    sig = 0.5 ** np.arange(40)
    A = _matrix(m, n, sig, seed=61)
    Om = inputs.omega(m, d, 62).astype(np.float64)
    errs = []
    for q in (0, 2, 40):
        L = orc.rand_qlp(A, Om, q).L
        errs.append(np.max(np.abs(np.diag(L)[:4] - sig[:4]) / sig[:4]))
    assert errs[2] < 1e-9
    assert errs[0] > errs[1] > errs[2]


def test_interlacing_against_jacobi():
    """sigma_i(L_11) <= sigma_i(A) (proof of Theorem 1), brute force on 12 x 10."""
    m, n, k, d = 12, 10, 3, 5
    for seed in range(4):
        A = inputs.rng(70 + seed).standard_normal((m, n))
        Om = inputs.omega(m, d, 80 + seed).astype(np.float64)
        _, sA, _ = jacobi_svd(A)
        for fn in (orc.rand_qlp, orc.rand_qlp_literal):
            L = fn(A, Om, 0).L
            _, sL, _ = jacobi_svd(L[:k, :k])
            assert np.all(sL <= sA[:k] * (1 + 1e-12))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_theorems_hold(seed):
    """Theorems 1-3 with the exact U, V, Sigma of a square synthetic A, q = 0,
    on Algorithm 1 (full-size Omega) and on the truncated literal mode."""
    n, k = 60, 8
    g = inputs.rng(90 + seed)
    U = inputs.haar_columns(n, n, g)
    V = inputs.haar_columns(n, n, g)
    sig = np.concatenate([np.linspace(1.0, 0.5, k), 0.02 * 0.9 ** np.arange(n - k)])
    A = (U * sig) @ V.T
    for Om, fn in ((g.standard_normal((n, n)), orc.rand_qlp_full),
                   (g.standard_normal((n, k + 4)), lambda A_, O_: orc.rand_qlp_literal(A_, O_, 0))):
        Q, L, P = fn(A, Om)
        t = omega_ratio(U, Om, k)
        lower, l22b = theorem1(sig, t, k)
        sL11 = np.linalg.svd(L[:k, :k], compute_uv=False)
        assert np.all(sL11 >= lower * (1 - 1e-10))
        assert np.all(sL11 <= sig[:k] * (1 + 1e-10))
        assert np.linalg.norm(L[k:, k:], 2) <= l22b * (1 + 1e-10)
        b_tq, b_tp, b_pq, b_pp = theorem2(sig, t, k)
        assert subspace_sin(U[:, :k], Q[:, :k]) <= b_tq * (1 + 1e-10)
        assert subspace_sin(V[:, :k], P[:, :k]) <= b_tp * (1 + 1e-10)
        assert np.linalg.norm(U[:, :k].T @ Q[:, k:], 2) <= b_pq * (1 + 1e-10)
        assert np.linalg.norm(V[:, :k].T @ P[:, k:], 2) <= b_pp * (1 + 1e-10)
        for rho in ("fro", 2):
            nA = np.linalg.norm(A, rho)
            tail = np.linalg.norm(np.diag(sig[k:]), rho)
            bq, bp = theorem3(sig, t, k, nA, tail)
            Qk, Pk = Q[:, :k], P[:, :k]
            assert np.linalg.norm(A - Qk @ (Qk.T @ A), rho) <= bq * (1 + 1e-10)
            assert np.linalg.norm(A - (A @ Pk) @ Pk.T, rho) <= bp * (1 + 1e-10)


# ---------------------------------------------------------------- planted mistakes

def _pins_pass(fn):
    """Run a compact set of the pins above against a candidate chain ``fn``."""
    try:
        # exactness at rank <= d (any dropped or mis-indexed term breaks it)
        A = _matrix(40, 30, np.linspace(2.0, 0.5, 5), seed=101)
        Om = inputs.omega(40, 7, 102).astype(np.float64)
        Q, L, P = fn(A, Om, 1)
        if orc.residual_fro(A, Q, L, P) > 1e-12 * np.linalg.norm(A):
            return False
        if np.any(np.triu(L, 1) != 0) or np.any(np.diag(L) < 0):
            return False
        # power-pass subspace vs LAPACK (square, so a transposed operand still runs)
        A = _matrix(36, 36, np.linspace(1.0, 0.3, 36), seed=103)
        Om = inputs.omega(36, 5, 104).astype(np.float64)
        K = A.T @ (A @ (A.T @ Om))
        Pt_ref = _lib_qr(K)[0]
        Q, L, P = fn(A, Om, 1)
        if not np.allclose(Q, _lib_qr(A @ Pt_ref)[0], atol=1e-8):
            return False
        if not np.allclose(P @ P.T, Pt_ref @ Pt_ref.T, atol=1e-8):
            return False
        # covariance under orthogonal changes of basis
        g = inputs.rng(105)
        U0 = inputs.haar_columns(36, 36, g)
        V0 = inputs.haar_columns(36, 36, g)
        Q2, L2, P2 = fn(U0 @ A @ V0.T, U0 @ Om, 1)
        if not (np.allclose(L2, L, atol=1e-10) and np.allclose(Q2, U0 @ Q, atol=1e-8)
                and np.allclose(P2, V0 @ P, atol=1e-8)):
            return False
        return True
    except Exception:
        return False


def _mutant(kind):
    def chain(A, Om, q):
        A = np.asarray(A, float); Om = np.asarray(Om, float)
        if kind == "transposed_sketch":        # A Omega in place of A^T Omega
            Pt = orc.qf(A @ Om)
        else:
            Pt = orc.qf(A.T @ Om)
        passes = q if kind != "dropped_power_pass" else 0
        for _ in range(passes):
            Z = orc.qf(A @ Pt)
            Pt = orc.qf(A.T @ Z) if kind != "power_pass_sign" else orc.qf(-(A.T @ Z))
        Q, R = orc.householder_qr(A @ Pt)
        if kind == "no_transpose_step5":
            Ph, Rh = orc.householder_qr(R)
        else:
            Ph, Rh = orc.householder_qr(R.T)
        L = Rh.T
        P = Pt @ Ph if kind != "rotate_transposed" else Pt @ Ph.T
        if kind == "unsigned_qr":
            Q = -Q
        return Q, L, P
    return chain


def test_planted_mistakes_are_caught():
    assert _pins_pass(lambda A, O, q: tuple(orc.rand_qlp(A, O, q)))
    for kind in ("transposed_sketch", "dropped_power_pass", "no_transpose_step5",
                 "rotate_transposed", "unsigned_qr", "power_pass_sign"):
        assert not _pins_pass(_mutant(kind)), kind


# ---------------------------------------------------------------- closed forms of the bound helpers

def _planes(a, b, g):
    """Orthonormal X = [e1, e2] and Y = [cos a e1 + sin a e3, cos b e2 + sin b e4]
    in R^6, both rotated by one Haar matrix: their canonical angles are a and b
    (the definitions of section 4.1, Theorem 2, applied to two planes)."""
    E = np.eye(6)
    X = E[:, :2]
    Y = np.stack([np.cos(a) * E[:, 0] + np.sin(a) * E[:, 2], np.cos(b) * E[:, 1] + np.sin(b) * E[:, 3]], axis=1)
    W = inputs.haar_columns(6, 6, g)
    return W @ X, W @ Y


@pytest.mark.parametrize("a,b", [(0.3, 1.1), (1.2, 0.2), (0.0, 0.0), (np.pi / 2, 0.5), (0.7, 0.7)])
def test_subspace_sin_closed_form(a, b):
    g = inputs.rng(311)
    X, Y = _planes(a, b, g)
    want = max(np.sin(a), np.sin(b))
    assert abs(subspace_sin(X, Y) - want) < 1e-13
    assert abs(subspace_sin(Y, X) - want) < 1e-13          # symmetric for equal dimensions
    # any orthonormal basis of the same spans gives the same distance
    G = inputs.haar_columns(2, 2, g)
    assert abs(subspace_sin(X @ G, Y @ G.T) - want) < 1e-13


def test_subspace_sin_rejects_plausible_mistakes():
    """Candidate definitions a slip could produce disagree with the closed form."""
    g = inputs.rng(312)
    X, Y = _planes(0.4, 0.9, g)
    want = np.sin(0.9)
    wrong = {
        "norm_XtY_minus_1": abs(np.linalg.norm(X.T @ Y, 2) - 1.0),
        "smallest_angle": float(np.linalg.svd(Y - X @ (X.T @ Y), compute_uv=False)[-1]),
        "cosine": float(np.linalg.svd(X.T @ Y, compute_uv=False)[-1]),
        "frobenius": float(np.linalg.norm(Y - X @ (X.T @ Y))),
    }
    for name, v in wrong.items():
        assert abs(v - want) > 1e-3, name
    assert abs(subspace_sin(X, Y) - want) < 1e-13


def test_omega_ratio_closed_form():
    """Omega~ = U^T Omega_1 = [D1; D2] with D1 = diag(d), D2 = [diag(c); 0]:
    Omega~_2 Omega~_1^{-1} = [diag(c / d); 0], whose 2-norm is max |c_i / d_i|
    (the quantity t of section 4.1, eq. 3, that Theorems 1-3 carry)."""
    n, k = 12, 3
    g = inputs.rng(313)
    U = inputs.haar_columns(n, n, g)
    d = np.array([2.0, -0.5, 4.0])
    c = np.array([1.0, 0.75, -10.0])
    Ot = np.zeros((n, k + 2))
    Ot[:k, :k] = np.diag(d)
    Ot[k:2 * k, :k] = np.diag(c)
    Ot[:, k:] = g.standard_normal((n, 2))          # columns past k do not enter t
    Om = U @ Ot
    want = np.max(np.abs(c / d))
    assert abs(omega_ratio(U, Om, k) - want) < 1e-12 * want
    # planted slips: Omega~_1^{-1} Omega~_2 shape error, U in place of U^T, inverse dropped
    assert abs(float(np.linalg.norm((U @ Om[:, :k])[k:] @ np.linalg.inv((U @ Om[:, :k])[:k]), 2)) - want) > 1e-3
    assert abs(float(np.linalg.norm(Ot[k:, :k] @ Ot[:k, :k], 2)) - want) > 1e-3
    assert abs(float(np.linalg.norm(Ot[k:, :k], 2)) - want) > 1e-3


@pytest.mark.parametrize("a,b", [(0.3, 1.1), (1.2, 0.2), (0.0, 0.5)])
def test_subspace_sines_and_cosines_closed_form(a, b):
    """All canonical angles of the two rotated planes: sines {sin a, sin b},
    cosines {cos a, cos b}, largest first; the largest sine is subspace_sin."""
    from oracle.bounds import subspace_cosines, subspace_sines
    X, Y = _planes(a, b, inputs.rng(321))
    np.testing.assert_allclose(subspace_sines(X, Y), sorted([np.sin(a), np.sin(b)], reverse=True), atol=1e-13)
    np.testing.assert_allclose(subspace_cosines(X, Y), sorted([np.cos(a), np.cos(b)], reverse=True), atol=1e-13)
    assert abs(subspace_sines(X, Y)[0] - subspace_sin(X, Y)) < 1e-13


def test_rank_r_errors_identity():
    """The identity against the explicit residual of A_r = Q L(:, 1:r) P(:, 1:r)^T
    (section 5.2) for every r, and against the tail of an exact low-rank A
    (rank 6, d = 10: from r = 6 on the error is 0 up to rounding)."""
    m, n = 80, 60
    A = _matrix(m, n, inputs.exp_spectrum(n, 5.0), seed=131, noise=1e-3)
    Om = inputs.omega(m, 12, 132).astype(np.float64)
    Q, L, P = orc.rand_qlp(A, Om, 1)
    errs = orc.rank_r_errors(A, L)
    for r in range(1, 13):
        assert abs(errs[r - 1] - orc.rank_r_error_fro(A, Q, L, P, r)) < 1e-10 * np.linalg.norm(A)
    B = _matrix(m, n, np.linspace(2.0, 1.0, 6), seed=133)
    Q, L, P = orc.rand_qlp(B, inputs.omega(m, 10, 134).astype(np.float64), 0)
    e = orc.rank_r_errors(B, L)
    assert np.all(e[5:] < 1e-6 * np.linalg.norm(B)) and e[4] > 0.5
