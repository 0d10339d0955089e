"""Device evaluation utilities against the FP64 oracle: rank-r errors of
section 5.2 (identity and explicit residual) and the canonical-angle
distances of section 4.1 (Theorem 2)."""
import numpy as np
import pytest

from oracle import rqlp_oracle as orc
from oracle.bounds import omega_ratio, subspace_cosines, subspace_sines, theorem2
from paper_2110_01011_gb300 import inputs
from parity_util import run_gpu

pytestmark = pytest.mark.gpu


def _factored(m, n, k, p, q, prec, seed):
    A = inputs.low_rank_matrix(m, n, inputs.exp_spectrum(min(m, n), 15.0), 1e-4, seed=seed)
    Om = inputs.omega(m, k + p, seed=seed + 1)
    return A, Om, run_gpu(A, Om, k, p, q, precision=prec)


@pytest.mark.parametrize("prec", [0, 1], ids=["fp32", "bf16x3"])
def test_rank_errors_and_explicit_residual(prec):
    import torch

    from paper_2110_01011_gb300 import rqlp
    m, n, k, p, q = 1500, 900, 30, 8, 1
    A, Om, (Q, L, P, info, diag) = _factored(m, n, k, p, q, prec, seed=5150)
    d = k + p
    dL = torch.from_numpy(L.astype(np.float32)).cuda()
    ddiag = torch.from_numpy(diag).cuda()
    errs = rqlp.rank_errors(dL, ddiag).cpu().numpy()
    A64 = A.astype(np.float64)
    nA = np.linalg.norm(A64)
    # the identity on the device's L against the explicit FP64 residual of the same factors
    for r in (1, 5, k, d):
        ref = orc.rank_r_error_fro(A64, Q, L, P, r)
        assert abs(errs[r - 1] - ref) <= 1e-3 * ref + 2e-6 * nA, (r, errs[r - 1], ref)
    # the oracle's identity on the oracle's own factors (a different L: compare the leading-k errors)
    ref_chain = orc.rand_qlp(A64, Om.astype(np.float64), q)
    ref_errs = orc.rank_r_errors(A64, ref_chain.L)
    assert np.all(np.abs(errs[:k] - ref_errs[:k]) <= 1e-3 * ref_errs[:k] + 2e-6 * nA)
    dA = torch.from_numpy(A).cuda()
    dQ = torch.from_numpy(Q.astype(np.float32)).cuda()
    dP = torch.from_numpy(P.astype(np.float32)).cuda()
    for r in (1, 7, k, d):
        got = float(rqlp.rank_residual(dA, dQ, dL, dP, r).item())
        ref = orc.rank_r_error_fro(A64, Q, L, P, r)
        assert abs(got - ref) <= 1e-4 * ref + 1e-6 * nA, (r, got, ref)


def _orthonormal(rows, cols, seed):
    return inputs.haar_columns(rows, cols, inputs.rng(seed)).astype(np.float32)


@pytest.mark.parametrize("rows,a,b", [(5000, 40, 40), (777, 13, 9), (3000, 200, 200), (64, 1, 1)])
def test_subspace_angles_match_oracle(rows, a, b):
    import torch

    from paper_2110_01011_gb300 import rqlp
    X = _orthonormal(rows, a, rows + a)
    # Y: a mix of X's span and fresh directions, so the angles spread over (0, pi/2)
    Z = _orthonormal(rows, b, rows + b + 1).astype(np.float64)
    mix = X[:, :b].astype(np.float64) * np.linspace(1.0, 0.05, b) + Z
    Y = np.linalg.qr(mix)[0].astype(np.float32)
    dX, dY = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    sines = rqlp.subspace_angles(dX, dY).cpu().numpy()
    coss = rqlp.subspace_angles(dX, dY, cosines=True).cpu().numpy()
    X64, Y64 = X.astype(np.float64), Y.astype(np.float64)
    np.testing.assert_allclose(sines, subspace_sines(X64, Y64), atol=2e-6, rtol=0)
    np.testing.assert_allclose(coss, subspace_cosines(X64, Y64), atol=2e-6, rtol=0)


def test_subspace_angles_closed_form():
    """Two planes at angles a, b inside R^4000 (rotated by a Haar basis)."""
    import torch

    from paper_2110_01011_gb300 import rqlp
    n, a, b = 4000, 0.3, 1.1
    W = inputs.haar_columns(n, 4, inputs.rng(77))
    X = W[:, :2]
    Y = np.stack([np.cos(a) * W[:, 0] + np.sin(a) * W[:, 2], np.cos(b) * W[:, 1] + np.sin(b) * W[:, 3]], axis=1)
    dX, dY = (torch.from_numpy(np.ascontiguousarray(v, dtype=np.float32)).cuda() for v in (X, Y))
    np.testing.assert_allclose(rqlp.subspace_angles(dX, dY).cpu().numpy(), [np.sin(b), np.sin(a)], atol=1e-6)
    np.testing.assert_allclose(rqlp.subspace_angles(dX, dY, cosines=True).cpu().numpy(), [np.cos(a), np.cos(b)],
                               atol=1e-6)


@pytest.mark.parametrize("prec", [0, 1], ids=["fp32", "bf16x3"])
def test_theorem2_distances_on_device(prec):
    """Theorem 2 (section 4.1) on a square problem with known U, V, q = 0 and
    step 5 as Algorithm 1 prints it (the theorem's P comes from the QR of
    A^T Q): the device's distances between R(U_k), R(Q_k) and R(V_k), R(P_k)
    (and the sin phi forms) equal the oracle's on the same factors and stay
    below the theorem's bounds."""
    import torch

    from paper_2110_01011_gb300 import rqlp
    n, k, p = 400, 10, 6
    g = inputs.rng(4040)
    U = inputs.haar_columns(n, n, g)
    V = inputs.haar_columns(n, n, g)
    sig = np.concatenate([np.linspace(1.0, 0.6, k), 0.05 * 0.95 ** np.arange(n - k)])
    A = ((U * sig) @ V.T).astype(np.float32)
    Om = inputs.omega(n, k + p, seed=4041)
    Q, L, P, info, _ = run_gpu(A, Om, k, p, 0, precision=prec, literal=True)
    assert info[0] == 0
    t = omega_ratio(U, Om.astype(np.float64), k)
    b_tq, b_tp, b_pq, b_pp = theorem2(sig, t, k)
    f32 = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()
    s_tq = rqlp.subspace_angles(f32(U[:, :k]), f32(Q[:, :k])).cpu().numpy()[0]
    s_tp = rqlp.subspace_angles(f32(V[:, :k]), f32(P[:, :k])).cpu().numpy()[0]
    s_pq = rqlp.subspace_angles(f32(U[:, :k]), f32(Q[:, k:]), cosines=True).cpu().numpy()[0]
    s_pp = rqlp.subspace_angles(f32(V[:, :k]), f32(P[:, k:]), cosines=True).cpu().numpy()[0]
    Uf, Vf = U.astype(np.float32).astype(np.float64), V.astype(np.float32).astype(np.float64)
    assert abs(s_tq - subspace_sines(Uf[:, :k], Q[:, :k])[0]) < 2e-6
    assert abs(s_tp - subspace_sines(Vf[:, :k], P[:, :k])[0]) < 2e-6
    assert abs(s_pq - subspace_cosines(Uf[:, :k], Q[:, k:])[0]) < 2e-6
    assert abs(s_pp - subspace_cosines(Vf[:, :k], P[:, k:])[0]) < 2e-6
    assert s_tq <= b_tq and s_tp <= b_tp and s_pq <= b_pq and s_pp <= b_pp
