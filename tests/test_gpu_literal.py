"""Step 5 as Algorithm 1 prints it (section 3.1): the QR of (Q^T A)^T = A^T Q,
a third pass over A, against the oracle's literal chain; and Algorithm 1
itself (d = n, q = 0) against the oracle's full-size Algorithm 1."""
import numpy as np
import pytest

from oracle import rqlp_oracle as orc
from paper_2110_01011_gb300 import inputs
from parity_util import compare, run_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m,n,k,p,q", [(1000, 1000, 20, 5, 1), (700, 1300, 24, 8, 0), (2049, 777, 40, 6, 2)])
@pytest.mark.parametrize("prec", [0, 1], ids=["fp32", "bf16x3"])
def test_literal_step5_matches_oracle(m, n, k, p, q, prec):
    """rank(A) > d, so the literal L and P differ from the d x d form's."""
    A = inputs.low_rank_matrix(m, n, inputs.poly_spectrum(min(m, n), 1.0), 1e-4, seed=m + n)
    Om = inputs.omega(m, k + p, seed=m * 3 + n)
    gpu = run_gpu(A, Om, k, p, q, precision=prec, literal=True)
    err = compare(A, Om, k, p, q, gpu, elem_atol=5e-4, precision=prec, literal=True)
    # the two readings of step 5 really differ on this input
    d_form = orc.rand_qlp(A.astype(np.float64), Om.astype(np.float64), q)
    lit = orc.rand_qlp_literal(A.astype(np.float64), Om.astype(np.float64), q)
    gap = np.max(np.abs(np.diag(d_form.L)[:k] - np.diag(lit.L)[:k]) / np.diag(lit.L)[:k])
    assert gap > 10 * err["Lii_rel"], (gap, err["Lii_rel"])


@pytest.mark.parametrize("n", [64, 150, 256])
def test_algorithm1_full_size(n):
    """d = n, q = 0, literal step 5: Algorithm 1 exactly (square Omega)."""
    A = inputs.low_rank_matrix(n, n, inputs.exp_spectrum(n, n / 6), 1e-6, seed=900 + n)
    Om = inputs.omega(n, n, seed=901 + n)
    Q, L, P, info, _ = run_gpu(A, Om, n, 0, 0, literal=True)
    assert info[0] == 0
    ref = orc.rand_qlp_full(A.astype(np.float64), Om.astype(np.float64))
    k = n // 4   # leading block: the trailing columns of a numerically low-rank A are not unique
    assert np.max(np.abs(np.diag(L)[:k] - np.diag(ref.L)[:k]) / np.diag(ref.L)[:k]) < 1e-4
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) < 1e-4 and np.linalg.norm(P.T @ P - np.eye(n)) < 1e-4
    assert np.linalg.norm(A - (Q @ L) @ P.T) < 1e-5 * np.linalg.norm(A)
