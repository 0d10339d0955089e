"""Property tests of the FP64 oracle over random small problems (hypothesis):
for any full-rank A, any Gaussian Omega and any q, Rand-QLP (Algorithm 1,
truncated to d = k + p columns) returns Q and P with orthonormal columns and
L lower triangular with a positive diagonal, Q L P^T is the projection
A P~ P~^T (so ||A||_F^2 = ||L||_F^2 + ||A - Q L P^T||_F^2 and the same for
the leading r columns), and with d = min(m, n) it reproduces A."""
import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

from oracle import rqlp_oracle as orc  # noqa: E402


@st.composite
def problems(draw, full=False):
    m = draw(st.integers(3, 24))
    n = draw(st.integers(3, 24))
    mn = min(m, n)
    d = mn if full else draw(st.integers(1, mn))
    k = draw(st.integers(1, d))
    q = draw(st.integers(0, 3))
    seed = draw(st.integers(0, 2 ** 31 - 1))
    g = np.random.default_rng(seed)
    A = g.standard_normal((m, n)) * np.exp(-np.arange(n) / draw(st.floats(1.0, 20.0)))[None, :]
    Om = g.standard_normal((m, d))
    return A, Om, k, q


@settings(max_examples=150, deadline=None, derandomize=True)
@given(problems())
def test_structure_and_projection_identities(prob):
    A, Om, k, q = prob
    d = Om.shape[1]
    r = orc.rand_qlp(A, Om, q)
    Q, L, P = r.Q, r.L, r.P
    assert Q.shape == (A.shape[0], d) and P.shape == (A.shape[1], d) and L.shape == (d, d)
    assert np.linalg.norm(Q.T @ Q - np.eye(d)) < 1e-10
    assert np.linalg.norm(P.T @ P - np.eye(d)) < 1e-10
    assert np.all(np.triu(L, 1) == 0.0) and np.all(np.diag(L) > 0)
    nA2 = np.linalg.norm(A) ** 2
    assert abs(orc.residual_fro(A, Q, L, P) ** 2 - (nA2 - np.linalg.norm(L) ** 2)) <= 1e-10 * nA2
    er = orc.rank_r_error_fro(A, Q, L, P, k)
    assert abs(er ** 2 - (nA2 - np.linalg.norm(L[:, :k]) ** 2)) <= 1e-10 * nA2


@settings(max_examples=60, deadline=None, derandomize=True)
@given(problems(full=True))
def test_full_width_reproduces_a(prob):
    A, Om, _, q = prob
    r = orc.rand_qlp(A, Om, q)
    assert np.linalg.norm(A - r.Q @ r.L @ r.P.T) <= 1e-9 * np.linalg.norm(A)
