"""Pins for the FP64 reference of the learned (q, p) predictor: gradients
against central finite differences, closed forms (zero network, first Adam
step, geometric probe diagonal), and the label rule on hand-built tables."""
import numpy as np

from oracle import mlp_oracle as mo
from oracle import rqlp_oracle as orc
from paper_2110_01011_gb300 import inputs


def _theta(seed, scale=0.3):
    return inputs.rng(seed).standard_normal(mo.n_params()) * scale


def test_param_count():
    assert mo.n_params() == 12 * 64 + 64 + 64 * 64 + 64 + 64 * 15 + 15 + 1 == 5968


def test_zero_network_loss_is_the_mean_square_target():
    """All-zero weights estimate 0 everywhere: the loss is mean(Y^2) and only
    the output biases see a gradient, -2 mean(Y) per output; none for delta."""
    g0 = inputs.rng(1)
    X = g0.standard_normal((7, mo.N_FEATURES))
    Y = g0.uniform(-4, 1, (7, mo.N_OUT))
    loss, g = mo.loss_and_grads(np.zeros(mo.n_params()), X, Y)
    assert abs(loss - float((Y ** 2).mean())) < 1e-14
    p = mo.unpack(g)
    assert np.allclose(p["W1"], 0) and np.allclose(p["W2"], 0) and np.allclose(p["W3"], 0)
    assert np.allclose(p["b3"], -2.0 * Y.mean(axis=0) / mo.N_OUT, atol=1e-15)
    assert p["delta"][0] == 0.0


def test_gradient_matches_finite_differences():
    g0 = inputs.rng(2)
    X = g0.standard_normal((9, mo.N_FEATURES))
    Y = g0.uniform(-4, 1, (9, mo.N_OUT))
    th = _theta(3)
    _, g = mo.loss_and_grads(th, X, Y)
    idx = inputs.rng(4).choice(mo.n_params() - 1, 60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(th)
        e[i] = h
        fd = (mo.loss_and_grads(th + e, X, Y)[0] - mo.loss_and_grads(th - e, X, Y)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i])), (i, fd, g[i])
    # delta does not enter the loss
    e = np.zeros_like(th)
    e[-1] = 0.3
    assert mo.loss_and_grads(th + e, X, Y)[0] == mo.loss_and_grads(th, X, Y)[0]


def test_first_adam_step_is_lr_times_sign():
    g = inputs.rng(5).standard_normal(50)
    th = np.zeros(50)
    th1, m1, m2 = mo.adam(th, g, np.zeros(50), np.zeros(50), 1, lr=0.01, eps=0.0)
    assert np.allclose(th1, -0.01 * np.sign(g), atol=1e-15)


def test_features_of_geometric_diagonal():
    rho, k, w = 0.8, 30, 50
    r = rho ** np.arange(w)
    f = mo.probe_features(r, k, 400, 300)
    lg = np.log10(rho)
    h = (k + 1) // 2
    expect = [(k - 1) * lg, (h - 1) * lg, (k - h) * lg, lg, 5 * lg, 10 * lg, 20 * lg, 10 * lg, 0.0,
              np.log10(k), np.log10(300), k / 300]
    assert np.allclose(f, expect, atol=1e-12)


def test_choose_rule():
    """Cheapest pair whose estimate plus delta is within the request."""
    k = 40
    est = np.full(mo.N_OUT, 0.0)          # log10 eps = 0: nothing qualifies
    assert mo.choose(est, k, 1e-2, 0.0) == (4, 2)
    est[1 * 3 + 2] = -3.0                 # (1, 20): cost 4 * 60 = 240
    est[2 * 3 + 0] = -3.0                 # (2, 5): cost 6 * 45 = 270
    assert mo.choose(est, k, 1e-2, 0.0) == (1, 2)
    assert mo.choose(est, k, 1e-2, 0.5) == (1, 2)       # -3 + 0.5 <= -2
    assert mo.choose(est, k, 1e-2, 1.5) == (4, 2)       # the margin rules both out
    est[0 * 3 + 2] = -2.0                 # (0, 20): cost 2 * 60 = 120, exactly at the request
    assert mo.choose(est, k, 1e-2, 0.0) == (0, 2)
    assert mo.choose(est, k, 1e-2, 1e-9) == (1, 2)
    # ties on cost go to the smaller q: (1, 5) cost 4 * 45 = 180 vs (0, 50)? no such p; use k = 10:
    # (1, 5) cost 60 and (0, 20) cost 60
    e2 = np.full(mo.N_OUT, 0.0)
    e2[1 * 3 + 0] = -3.0
    e2[0 * 3 + 2] = -3.0
    assert mo.choose(e2, 10, 1e-2, 0.0) == (0, 2)


def test_error_target_clips_and_maps_failures():
    tab = np.array([[1e-6, 1e-3, 0.5], [20.0, np.inf, -0.1], [1e-2, 1e-1, 1.0], [3e-4, 3e-3, 3e-2], [1, 2, 3]])
    y = mo.error_target(tab)
    assert y.shape == (1, 15)
    assert np.allclose(y[0, :3], [-4.0, -3.0, np.log10(0.5)])
    assert np.allclose(y[0, 3:6], [1.0, 1.0, -4.0])        # above 10, a failed run, a negative error
    assert np.all(y >= mo.LOG_FLOOR) and np.all(y <= mo.LOG_CEIL)


def test_label_rule():
    inf = np.inf
    # feasible: (1, 20) cost 4*(k+20); (2, 5) cost 6*(k+5); k = 40 -> 240 vs 270
    tab = np.full((5, 3), inf)
    tab[1][2] = 0.0
    tab[2][0] = 0.0
    assert mo.label(tab, 40, 1e-3) == (1, 2)
    # tie on cost -> smaller q: (0, 20) cost 2*60 = 120 vs nothing cheaper
    tab = np.full((5, 3), inf)
    tab[0][2] = 1e-4
    assert mo.label(tab, 40, 1e-3) == (0, 2)
    assert mo.label(np.full((5, 3), inf), 40, 1e-3) == (4, 2)


def test_excess_error_matches_explicit_residual():
    m = n = 120
    k, p, q = 10, 5, 1
    sig = inputs.exp_spectrum(n, 6.0)
    A = inputs.low_rank_matrix(m, n, sig, 0.0, seed=7, dtype=np.float64)
    Om = inputs.omega(m, k + p, seed=8).astype(np.float64)
    Q, L, P = orc.rand_qlp(A, Om, q)
    tail2 = float((sig[k:] ** 2).sum())
    eps = mo.excess_error(float(np.linalg.norm(A) ** 2), float(np.linalg.norm(L[:, :k]) ** 2), tail2)
    direct = orc.rank_r_error_fro(A, Q, L, P, k) / np.sqrt(tail2) - 1.0
    assert abs(eps - direct) < 1e-9
    assert eps >= -1e-9   # no rank-k approximation beats the SVD's
