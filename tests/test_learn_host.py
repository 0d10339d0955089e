"""Host logic of the predictor's training module, checked against the FP64
reference: labels from a table of excess errors, and the folding of the
feature standardisation into the first layer."""
import numpy as np

from oracle import mlp_oracle as mo
from paper_2110_01011_gb300 import inputs, learn


def test_label_matches_reference():
    g = inputs.rng(3)
    for trial in range(300):
        k = int(g.integers(1, 200))
        tab = 10.0 ** g.uniform(-5, -1, size=(5, 3))
        tab[g.random((5, 3)) < 0.2] = np.inf      # failed runs
        assert learn.label_from_table(tab, k, 1e-3) == mo.label(tab, k, 1e-3)


def test_label_infeasible_and_ties():
    tab = np.full((5, 3), 1.0)
    assert learn.label_from_table(tab, 10, 1e-3) == (4, 2)
    tab = np.full((5, 3), 0.0)
    assert learn.label_from_table(tab, 10, 1e-3) == (0, 0)
    # (q=1, p=5): cost 4 * 15 = 60; (q=0, p=20): cost 2 * 30 = 60 -> the smaller q wins
    tab = np.full((5, 3), 1.0)
    tab[1, 0] = 0.0
    tab[0, 2] = 0.0
    assert learn.label_from_table(tab, 10, 1e-3) == (0, 2)


def test_fold_standardisation():
    g = inputs.rng(8)
    theta = g.standard_normal(mo.n_params()) * 0.3
    X = g.standard_normal((50, mo.N_FEATURES)) * 3.0 + 1.5
    mu, sd = X.mean(axis=0), X.std(axis=0)
    ref, _ = mo.forward(theta, (X - mu) / sd)
    got, _ = mo.forward(learn.fold_standardisation(theta, mu, sd), X)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_unfold_inverts_fold():
    """Resuming training: unfolding saved (folded) weights with the new
    dataset's mu, sd gives the network on standardised features, and folding
    it back returns the saved weights."""
    g = inputs.rng(9)
    saved = g.standard_normal(mo.n_params()) * 0.3
    X = g.standard_normal((40, mo.N_FEATURES)) * 2.0 - 0.7
    mu, sd = X.mean(axis=0), X.std(axis=0)
    theta = learn.unfold_standardisation(saved, mu, sd)
    ref, _ = mo.forward(saved, X)
    got, _ = mo.forward(theta, (X - mu) / sd)
    np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(learn.fold_standardisation(theta, mu, sd), saved, rtol=1e-12, atol=1e-12)


def test_draw_problem_tail_window():
    g = inputs.rng(21)
    for _ in range(20):
        m, n, k, sig, kind = learn.draw_problem(g)
        assert 16 <= k <= min(m, n) // 2 - 20 and len(sig) == min(m, n)
        assert 0.5 * n - 1 <= m <= 2 * n
        tail = np.sqrt((sig[k:] ** 2).sum() / (sig ** 2).sum())
        assert 0.003 <= tail <= 0.30


def test_rows_and_targets():
    feats = np.arange(24, dtype=float).reshape(2, 12)
    tab = np.full((5, 3), np.inf)
    tab[3, 0] = 5e-3
    tab[4, 2] = 5e-5
    X, Y = learn.rows(feats, np.array([tab, tab]))
    assert X.shape == (2, 12) and Y.shape == (2, 15)
    np.testing.assert_allclose(Y[0], mo.error_target(tab)[0])
    assert Y[0, 3 * 3 + 0] == np.log10(5e-3) and Y[0, 4 * 3 + 2] == -4.0 and Y[0, 0] == 1.0


def test_choose_and_targets_match_reference():
    g = inputs.rng(13)
    for trial in range(300):
        k = int(g.integers(1, 200))
        est = g.uniform(-4, 0.5, mo.N_OUT)
        t = 10.0 ** g.uniform(-3, -1)
        delta = float(g.uniform(0, 0.5))
        assert learn.choose_from_estimates(est, k, t, delta) == mo.choose(est, k, t, delta)
    tab = 10.0 ** g.uniform(-6, 2, size=(5, 3))
    tab[0, 1] = np.inf
    np.testing.assert_array_equal(learn.error_target(tab), mo.error_target(tab))


def test_calibrate_is_the_residual_quantile():
    """delta = the chosen quantile of measured - estimated over the entries
    within a decade of the request range; estimates off by a constant c give
    delta = c."""
    g = inputs.rng(14)
    tabs = 10.0 ** g.uniform(-3.5, -0.5, size=(40, 5, 3))
    Y = np.concatenate([mo.error_target(t) for t in tabs])
    assert abs(learn.calibrate(Y - 0.25, tabs) - 0.25) < 1e-12
    r = g.standard_normal(Y.shape) * 0.1
    d = learn.calibrate(Y - r, tabs, quantile=0.9)
    assert abs(d - np.quantile(r, 0.9)) < 1e-12


def test_evaluate_at_counts():
    ks = np.array([10, 10])
    t0 = np.full((5, 3), 1.0)
    t0[2, 1] = 0.0
    t1 = np.full((5, 3), 1.0)
    t1[0, 0] = 0.0
    tabs = np.array([t0, t1])
    r = learn.evaluate_at(np.array([2, 0]), np.array([1, 0]), tabs, ks, 1e-2)
    assert r["learned_success"] == 1.0 and r["feasible"] == 1.0
    assert r["learned_cost"] == (6 * 20 + 2 * 15) / 2
    assert r["default_success"] == 0.5 and r["matched_fixed"] is None
    r = learn.evaluate_at(np.array([0, 0]), np.array([0, 0]), tabs, ks, 1e-2)
    assert r["learned_success"] == 0.5 and r["matched_fixed"] == [0, 5]
