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
    assert learn.label_from_table(tab, 10) == (4, 2)
    tab = np.full((5, 3), 0.0)
    assert learn.label_from_table(tab, 10) == (0, 0)
    # (q=1, p=5): cost 4 * 15 = 60; (q=0, p=20): cost 2 * 30 = 60 -> the smaller q wins
    tab = np.full((5, 3), 1.0)
    tab[1, 0] = 0.0
    tab[0, 2] = 0.0
    assert learn.label_from_table(tab, 10) == (0, 2)


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


def test_rows_and_labels():
    feats = np.arange(24, dtype=float).reshape(2, 12)
    tab = np.full((5, 3), np.inf)
    tab[3, 0] = 5e-3        # feasible for requests >= 5e-3
    tab[4, 2] = 5e-4        # feasible for requests >= 5e-4
    tabs = np.array([tab, tab])
    X, yq, yp, idx, ts = learn.rows(feats, np.array([20, 40]), tabs, [[1e-2, 1e-3], [1e-4]], margin=1.0)
    assert X.shape == (3, 13) and list(idx) == [0, 0, 1]
    np.testing.assert_allclose(X[:, 12], np.log10([1e-2, 1e-3, 1e-4]))
    assert (yq[0], yp[0]) == (3, 0) and (yq[1], yp[1]) == (4, 2) and (yq[2], yp[2]) == (4, 2)


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


def test_rows_margin_tightens_labels():
    feats = np.zeros((1, 12))
    tab = np.full((5, 3), np.inf)
    tab[1, 0] = 8e-3        # reaches 1e-2, not 1e-2 / 2
    tab[3, 0] = 4e-3        # reaches both
    tabs = np.array([tab])
    _, yq, yp, _, _ = learn.rows(feats, np.array([20]), tabs, [[1e-2]], margin=1.0)
    assert (yq[0], yp[0]) == (1, 0)
    _, yq, yp, _, _ = learn.rows(feats, np.array([20]), tabs, [[1e-2]], margin=2.0)
    assert (yq[0], yp[0]) == (3, 0)
