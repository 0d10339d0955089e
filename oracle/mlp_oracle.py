"""FP64 reference of the learned (q, p) predictor -- TEST INFRASTRUCTURE ONLY.

The predictor picks the number of power passes q in {0..4} and the
oversampling p in {5, 10, 20} for a requested accuracy, from cheap statistics
of a probe sketch. The paper has no such component (its Rand-QLP has neither
q nor p); this file is the plain definition the CUDA kernels are checked
against.

* ``probe_features``: 12 features of the R-diagonal r_1..r_w of
  qf(A^T Omega_w), the probe sketch of width w = k + 20 (the widest sketch
  any p in {5, 10, 20} needs, so the probe is also the first sketch of the
  chain).
* ``forward`` / ``loss_and_grads``: 3-layer MLP, F -> H -> H -> 15, ReLU,
  whose 15 outputs estimate log10 of the excess rank-k error of every
  (q, p) (pair j = 3 qi + pi), trained by mean squared error against
  ``error_target`` of the measured errors.
* ``choose``: the cheapest pair, by cost (2q + 2)(k + p) (ties: smaller q,
  then smaller p), whose estimate plus the calibrated margin delta stays at
  or below log10 of the request; (4, 20) when none does.
* ``adam``: one Adam step (Kingma & Ba 2015), bias-corrected.
* ``label``: the cheapest pair that truly reaches a request (evaluation).

The flat parameter block is W1 (F x H), b1, W2 (H x H), b2, W3 (H x 15), b3
and, last, the margin delta (log10 units; set by calibration, not by the
gradient, whose entry for it is 0).
"""
from __future__ import annotations

import numpy as np

__all__ = ["Q_CHOICES", "P_CHOICES", "N_FEATURES", "HIDDEN", "N_OUT", "param_shapes", "n_params", "unpack",
           "probe_features", "forward", "loss_and_grads", "adam", "error_target", "choose", "label",
           "excess_error", "pair_cost", "LOG_FLOOR", "LOG_CEIL"]

Q_CHOICES = (0, 1, 2, 3, 4)
P_CHOICES = (5, 10, 20)
N_FEATURES = 12
HIDDEN = 64
N_OUT = len(Q_CHOICES) * len(P_CHOICES)
LOG_FLOOR, LOG_CEIL = -4.0, 1.0   # error targets are clipped to [1e-4, 10]


def param_shapes(F=N_FEATURES, H=HIDDEN):
    """(name, shape) in the flat order."""
    return [("W1", (F, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, N_OUT)), ("b3", (N_OUT,)),
            ("delta", (1,))]


def n_params(F=N_FEATURES, H=HIDDEN):
    return sum(int(np.prod(s)) for _, s in param_shapes(F, H))


def unpack(theta, F=N_FEATURES, H=HIDDEN):
    out, off = {}, 0
    for name, shape in param_shapes(F, H):
        size = int(np.prod(shape))
        out[name] = np.asarray(theta[off:off + size], dtype=np.float64).reshape(shape)
        off += size
    return out


def pair_cost(q, p, k):
    """Flops of the passes over A, up to a constant: (2q + 2) passes of width k + p."""
    return (2 * q + 2) * (k + p)


def probe_features(r, k, m, n):
    """Features of the probe R-diagonal r (length w >= k + 1, positive).

    With l_i = log10(r_i / r_1) (1-based i, indices clamped to [1, w]):
    [l_k, l_ceil(k/2), l_k - l_ceil(k/2), l_{k+1} - l_k, l_{k+5} - l_k,
     l_{k+10} - l_k, l_{k+20} - l_k, l_{k+20} - l_{k+10}, std of the steps
     l_{i+1} - l_i over i < w, log10 k, log10 min(m, n), k / min(m, n)].
    """
    r = np.asarray(r, dtype=np.float64)
    w = r.shape[0]
    lr = np.log10(np.maximum(r, 1e-30) / r[0])

    def L(i):   # 1-based, clamped
        return lr[min(max(i, 1), w) - 1]

    steps = np.diff(lr)
    mn = min(m, n)
    h = (k + 1) // 2
    return np.array([
        L(k), L(h), L(k) - L(h), L(k + 1) - L(k), L(k + 5) - L(k), L(k + 10) - L(k), L(k + 20) - L(k),
        L(k + 20) - L(k + 10), float(np.std(steps)) if steps.size else 0.0,
        np.log10(k), np.log10(mn), k / mn,
    ])


def forward(theta, X, F=N_FEATURES, H=HIDDEN):
    """Estimates (B x 15) and the activations needed by the gradient."""
    p = unpack(theta, F, H)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ p["W1"] + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"] + p["b2"]
    h2 = np.maximum(z2, 0.0)
    out = h2 @ p["W3"] + p["b3"]
    return out, (X, z1, h1, z2, h2)


def loss_and_grads(theta, X, Y, F=N_FEATURES, H=HIDDEN):
    """Mean over the batch and the 15 outputs of (estimate - Y)^2, and its
    gradient w.r.t. theta (0 for delta)."""
    p = unpack(theta, F, H)
    out, (X, z1, h1, z2, h2) = forward(theta, X, F, H)
    Y = np.asarray(Y, dtype=np.float64)
    B = X.shape[0]
    r = out - Y
    loss = float((r * r).sum() / (B * N_OUT))
    d3 = 2.0 * r / (B * N_OUT)
    gW3 = h2.T @ d3
    gb3 = d3.sum(axis=0)
    dz2 = (d3 @ p["W3"].T) * (z2 > 0)
    gW2 = h1.T @ dz2
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ p["W2"].T) * (z1 > 0)
    gW1 = X.T @ dz1
    gb1 = dz1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3, [0.0]])
    return loss, g


def adam(theta, g, m1, m2, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (step is 1-based); returns new (theta, m1, m2)."""
    m1 = beta1 * m1 + (1 - beta1) * g
    m2 = beta2 * m2 + (1 - beta2) * g * g
    mh = m1 / (1 - beta1 ** step)
    vh = m2 / (1 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m1, m2


def error_target(eps_table):
    """Training targets: log10 of the excess errors, clipped to [1e-4, 10]
    (requests live in [1e-3, 1e-1]; failed runs, inf, become 10)."""
    e = np.asarray(eps_table, dtype=np.float64).reshape(-1, N_OUT)
    e = np.where(np.isfinite(e), e, 10.0)
    return np.log10(np.clip(e, 10.0 ** LOG_FLOOR, 10.0 ** LOG_CEIL))


def choose(est, k, target, delta):
    """(qi, pi) of the cheapest pair with est[3 qi + pi] + delta <= log10(target);
    (4, 2) -- q = 4, p = 20 -- when none qualifies."""
    best = None
    lt = np.log10(target)
    for qi, q in enumerate(Q_CHOICES):
        for pi, p in enumerate(P_CHOICES):
            if est[qi * len(P_CHOICES) + pi] + delta <= lt:
                key = (pair_cost(q, p, k), q, p)
                if best is None or key < best[0]:
                    best = (key, qi, pi)
    if best is None:
        return len(Q_CHOICES) - 1, len(P_CHOICES) - 1
    return best[1], best[2]


def excess_error(normA2, lead_L_sq, tail2):
    """epsilon = ||A - A P_k P_k^T||_F / sqrt(tail2) - 1, with the residual from
    ||A||_F^2 - ||L(:, 1:k)||_F^2 (orthogonal projection identity) and tail2 =
    sum_{i > k} sigma_i^2 (the optimum)."""
    res2 = max(normA2 - lead_L_sq, 0.0)
    return float(np.sqrt(res2 / tail2) - 1.0)


def label(eps_table, k, target):
    """eps_table[qi][pi] = excess error of (Q_CHOICES[qi], P_CHOICES[pi]).
    Returns (qi, pi) of the cheapest feasible pair, else the largest one."""
    best = None
    for qi, q in enumerate(Q_CHOICES):
        for pi, p in enumerate(P_CHOICES):
            if eps_table[qi][pi] <= target:
                key = (pair_cost(q, p, k), q, p)
                if best is None or key < best[0]:
                    best = (key, qi, pi)
    if best is None:
        return len(Q_CHOICES) - 1, len(P_CHOICES) - 1
    return best[1], best[2]
