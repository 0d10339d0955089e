"""Training data, training and evaluation of the learned (q, p) predictor.

Everything runs on the GPU through the library's C ABI. For each generated
matrix A and Gaussian Omega of width w = k + 20:

* features: ``rqlp_probe_features`` (12 statistics of the probe sketch's
  R-diagonal);
* error table: the chain is run once at width w with ``rqlp_sketch`` and
  ``rqlp_orth`` (Y = A^T Omega, P~ = qf(Y); each power pass Z = qf(A P~),
  P~ = qf(A^T Z)), saving after q = 0..4 passes the R factor of B = A P~.
  QR factors are prefix-consistent (the first d' columns of qf(X) and the
  leading d' x d' block of R belong to X(:, 1:d')), so the width-(k + p)
  chain's rank-k basis is P_k = P~(:, 1:k+p) P^(:, 1:k) with
  R(1:k+p, 1:k+p)^T = P^ R^: one chain gives all 15 (q, p) pairs
  (14 passes over A instead of 90);
* excess error eps = ||A - A P_k P_k^T||_F / (sum_{i>k} sigma_i^2)^(1/2) - 1,
  in FP64 from P_k re-orthonormalised in FP64 (||A||^2 - ||A P_k||^2 is then
  exact to ~1e-11 of the tail for tails >= 0.3 % of ||A||_F).

The network maps the features to estimates of log10 eps for all 15 pairs
(targets clipped to [1e-4, 10]) and is trained by mean squared error with the
library's kernels (``rqlp_mlp_grad``, ``rqlp_mlp_adam``). A request t is then
answered with the cheapest pair, by cost (2q + 2)(k + p), whose estimate plus
a margin delta is at most log10 t. delta is calibrated on the validation
matrices: the 90th percentile of (measured - estimated) log10 eps over the
entries near the requests' range, so that a pair picked as feasible reaches
the request about nine times in ten. Trained weights (standardisation folded
into the first layer, so the network takes raw features; delta last) are
stored as little-endian float32 in ``data/qp_mlp.f32`` with a JSON
description beside them.

    python -m paper_2110_01011_gb300.learn --train 4000 --test 500 --out <dir> --save
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

from . import inputs, rqlp

TARGET_RANGE = (1e-3, 1e-1)      # requests the predictor is calibrated for
EVAL_TARGETS = (1e-3, 3e-3, 1e-2, 3e-2, 1e-1)
CALIBRATION_QUANTILE = 0.9       # delta: this quantile of (measured - estimated) log10 eps
LOG_FLOOR, LOG_CEIL = -4.0, 1.0  # training targets: log10 eps clipped to [1e-4, 10]
Q_CHOICES = rqlp.Q_CHOICES
P_CHOICES = rqlp.P_CHOICES
HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "data", "qp_mlp.f32")
FALLBACK = (2, 10)


def cost(q, p, k):
    return (2 * q + 2) * (k + p)


def label_from_table(eps, k, target):
    """The cheapest pair that truly reaches `target` (ties: smaller q, then p);
    (4, 20) when none does."""
    best = None
    for qi, q in enumerate(Q_CHOICES):
        for pi, p in enumerate(P_CHOICES):
            if eps[qi][pi] <= target:
                key = (cost(q, p, k), q, p)
                if best is None or key < best[0]:
                    best = (key, qi, pi)
    return (len(Q_CHOICES) - 1, len(P_CHOICES) - 1) if best is None else (best[1], best[2])


def error_target(tab):
    """log10 eps of a (5 x 3) table as the 15 training targets, clipped to
    [1e-4, 10] (failed runs, inf, count as 10)."""
    e = np.asarray(tab, dtype=np.float64).reshape(-1, len(Q_CHOICES) * len(P_CHOICES))
    e = np.where(np.isfinite(e), e, 10.0 ** LOG_CEIL)
    return np.log10(np.clip(e, 10.0 ** LOG_FLOOR, 10.0 ** LOG_CEIL))


def choose_from_estimates(est, k, target, delta):
    """The device's selection on the host: (qi, pi) of the cheapest pair whose
    estimate plus delta is at most log10(target); (4, 20) when none is."""
    lt = np.log10(target)
    best = None
    for qi, q in enumerate(Q_CHOICES):
        for pi, p in enumerate(P_CHOICES):
            if est[qi * len(P_CHOICES) + pi] + delta <= lt:
                key = (cost(q, p, k), q, p)
                if best is None or key < best[0]:
                    best = (key, qi, pi)
    return (len(Q_CHOICES) - 1, len(P_CHOICES) - 1) if best is None else (best[1], best[2])


def draw_problem(g, n_range=(384, 2048), k_range=(16, 236), square=False):
    """Sizes (m / n in [1/2, 2], or m = n), spectrum (exponential, rate in
    [5, 100], or polynomial, alpha in [0.5, 3]) and k (log-uniform in
    [16, 236], so that k + 20 fits the widest sketch of 256 columns, and
    k + 20 <= min(m, n) / 2) with the optimal rank-k tail at 0.3-30 % of
    ||A||_F."""
    while True:
        n = int(math.exp(g.uniform(math.log(n_range[0]), math.log(n_range[1]))))
        m = n if square else int(n * math.exp(g.uniform(math.log(0.5), math.log(2.0))))
        mn = min(m, n)
        if g.random() < 0.5:
            sig = inputs.exp_spectrum(mn, float(g.uniform(5.0, 100.0)))
            kind = "exp"
        else:
            sig = inputs.poly_spectrum(mn, float(g.uniform(0.5, 3.0)))
            kind = "poly"
        total = float((sig ** 2).sum())
        kmax = min(k_range[1], mn // 2 - 20)
        if kmax < k_range[0]:
            continue
        k = int(round(math.exp(g.uniform(math.log(k_range[0]), math.log(kmax)))))
        tail = math.sqrt(float((sig[k:] ** 2).sum()) / total)
        if 0.003 <= tail <= 0.30:
            return m, n, k, sig, kind


def make_matrix(m, n, sig, seed, device):
    """U diag(sig) V^T with Haar U (m x r), V (n x r), r = min(m, n), FP32
    (the Q factors of Gaussians, R-diagonal made positive)."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    r = min(m, n)

    def haar(rows):
        G = torch.randn(rows, r, generator=gen, device=device, dtype=torch.float32)
        Qh, Rh = torch.linalg.qr(G)
        s = torch.sign(torch.diagonal(Rh))
        s[s == 0] = 1.0
        return Qh * s

    U, V = haar(m), haar(n)
    sg = torch.as_tensor(sig, device=device, dtype=torch.float32)
    return ((U * sg) @ V.T).contiguous()


def eps_table(A, Om, k, tail2):
    """eps[qi][pi] for every (q, p) from one width-(k + 20) chain (see the
    module docstring)."""
    import torch
    A64 = A.double()
    nA2 = float((A64 * A64).sum())
    tab = np.full((len(Q_CHOICES), len(P_CHOICES)), np.inf)
    Y, _ = rqlp.sketch(A, Om, 1)
    Pt, _, info, _ = rqlp.orth(Y)
    bad = int(info[0]) != 0
    for qi, q in enumerate(Q_CHOICES):
        if q > 0:
            Z, _ = rqlp.sketch(A, Pt, 0)
            _, _, i1, _ = rqlp.orth(Z)
            Y, _ = rqlp.sketch(A, Z, 1)
            Pt, _, i2, _ = rqlp.orth(Y)
            bad = bad or int(i1[0]) != 0 or int(i2[0]) != 0
        if bad:
            break
        B, _ = rqlp.sketch(A, Pt, 0)
        R = torch.linalg.qr(B.double(), mode="r")[1]
        Pt64 = Pt.double()
        bases = []
        for p in P_CHOICES:
            d = k + p
            Ph = torch.linalg.qr(R[:d, :d].T)[0]
            bases.append(torch.linalg.qr(Pt64[:, :d] @ Ph[:, :k])[0])
        AP = A64 @ torch.cat(bases, dim=1)
        for pi in range(len(P_CHOICES)):
            blk = AP[:, pi * k:(pi + 1) * k]
            res2 = max(nA2 - float((blk * blk).sum()), 0.0)
            tab[qi, pi] = math.sqrt(res2 / tail2) - 1.0
    return tab


def build_dataset(count, seed, device, log_every=500, n_range=(384, 2048), square=False):
    """Probe features (12 statistics), error tables, k and sizes for
    ``count`` generated matrices."""
    import torch
    g = inputs.rng(seed)
    feats, ks, tabs, meta = [], [], [], []
    t0 = time.time()
    for i in range(count):
        m, n, k, sig, kind = draw_problem(g, n_range=n_range, square=square)
        A = make_matrix(m, n, sig, seed * 1000003 + i, device)
        Om = torch.from_numpy(inputs.omega(m, k + 20, seed=seed * 7919 + i)).to(device)
        tail2 = float((sig[k:] ** 2).sum())
        tabs.append(eps_table(A, Om, k, tail2))
        f, _ = rqlp.probe_features(A, k, Om, precision=rqlp.PREC_BF16X3)
        feats.append(f.cpu().numpy().astype(np.float64)[:12])
        ks.append(k)
        meta.append((m, n, k, kind))
        if log_every and (i + 1) % log_every == 0:
            print(f"  {i + 1}/{count} matrices, {time.time() - t0:.0f} s", flush=True)
    return np.array(feats), np.array(ks), np.array(tabs), np.array(meta, dtype=object)


def rows(feats, tabs):
    """Training rows: the features of each matrix and the 15 targets of its
    error table."""
    X = np.asarray(feats, dtype=np.float64)
    Y = np.concatenate([error_target(t) for t in tabs]) if len(tabs) else np.zeros((0, 15))
    return X, Y


def init_params(seed, F=rqlp.MLP_FEATURES, H=rqlp.MLP_HIDDEN, O=rqlp.MLP_OUTPUTS):
    g = inputs.rng(seed)
    W1 = g.standard_normal((F, H)) * math.sqrt(2.0 / F)
    W2 = g.standard_normal((H, H)) * math.sqrt(2.0 / H)
    W3 = g.standard_normal((H, O)) * math.sqrt(1.0 / H)
    return np.concatenate([W1.ravel(), np.zeros(H), W2.ravel(), np.zeros(H), W3.ravel(), np.zeros(O), [0.0]])


def train(X, Y, steps=3000, lr=3e-3, seed=11, device="cuda", val=None, every=50, init=None):
    """Full-batch Adam with the library's kernels on the mean squared error of
    the 15 log10-error estimates. With val = (Xv, Yv), the parameters of the
    lowest validation loss (checked every ``every`` steps) are returned.
    init: parameters to start from (on standardised features, see
    unfold_standardisation); Adam's moments start at zero. Returns (params,
    curve of (step, loss, val_loss))."""
    import torch
    dev = torch.device(device)

    def upload(Xa, Ya):
        B = Xa.shape[0]
        nb = rqlp.rqlp_mlp_workspace_bytes(B)
        return (B, torch.from_numpy(np.ascontiguousarray(Xa, dtype=np.float32)).to(dev),
                torch.from_numpy(np.ascontiguousarray(Ya, dtype=np.float32)).to(dev),
                torch.empty(nb // 4 + 64, dtype=torch.float32, device=dev), nb)

    start = init_params(seed) if init is None else np.asarray(init, dtype=np.float64)
    if start.size != rqlp.MLP_PARAMS:
        raise ValueError(f"init: {start.size} parameters, expected {rqlp.MLP_PARAMS}")
    prm = torch.from_numpy(start.astype(np.float32)).to(dev)
    m1 = torch.zeros_like(prm)
    m2 = torch.zeros_like(prm)
    grad = torch.empty_like(prm)
    vgrad = torch.empty_like(prm)
    loss = torch.empty(1, device=dev)
    vloss = torch.empty(1, device=dev)
    tr = upload(X, Y)
    va = upload(*val) if val is not None else None
    st = torch.cuda.current_stream().cuda_stream

    def grad_of(data, g, lo):
        B, Xd, Yd, ws, nb = data
        s = rqlp.rqlp_mlp_grad(prm.data_ptr(), Xd.data_ptr(), Yd.data_ptr(), B, g.data_ptr(), lo.data_ptr(),
                               ws.data_ptr(), nb, st)
        if s != 0:
            raise rqlp.RqlpError(s, "rqlp_mlp_grad")

    curve, best, best_val = [], None, math.inf
    for step in range(1, steps + 1):
        grad_of(tr, grad, loss)
        s = rqlp.rqlp_mlp_adam(prm.data_ptr(), grad.data_ptr(), m1.data_ptr(), m2.data_ptr(), prm.numel(),
                               lr, 0.9, 0.999, 1e-8, step, st)
        if s != 0:
            raise rqlp.RqlpError(s, "rqlp_mlp_adam")
        if step % every == 0 or step == steps:
            v = math.nan
            if va is not None:
                grad_of(va, vgrad, vloss)
                v = float(vloss.item())
                if v < best_val:
                    best_val, best = v, prm.clone()
            curve.append((step, float(loss.item()), v))
    out = best if best is not None else prm
    return out.cpu().numpy().astype(np.float64), curve


def fold_standardisation(params, mu, sd, F=rqlp.MLP_FEATURES, H=rqlp.MLP_HIDDEN):
    """Network on (x - mu) / sd  ->  the same network on raw x."""
    p = params.copy()
    W1 = p[:F * H].reshape(F, H)
    b1 = p[F * H:F * H + H]
    W1n = W1 / sd[:, None]
    b1n = b1 - (mu / sd) @ W1
    p[:F * H] = W1n.ravel()
    p[F * H:F * H + H] = b1n
    return p


def unfold_standardisation(params, mu, sd, F=rqlp.MLP_FEATURES, H=rqlp.MLP_HIDDEN):
    """Inverse of fold_standardisation: the network on raw x -> the same
    network on (x - mu) / sd (to resume training from saved weights)."""
    p = np.asarray(params, dtype=np.float64).copy()
    W1n = p[:F * H].reshape(F, H)
    b1n = p[F * H:F * H + H]
    W1 = W1n * sd[:, None]
    b1 = b1n + mu @ W1n
    p[:F * H] = W1.ravel()
    p[F * H:F * H + H] = b1
    return p


def predict_estimates(params, X):
    """The network's 15 log10-error estimates per row, on the device with
    rqlp_mlp_forward."""
    import torch
    dev = torch.device("cuda")
    prm = torch.from_numpy(np.asarray(params, dtype=np.float32)).to(dev)
    Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to(dev)
    out = torch.empty(X.shape[0], rqlp.MLP_OUTPUTS, device=dev)
    s = rqlp.rqlp_mlp_forward(prm.data_ptr(), Xd.data_ptr(), X.shape[0], out.data_ptr(),
                              torch.cuda.current_stream().cuda_stream)
    if s != 0:
        raise rqlp.RqlpError(s, "rqlp_mlp_forward")
    return out.cpu().numpy().astype(np.float64)


def calibrate(est, tabs, quantile=CALIBRATION_QUANTILE):
    """delta: the `quantile` of (measured - estimated) log10 eps over the
    entries whose measured error lies within a decade of the requests' range
    (the entries that decide a pick)."""
    Y = np.concatenate([error_target(t) for t in tabs])
    r = Y - np.asarray(est)
    lo, hi = math.log10(TARGET_RANGE[0]) - 1.0, math.log10(TARGET_RANGE[1]) + 1.0
    sel = (Y >= lo) & (Y <= hi)
    return float(np.quantile(r[sel], quantile)) if sel.any() else 0.0


def choose(est, ks, target, delta):
    """(qi, pi) arrays of the picks for every row."""
    picks = [choose_from_estimates(est[i], int(ks[i]), target, delta) for i in range(len(ks))]
    return np.array([a for a, _ in picks]), np.array([b for _, b in picks])


def evaluate_at(qi, pi, tabs, ks, target):
    """Success (eps <= target) and mean cost of the chosen pairs, against every
    fixed pair; ``matched_fixed`` is the cheapest fixed pair whose success rate
    is at least the chosen pairs'."""
    n = len(ks)
    ok = np.array([tabs[i][qi[i], pi[i]] <= target for i in range(n)])
    c = np.array([cost(Q_CHOICES[qi[i]], P_CHOICES[pi[i]], ks[i]) for i in range(n)], dtype=np.float64)
    fixed = {}
    for a, q in enumerate(Q_CHOICES):
        for b, p in enumerate(P_CHOICES):
            okf = np.array([tabs[i][a, b] <= target for i in range(n)])
            fixed[(q, p)] = (float(okf.mean()), float(np.mean([cost(q, p, kk) for kk in ks])))
    match = sorted((cf, qp) for qp, (sr, cf) in fixed.items() if sr >= ok.mean())
    feasible = np.array([(t <= target).any() for t in tabs])
    best = [min((cost(q, p, ks[i]) for a, q in enumerate(Q_CHOICES) for b, p in enumerate(P_CHOICES)
                 if tabs[i][a, b] <= target), default=math.nan) for i in range(n)]
    return {
        "target": target,
        "n": int(n),
        "feasible": float(feasible.mean()),
        "learned_success": float(ok.mean()),
        "learned_cost": float(c.mean()),
        "default_success": fixed[FALLBACK][0],
        "default_cost": fixed[FALLBACK][1],
        "matched_fixed": list(match[0][1]) if match else None,
        "matched_fixed_cost": match[0][0] if match else None,
        "cost_vs_matched": float(c.mean() / match[0][0]) if match else None,
        "best_cost_feasible": float(np.nanmean(best)) if feasible.any() else None,
    }


def evaluate(params, feats, tabs, ks, targets=EVAL_TARGETS):
    est = predict_estimates(params, feats)
    delta = float(np.asarray(params)[-1])
    return [evaluate_at(*choose(est, ks, t, delta), tabs, ks, t) for t in targets]


def save_weights(params, meta, path=WEIGHTS):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    params.astype("<f4").tofile(path)
    with open(path[:-4] + ".json", "w") as f:
        json.dump(meta, f, indent=1)


def load_weights(path=WEIGHTS):
    w = np.fromfile(path, dtype="<f4")
    if w.size != rqlp.MLP_PARAMS:
        raise ValueError(f"{path}: {w.size} parameters, expected {rqlp.MLP_PARAMS}")
    return w.astype(np.float32)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=4000)
    ap.add_argument("--test", type=int, default=500)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--out", default="learn_out")
    ap.add_argument("--data", default=None, help="reuse a qp_dataset.npz instead of generating one")
    ap.add_argument("--large", type=int, default=0,
                    help="add this many square training matrices with n in [1000, 8000] (and a fifth as many to test)")
    ap.add_argument("--save", action="store_true", help="write data/qp_mlp.f32")
    ap.add_argument("--resume", default=None,
                    help="start from saved weights (a qp_mlp.f32); Adam's moments restart from zero")
    a = ap.parse_args()
    import torch
    torch.cuda.set_device(0)
    t0 = time.time()
    if a.data:
        z = np.load(a.data, allow_pickle=True)
        ftr, ktr, tabtr, fte, kte, tabte = (z[n] for n in ("ftr", "ktr", "tabtr", "fte", "kte", "tabte"))
    else:
        ftr, ktr, tabtr, _ = build_dataset(a.train, seed=501, device="cuda")
        fte, kte, tabte, _ = build_dataset(a.test, seed=909, device="cuda")
    if a.large > 0:
        big = (1000, 8000)   # square, as the 20000-matrix specification of the training set draws them
        f2, k2, t2, _ = build_dataset(a.large, seed=601, device="cuda", log_every=100, n_range=big, square=True)
        f3, k3, t3, _ = build_dataset(max(1, a.large // 5), seed=919, device="cuda", log_every=100, n_range=big,
                                      square=True)
        # interleave so that the validation slice (the first tenth) holds both sizes
        order = np.random.default_rng(5).permutation(len(ktr) + len(k2))
        ftr, ktr, tabtr = (np.concatenate([x, y])[order] for x, y in ((ftr, f2), (ktr, k2), (tabtr, t2)))
        fte, kte, tabte = (np.concatenate([x, y]) for x, y in ((fte, f3), (kte, k3), (tabte, t3)))
    t_data = time.time() - t0
    # 10 % of the training matrices validate the early stop and calibrate delta
    nv = max(1, len(ktr) // 10)
    Xtr, Ytr = rows(ftr[nv:], tabtr[nv:])
    Xva, Yva = rows(ftr[:nv], tabtr[:nv])
    mu = Xtr.mean(axis=0)
    sd = Xtr.std(axis=0)
    sd[sd < 1e-6] = 1.0
    t1 = time.time()
    init = unfold_standardisation(load_weights(a.resume), mu, sd) if a.resume else None
    params, curve = train((Xtr - mu) / sd, Ytr, steps=a.steps, lr=a.lr, val=((Xva - mu) / sd, Yva), init=init)
    t_train = time.time() - t1
    params = fold_standardisation(params, mu, sd)
    params[-1] = calibrate(predict_estimates(params, ftr[:nv]), tabtr[:nv])
    ev = evaluate(params, fte, tabte, kte)
    est_te = predict_estimates(params, fte)
    Yte = np.concatenate([error_target(t) for t in tabte])
    report = {"train_matrices": int(len(ktr)), "train_rows": int(len(Ytr)), "val_rows": int(len(Yva)),
              "delta": float(params[-1]), "calibration_quantile": CALIBRATION_QUANTILE,
              "test_matrices": int(len(kte)), "steps": a.steps, "lr": a.lr, "target_range": TARGET_RANGE,
              "test_rmse_log10": float(np.sqrt(np.mean((est_te - Yte) ** 2))),
              "seconds_data": t_data, "seconds_train": t_train, "curve": curve, "test": ev}
    os.makedirs(a.out, exist_ok=True)
    if not a.data or a.large > 0:
        np.savez(os.path.join(a.out, "qp_dataset.npz"), ftr=ftr, ktr=ktr, tabtr=tabtr, fte=fte, kte=kte,
                 tabte=tabte)
    with open(os.path.join(a.out, "qp_report.json"), "w") as f:
        json.dump(report, f, indent=1)
    params.astype("<f4").tofile(os.path.join(a.out, "qp_mlp.f32"))
    if a.save:
        save_weights(params, {k: v for k, v in report.items() if k != "curve"})
    print(json.dumps({k: v for k, v in report.items() if k != "curve"}, indent=1))
    print("curve tail", curve[-3:])


if __name__ == "__main__":
    main()
