"""Training data, training and evaluation of the learned (q, p) predictor.

Everything runs on the GPU through the library's C ABI. For each generated
matrix A and Gaussian Omega of width w = k + 20:

* features: ``rqlp_probe_features`` (statistics of the probe sketch's
  R-diagonal; the 13th input is log10 of the requested error);
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
  exact to ~1e-11 of the tail for tails >= 0.3 % of ||A||_F);
* rows: several requested errors per matrix, log-uniform in [1e-3, 1e-1];
  label = the cheapest pair, by cost (2q + 2)(k + p) (ties: smaller q, then
  smaller p), whose eps is at most the request / LABEL_MARGIN; (4, 20) when
  none is. The margin keeps the prediction on the safe side of a boundary
  that the features only approximate: without it about a third of the
  predictions for 1-3 % requests missed the request.

The MLP is trained with the library's kernels (``rqlp_mlp_grad``,
``rqlp_mlp_adam``). Trained weights (standardisation folded into the first
layer, so the network takes raw features) are stored as little-endian
float32 in ``data/qp_mlp.f32`` with a JSON description beside them.

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

TARGET = 1e-3                    # the headline request
LABEL_MARGIN = 2.0               # labels aim at request / LABEL_MARGIN
TARGET_RANGE = (1e-3, 1e-1)      # requests seen in training
EVAL_TARGETS = (1e-3, 3e-3, 1e-2, 3e-2, 1e-1)
Q_CHOICES = rqlp.Q_CHOICES
P_CHOICES = rqlp.P_CHOICES
HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "data", "qp_mlp.f32")
FALLBACK = (2, 10)


def cost(q, p, k):
    return (2 * q + 2) * (k + p)


def label_from_table(eps, k, target=TARGET):
    best = None
    for qi, q in enumerate(Q_CHOICES):
        for pi, p in enumerate(P_CHOICES):
            if eps[qi][pi] <= target:
                key = (cost(q, p, k), q, p)
                if best is None or key < best[0]:
                    best = (key, qi, pi)
    return (len(Q_CHOICES) - 1, len(P_CHOICES) - 1) if best is None else (best[1], best[2])


def draw_problem(g, n_range=(384, 2048), k_range=(16, 236)):
    """Sizes (m / n in [1/2, 2]), spectrum (exponential, rate in [5, 100], or
    polynomial, alpha in [0.5, 3]) and k (log-uniform in [16, 236], so that k + 20
    fits the widest sketch of 256 columns, and k + 20 <= min(m, n) / 2)
    with the optimal rank-k tail at 0.3-30 % of ||A||_F."""
    while True:
        n = int(math.exp(g.uniform(math.log(n_range[0]), math.log(n_range[1]))))
        m = int(n * math.exp(g.uniform(math.log(0.5), math.log(2.0))))
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


def build_dataset(count, seed, device, log_every=500, n_range=(384, 2048)):
    """Probe features (12 statistics; the 13th input is added per request),
    error tables, k and sizes for ``count`` generated matrices."""
    import torch
    g = inputs.rng(seed)
    feats, ks, tabs, meta = [], [], [], []
    t0 = time.time()
    for i in range(count):
        m, n, k, sig, kind = draw_problem(g, n_range=n_range)
        A = make_matrix(m, n, sig, seed * 1000003 + i, device)
        Om = torch.from_numpy(inputs.omega(m, k + 20, seed=seed * 7919 + i)).to(device)
        tail2 = float((sig[k:] ** 2).sum())
        tabs.append(eps_table(A, Om, k, tail2))
        f, _ = rqlp.probe_features(A, k, Om, TARGET, precision=rqlp.PREC_BF16X3)
        feats.append(f.cpu().numpy().astype(np.float64)[:12])
        ks.append(k)
        meta.append((m, n, k, kind))
        if log_every and (i + 1) % log_every == 0:
            print(f"  {i + 1}/{count} matrices, {time.time() - t0:.0f} s", flush=True)
    return np.array(feats), np.array(ks), np.array(tabs), np.array(meta, dtype=object)


def rows(feats, ks, tabs, targets, margin=LABEL_MARGIN):
    """Training rows: for matrix i and request t, features + log10 t and the
    label for t / margin."""
    X, yq, yp, idx, ts = [], [], [], [], []
    for i in range(len(ks)):
        for t in targets[i]:
            X.append(np.concatenate([feats[i], [math.log10(t)]]))
            a, b = label_from_table(tabs[i], ks[i], t / margin)
            yq.append(a)
            yp.append(b)
            idx.append(i)
            ts.append(t)
    return np.array(X), np.array(yq, np.int32), np.array(yp, np.int32), np.array(idx), np.array(ts)


def draw_targets(count, per, seed):
    g = inputs.rng(seed)
    lo, hi = (math.log(v) for v in TARGET_RANGE)
    return [np.exp(g.uniform(lo, hi, per)) for _ in range(count)]


def init_params(seed, F=rqlp.MLP_FEATURES, H=rqlp.MLP_HIDDEN):
    g = inputs.rng(seed)
    W1 = g.standard_normal((F, H)) * math.sqrt(2.0 / F)
    W2 = g.standard_normal((H, H)) * math.sqrt(2.0 / H)
    W3 = g.standard_normal((H, 8)) * math.sqrt(1.0 / H)
    return np.concatenate([W1.ravel(), np.zeros(H), W2.ravel(), np.zeros(H), W3.ravel(), np.zeros(8)])


def train(X, yq, yp, steps=3000, lr=3e-3, seed=11, device="cuda", val=None, every=50, init=None):
    """Full-batch Adam with the library's kernels. With val = (Xv, yqv, ypv),
    the parameters of the lowest validation loss (checked every ``every``
    steps) are returned. init: parameters to start from (on standardised
    features, see unfold_standardisation); Adam's moments start at zero.
    Returns (params, curve of (step, loss, val_loss))."""
    import torch
    dev = torch.device(device)

    def upload(Xa, qa, pa):
        B = Xa.shape[0]
        nb = rqlp.rqlp_mlp_workspace_bytes(B)
        return (B, torch.from_numpy(np.ascontiguousarray(Xa, dtype=np.float32)).to(dev),
                torch.from_numpy(np.ascontiguousarray(qa, dtype=np.int32)).to(dev),
                torch.from_numpy(np.ascontiguousarray(pa, dtype=np.int32)).to(dev),
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
    tr = upload(X, yq, yp)
    va = upload(*val) if val is not None else None
    st = torch.cuda.current_stream().cuda_stream

    def grad_of(data, g, lo):
        B, Xd, qd, pd, ws, nb = data
        s = rqlp.rqlp_mlp_grad(prm.data_ptr(), Xd.data_ptr(), qd.data_ptr(), pd.data_ptr(), B, g.data_ptr(),
                               lo.data_ptr(), ws.data_ptr(), nb, st)
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


def predict_logits(params, X):
    """Logits on the device with rqlp_mlp_forward."""
    import torch
    dev = torch.device("cuda")
    prm = torch.from_numpy(params.astype(np.float32)).to(dev)
    Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to(dev)
    out = torch.empty(X.shape[0], 8, device=dev)
    s = rqlp.rqlp_mlp_forward(prm.data_ptr(), Xd.data_ptr(), X.shape[0], out.data_ptr(),
                              torch.cuda.current_stream().cuda_stream)
    if s != 0:
        raise rqlp.RqlpError(s, "rqlp_mlp_forward")
    return out.cpu().numpy()


def choose(logits):
    return logits[:, :5].argmax(axis=1), logits[:, 5:].argmax(axis=1)


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
    out = []
    for t in targets:
        X = np.concatenate([feats, np.full((len(ks), 1), math.log10(t))], axis=1)
        qi, pi = choose(predict_logits(params, X))
        out.append(evaluate_at(qi, pi, tabs, ks, t))
    return out


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
    ap.add_argument("--per", type=int, default=5, help="requests per training matrix")
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--out", default="learn_out")
    ap.add_argument("--data", default=None, help="reuse a qp_dataset.npz instead of generating one")
    ap.add_argument("--large", type=int, default=0,
                    help="add this many training matrices with n in [2048, 8192] (and a fifth as many to test)")
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
        big = (2048, 8192)
        f2, k2, t2, _ = build_dataset(a.large, seed=601, device="cuda", log_every=50, n_range=big)
        f3, k3, t3, _ = build_dataset(max(1, a.large // 5), seed=919, device="cuda", log_every=50, n_range=big)
        # interleave so that the validation slice (the first tenth) holds both sizes
        order = np.random.default_rng(5).permutation(len(ktr) + len(k2))
        ftr, ktr, tabtr = (np.concatenate([x, y])[order] for x, y in ((ftr, f2), (ktr, k2), (tabtr, t2)))
        fte, kte, tabte = (np.concatenate([x, y]) for x, y in ((fte, f3), (kte, k3), (tabte, t3)))
    t_data = time.time() - t0
    # 10 % of the training matrices (all their requests) validate the early stop
    nv = max(1, len(ktr) // 10)
    tg = draw_targets(len(ktr), a.per, seed=77)
    Xtr, yqtr, yptr, _, _ = rows(ftr[nv:], ktr[nv:], tabtr[nv:], tg[nv:])
    Xva, yqva, ypva, _, _ = rows(ftr[:nv], ktr[:nv], tabtr[:nv], tg[:nv])
    mu = Xtr.mean(axis=0)
    sd = Xtr.std(axis=0)
    sd[sd < 1e-6] = 1.0
    t1 = time.time()
    init = unfold_standardisation(load_weights(a.resume), mu, sd) if a.resume else None
    params, curve = train((Xtr - mu) / sd, yqtr, yptr, steps=a.steps, lr=a.lr,
                          val=((Xva - mu) / sd, yqva, ypva), init=init)
    t_train = time.time() - t1
    params = fold_standardisation(params, mu, sd)
    ev = evaluate(params, fte, tabte, kte)
    report = {"train_matrices": int(len(ktr)), "train_rows": int(len(yqtr)), "val_rows": int(len(yqva)),
              "label_margin": LABEL_MARGIN,
              "test_matrices": int(len(kte)), "steps": a.steps, "lr": a.lr, "target_range": TARGET_RANGE,
              "seconds_data": t_data, "seconds_train": t_train, "curve": curve,
              "label_hist_q": np.bincount(yqtr, minlength=5).tolist(),
              "label_hist_p": np.bincount(yptr, minlength=3).tolist(), "test": ev}
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
