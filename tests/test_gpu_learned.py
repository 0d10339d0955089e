"""GPU parity of the learned (q, p) predictor.

* MLP kernels (forward, mean-squared-error gradient, Adam) against the FP64
  reference on the same FP32 parameters, features and targets. A ReLU mask is an FP decision: samples whose
  FP64 pre-activations come within 1e-4 of zero are dropped so that both sides
  take the same branch.
* Probe features against the FP64 reference computed from the R-diagonal of a
  Householder QR of the same probe sketch A^T Omega_w (w = k + 20).
* The learned factorisation against the oracle run with the same (q, p) and
  the first k + p columns of Omega, for every p width and q from 0 to 4
  (forced through the output bias), and with a random network whose pick is
  checked against the FP64 selection rule.
"""
import ctypes
import os

import numpy as np
import pytest

from oracle import mlp_oracle as mo
from oracle import rqlp_oracle as orc
from paper_2110_01011_gb300 import inputs
from parity_util import compare

pytestmark = pytest.mark.gpu

F, H = mo.N_FEATURES, mo.HIDDEN


def _theta(seed, scale=0.3):
    return (inputs.rng(seed).standard_normal(mo.n_params()) * scale).astype(np.float32).astype(np.float64)


def _features(seed, B):
    return inputs.rng(seed).standard_normal((B, F)).astype(np.float32).astype(np.float64)


def _safe_rows(theta, X, margin=1e-4):
    _, (_, z1, _, z2, _) = mo.forward(theta, X)
    ok = (np.abs(z1).min(axis=1) > margin) & (np.abs(z2).min(axis=1) > margin)
    return X[ok]


def _dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    return (t.to(dtype) if dtype is not None else t).cuda()


def _st():
    import torch
    return torch.cuda.current_stream().cuda_stream


def test_mlp_params_count():
    from paper_2110_01011_gb300 import rqlp
    assert rqlp.MLP_PARAMS == mo.n_params()
    assert (rqlp.MLP_FEATURES, rqlp.MLP_HIDDEN, rqlp.MLP_OUTPUTS) == (F, H, mo.N_OUT)


@pytest.mark.parametrize("B", [1, 37, 1300])
def test_mlp_forward(B):
    import torch

    from paper_2110_01011_gb300 import rqlp
    theta = _theta(5 + B)
    X = _features(9 + B, B)
    ref, _ = mo.forward(theta, X)
    out = torch.empty(B, mo.N_OUT, device="cuda")
    dt, dX = _dev(theta, torch.float32), _dev(X, torch.float32)   # kept alive across the launch
    st = rqlp.rqlp_mlp_forward(dt.data_ptr(), dX.data_ptr(), B, out.data_ptr(), _st())
    assert st == 0
    got = out.double().cpu().numpy()
    # dot products of <= 64 FP32 terms: error well below 1e-5 of the magnitude
    assert np.abs(got - ref).max() <= 1e-5 * (1.0 + np.abs(ref).max())


@pytest.mark.parametrize("B", [1, 64, 500])
def test_mlp_grad(B):
    import torch

    from paper_2110_01011_gb300 import rqlp
    theta = _theta(100 + B)
    X = _safe_rows(theta, _features(200 + B, B + 40))[:B]
    B = X.shape[0]
    Y = inputs.rng(300 + B).uniform(-4, 1, (B, mo.N_OUT)).astype(np.float32).astype(np.float64)
    loss_ref, grad_ref = mo.loss_and_grads(theta, X, Y)
    nb = rqlp.rqlp_mlp_workspace_bytes(B)
    ws = torch.empty(nb // 4 + 1, device="cuda")
    grad = torch.empty(mo.n_params(), device="cuda")
    loss = torch.empty(1, device="cuda")
    dt, dX, dY = _dev(theta, torch.float32), _dev(X, torch.float32), _dev(Y, torch.float32)
    st = rqlp.rqlp_mlp_grad(dt.data_ptr(), dX.data_ptr(), dY.data_ptr(), B, grad.data_ptr(), loss.data_ptr(),
                            ws.data_ptr(), nb, _st())
    assert st == 0
    gg = grad.double().cpu().numpy()
    # sums over the batch of FP32 products: relative 1e-4 of the largest entry
    assert np.abs(gg - grad_ref).max() <= 1e-4 * np.abs(grad_ref).max() + 1e-7
    assert abs(float(loss.item()) - loss_ref) <= 1e-5 * abs(loss_ref) + 1e-6


def test_mlp_grad_workspace_too_small():
    import torch

    from paper_2110_01011_gb300 import rqlp
    B = 10
    nb = rqlp.rqlp_mlp_workspace_bytes(B)
    ws = torch.empty(nb // 4, device="cuda")
    z = torch.zeros(mo.n_params(), device="cuda")
    X = torch.zeros(B, F, device="cuda")
    Y = torch.zeros(B, mo.N_OUT, device="cuda")
    st = rqlp.rqlp_mlp_grad(z.data_ptr(), X.data_ptr(), Y.data_ptr(), B, z.data_ptr(), None, ws.data_ptr(), nb - 4,
                            _st())
    assert st == 6   # RQLP_ERR_WORKSPACE


@pytest.mark.parametrize("step", [1, 7, 1000])
def test_mlp_adam(step):
    """Same FP32 inputs (hyper-parameters included); the moments are compared
    at 3 roundings of their terms, the update at 1e-5 relative plus one FP32
    rounding of theta."""
    import torch

    from paper_2110_01011_gb300 import rqlp
    n = mo.n_params()
    g = inputs.rng(step)
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    theta = f32(g.standard_normal(n))
    grad = f32(g.standard_normal(n))
    m1 = f32(g.standard_normal(n) * 0.1)
    m2 = f32(np.abs(g.standard_normal(n)) * 0.01)
    lr, b1, b2, eps = (float(np.float32(v)) for v in (1e-3, 0.9, 0.999, 1e-8))
    t_ref, m1_ref, m2_ref = mo.adam(theta, grad, m1, m2, step, lr, b1, b2, eps)
    dt, dm1, dm2 = _dev(theta, torch.float32), _dev(m1, torch.float32), _dev(m2, torch.float32)
    dg = _dev(grad, torch.float32)
    st = rqlp.rqlp_mlp_adam(dt.data_ptr(), dg.data_ptr(), dm1.data_ptr(), dm2.data_ptr(), n, lr, b1, b2, eps, step,
                            _st())
    assert st == 0
    u = 2.0 ** -24
    assert (np.abs(dm1.double().cpu().numpy() - m1_ref) <= 3 * u * (b1 * np.abs(m1) + (1 - b1) * np.abs(grad))).all()
    assert (np.abs(dm2.double().cpu().numpy() - m2_ref) <= 3 * u * (b2 * m2 + (1 - b2) * grad ** 2) + 1e-30).all()
    upd, upd_ref = dt.double().cpu().numpy() - theta, t_ref - theta
    assert (np.abs(upd - upd_ref) <= 1e-5 * np.abs(upd_ref) + 2.0 ** -23 * np.abs(theta) + 1e-12).all()


def _probe_problem(m, n, k, rate, seed):
    sig = inputs.exp_spectrum(min(m, n), rate=rate)
    A = inputs.low_rank_matrix(m, n, sig, 1e-4, seed=seed)
    Om = inputs.omega(m, k + 20, seed=seed + 1)
    return A, Om


def _oracle_features(A, Om, k):
    Y = np.asarray(A, np.float64).T @ np.asarray(Om, np.float64)
    _, R = orc.householder_qr(Y)
    return mo.probe_features(np.diag(R), k, *A.shape), np.diag(R)


@pytest.mark.parametrize("m,n,k,rate", [(700, 500, 20, 25.0), (333, 900, 7, 12.0), (1200, 1200, 60, 60.0),
                                        (260, 300, 1, 10.0), (700, 500, 20, 8.0), (333, 900, 7, 5.0)])
@pytest.mark.parametrize("prec", [0, 1], ids=["fp32", "bf16x3"])
def test_probe_features(m, n, k, rate, prec):
    """The device R-diagonal comes from one CholeskyQR (FP32 Cholesky of the
    Gram), whose relative error grows like u * kappa(Y)^2 with u = 2^-24 and
    kappa(Y) >= r_1 / r_w; the log10 features are compared at
    1e-4 + 40 u (r_1 / r_w)^2 (about 1e-4 for the mild spectra, 2e-3 to 2e-2
    for the two steep ones)."""
    from paper_2110_01011_gb300 import rqlp
    A, Om = _probe_problem(m, n, k, rate, seed=m + n + k)
    ref, r = _oracle_features(A, Om, k)
    kappa = r[0] / r[-1]
    tol = 1e-4 + 40 * 2.0 ** -24 * kappa ** 2
    dA, dO = _dev(A), _dev(Om)
    feat, info = rqlp.probe_features(dA, k, dO, precision=prec)
    got = feat.double().cpu().numpy()
    assert int(info[0].item()) == 0
    np.testing.assert_allclose(got[:9], ref[:9], atol=tol, rtol=0)
    np.testing.assert_allclose(got[9:], ref[9:], rtol=1e-6, atol=1e-7)


def _forced_params(qi, pi):
    """Zero weights, output biases +5 (error 1e5: never feasible) except pair
    (qi, pi) at -5: the only pair within any request."""
    theta = np.zeros(mo.n_params())
    b3 = mo.n_params() - 1 - mo.N_OUT
    theta[b3:b3 + mo.N_OUT] = 5.0
    theta[b3 + 3 * qi + pi] = -5.0
    return theta.astype(np.float32)


def _learned(A, Om, k, theta, prec):
    import torch

    from paper_2110_01011_gb300 import rqlp
    dA, dO, dt = _dev(A), _dev(Om), _dev(theta, torch.float32)
    Q, L, P, info, diag, qp = rqlp.factor_learned(dA, k, dO, dt, 1e-2, precision=prec)
    torch.cuda.synchronize()
    gpu = (Q.double().cpu().numpy(), L.double().cpu().numpy(), P.double().cpu().numpy(), info.cpu().numpy(),
           diag.cpu().numpy())
    return gpu, qp


@pytest.mark.parametrize("qi,pi", [(0, 0), (1, 1), (4, 2), (2, 0), (3, 2)])
@pytest.mark.parametrize("prec", [0, 1], ids=["fp32", "bf16x3"])
def test_factor_learned_forced(qi, pi, prec):
    m, n, k = 900, 640, 24
    A, Om = _probe_problem(m, n, k, 20.0, seed=4242)
    gpu, qp = _learned(A, Om, k, _forced_params(qi, pi), prec)
    q, p = mo.Q_CHOICES[qi], mo.P_CHOICES[pi]
    assert qp == (q, p)
    compare(A, Om[:, :k + p], k, p, q, gpu, elem_atol=5e-4, precision=prec)


def test_factor_learned_random_net():
    """The device's pick equals the FP64 selection of the same network on the
    device's features (estimates at least 1e-3 from the request's boundary),
    and the chain runs that (q, p)."""
    m, n, k = 800, 800, 30
    A, Om = _probe_problem(m, n, k, 30.0, seed=777)
    dA, dO = _dev(A), _dev(Om)
    from paper_2110_01011_gb300 import rqlp
    feat, _ = rqlp.probe_features(dA, k, dO, precision=1)
    f = feat.double().cpu().numpy()[None, :]
    lt = np.log10(1e-2)
    for seed in range(200):
        theta = _theta(9000 + seed, scale=0.5)
        theta[-1] = 0.1
        theta = theta.astype(np.float32)
        est, _ = mo.forward(theta.astype(np.float64), f)
        qi, pi = mo.choose(est[0], k, 1e-2, float(theta[-1]))
        if np.abs(est[0] + float(theta[-1]) - lt).min() > 1e-3 and (qi, pi) != (4, 2):
            break
    want = (mo.Q_CHOICES[qi], mo.P_CHOICES[pi])
    gpu, qp = _learned(A, Om, k, theta, 1)
    assert qp == want
    compare(A, Om[:, :k + want[1]], k, want[1], want[0], gpu, elem_atol=5e-4, precision=1)


def test_predict_qp_matches_factor_learned():
    import torch

    from paper_2110_01011_gb300 import rqlp
    m, n, k = 500, 450, 16
    A, Om = _probe_problem(m, n, k, 15.0, seed=31)
    theta = _forced_params(3, 1)
    dA, dO, dP = _dev(A), _dev(Om), _dev(theta)
    nb = rqlp.rqlp_learned_workspace_bytes(m, n, k, rqlp._opts(1))
    buf, ws = rqlp._workspace(nb, dA.device)
    qp = torch.empty(2, dtype=torch.int32, device="cuda")
    info = torch.empty(2, dtype=torch.int32, device="cuda")
    st = rqlp.rqlp_predict_qp(dA.data_ptr(), m, n, n, k, dO.data_ptr(), k + 20, 1e-2, dP.data_ptr(), qp.data_ptr(),
                              ws, nb, info.data_ptr(), rqlp._opts(1), _st())
    assert st == 0
    assert tuple(qp.cpu().tolist()) == (3, 10)


def test_learned_argument_errors():
    import torch

    from paper_2110_01011_gb300 import rqlp
    assert rqlp.rqlp_learned_workspace_bytes(100, 30, 20) == 0      # k + 20 > min(m, n)
    assert rqlp.rqlp_learned_workspace_bytes(100, 100, 0) == 0
    A = torch.zeros(100, 30, device="cuda")
    Om = torch.zeros(100, 40, device="cuda")
    with pytest.raises(rqlp.RqlpError):
        rqlp.probe_features(A, 20, Om)
    A = torch.zeros(100, 60, device="cuda")
    prm = torch.zeros(mo.n_params(), device="cuda")
    for bad in (0.0, -1e-3, 1.0, float("nan")):
        with pytest.raises(rqlp.RqlpError):
            rqlp.factor_learned(A, 20, Om, prm, bad)


def test_shipped_weights_load():
    """The trained weights shipped with the package have the layout the kernels read."""
    from paper_2110_01011_gb300 import learn
    if not os.path.exists(learn.WEIGHTS):
        pytest.skip("no trained weights in the package")
    w = learn.load_weights()
    assert w.shape == (mo.n_params(),) and np.isfinite(w).all()


def test_predict_fallback_on_nonfinite_logits():
    """A network whose estimates or margin are not finite falls back to
    (q, p) = (2, 10)."""
    import torch

    from paper_2110_01011_gb300 import rqlp
    m, n, k = 400, 300, 12
    A, Om = _probe_problem(m, n, k, 10.0, seed=5)
    for where in (-2, -1):          # the last output bias, then delta
        theta = _forced_params(4, 2)
        theta[where] = np.nan
        dA, dO, dP = _dev(A), _dev(Om), _dev(theta)
        nb = rqlp.rqlp_learned_workspace_bytes(m, n, k, rqlp._opts(0))
        buf, ws = rqlp._workspace(nb, dA.device)
        qp = torch.empty(2, dtype=torch.int32, device="cuda")
        info = torch.empty(2, dtype=torch.int32, device="cuda")
        st = rqlp.rqlp_predict_qp(dA.data_ptr(), m, n, n, k, dO.data_ptr(), k + 20, 1e-2, dP.data_ptr(),
                                  qp.data_ptr(), ws, nb, info.data_ptr(), rqlp._opts(0), _st())
        assert st == 0
        assert tuple(qp.cpu().tolist()) == (2, 10)


def test_label_table_matches_oracle():
    """The training labeller's 15 excess errors (one width-(k+20) chain, all
    (q, p) from leading blocks) against the oracle run separately for each
    (q, p) with Omega's first k + p columns."""
    import torch

    from paper_2110_01011_gb300 import learn
    m, n, k = 300, 220, 12
    sig = inputs.poly_spectrum(n, 1.0)
    A = inputs.low_rank_matrix(m, n, sig, 0.0, seed=12)
    Om = inputs.omega(m, k + 20, seed=13)
    tail2 = float((sig[k:] ** 2).sum())
    dA, dO = _dev(A), _dev(Om)
    tab = learn.eps_table(dA, dO, k, tail2)
    A64 = np.asarray(A, np.float64)
    for qi, q in enumerate(mo.Q_CHOICES):
        for pi, p in enumerate(mo.P_CHOICES):
            Q, L, P = orc.rand_qlp(A64, np.asarray(Om[:, :k + p], np.float64), q)
            ref = orc.rank_r_error_fro(A64, Q, L, P, k) / np.sqrt(tail2) - 1.0
            assert abs(tab[qi, pi] - ref) <= 1e-4 + 1e-3 * abs(ref), (q, p, tab[qi, pi], ref)


@pytest.mark.parametrize("m,n,k", [(900, 640, 24), (5000, 3000, 40)])
@pytest.mark.parametrize("prec", [0, 1], ids=["fp32", "bf16x3"])
def test_factor_learned_host_overlapped_ingest(m, n, k, prec):
    """The host-buffer learned entry (row blocks of A copied on the library's
    streams, the probe sketch started per landed block) picks the same
    (q, p) as the device-buffer entry and matches the oracle at it."""
    import torch

    from paper_2110_01011_gb300 import rqlp
    A, Om = _probe_problem(m, n, k, 20.0, seed=m + k)
    theta = _forced_params(2, 1)
    dt = _dev(theta, torch.float32)
    hA = torch.from_numpy(A).pin_memory()
    hO = torch.from_numpy(Om).pin_memory()
    Q, L, P, info, diag, qp = rqlp.factor_learned_host(hA, k, hO, dt, 1e-2, precision=prec)
    assert qp == (2, 10) and int(info[0]) == 0
    gpu = (Q.double().numpy(), L.double().numpy(), P.double().numpy(), info.numpy(), diag.numpy())
    compare(A, Om[:, :k + 10], k, 10, 2, gpu, elem_atol=5e-4, precision=prec)
    dgpu, dqp = _learned(A, Om, k, theta, prec)
    assert dqp == qp
    assert np.max(np.abs(gpu[1] - dgpu[1])) <= 1e-5 * np.abs(dgpu[1]).max()
