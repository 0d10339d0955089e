"""GPU parity at the full benchmark sizes and on the E3 test spectra.

Full size: the 20000 x 20000 workload (sigma_i = exp(-i/50), rank 1000, noise
floor 1e-6; k = 200, p = 10, q = 2) and its rectangular variants 40000 x 10000
and 10000 x 40000, factored through the same entry point and launch
configuration the benchmark times, against the FP64 oracle run on the host on
the same A and Omega (about 1e12 flops per chain). Both arithmetic forms are
compared with the chain tolerances; the learned form is compared with the
oracle run at the (q, p) it picked.
"""
import numpy as np
import pytest

from paper_2110_01011_gb300 import inputs
from parity_util import compare

pytestmark = pytest.mark.gpu

K, P, Q = 200, 10, 2


def _workload(m, n):
    import torch
    sig = inputs.exp_spectrum(1000, 50.0)
    A = inputs.low_rank_matrix_torch(m, n, sig, 1e-6, seed=1002, rank=1000, device="cuda")
    Om = inputs.omega_torch(m, K + 20, seed=2002, device="cuda", bf16_exact=True)   # as the bench
    torch.cuda.synchronize()
    return A, Om


def _gpu(A, Om, k, p, q, prec):
    import torch

    from paper_2110_01011_gb300 import rqlp
    Qg, Lg, Pg, info, diag = rqlp.factor(A, k, p, q, Om[:, :k + p], precision=prec)
    torch.cuda.synchronize()
    out = (Qg.double().cpu().numpy(), Lg.double().cpu().numpy(), Pg.double().cpu().numpy(), info.cpu().numpy(),
           diag.cpu().numpy())
    del Qg, Lg, Pg
    return out


@pytest.mark.slow
@pytest.mark.parametrize("m,n", [(20000, 20000), (40000, 10000), (10000, 40000)],
                         ids=["20000x20000", "40000x10000", "10000x40000"])
def test_full_size_both_forms(m, n):
    from paper_2110_01011_gb300 import rqlp
    A, Om = _workload(m, n)
    runs = {prec: _gpu(A, Om, K, P, Q, prec) for prec in (rqlp.PREC_FP32, rqlp.PREC_BF16X3)}
    A64 = A.double().cpu().numpy()
    Om64 = Om[:, :K + P].double().cpu().numpy()
    del A, Om
    for prec, out in runs.items():
        err = compare(A64, Om64, K, P, Q, out, elem_atol=2e-4, precision=prec)
        print(m, n, ["fp32", "bf16x3"][prec], {k: float(v) for k, v in err.items()})


@pytest.mark.slow
def test_full_size_learned():
    import torch

    from paper_2110_01011_gb300 import learn, rqlp
    A, Om = _workload(20000, 20000)
    prm = torch.from_numpy(learn.load_weights()).cuda()
    Qg, Lg, Pg, info, diag, (q, p) = rqlp.factor_learned(A, K, Om, prm, 0.02, precision=rqlp.PREC_BF16X3)
    torch.cuda.synchronize()
    out = (Qg.double().cpu().numpy(), Lg.double().cpu().numpy(), Pg.double().cpu().numpy(), info.cpu().numpy(),
           diag.cpu().numpy())
    A64 = A.double().cpu().numpy()
    Om64 = Om[:, :K + p].double().cpu().numpy()
    err = compare(A64, Om64, K, p, q, out, elem_atol=2e-4, precision=rqlp.PREC_BF16X3)
    print("learned", (q, p), {k: float(v) for k, v in err.items()})


@pytest.mark.parametrize("family,noise", [("plus_noise", 1e-3), ("fast", 0.0), ("s_shaped", 0.0), ("slow", 0.0)])
@pytest.mark.parametrize("prec", [0, 1], ids=["fp32", "bf16x3"])
def test_e3_spectra(family, noise, prec):
    """The four singular-value families of section 5.2 on 1000 x 1000, k = 20,
    p = 5, q = 1."""
    from parity_util import run_gpu
    n = 1000
    A = inputs.low_rank_matrix(n, n, inputs.e3_spectrum(family, n, 200), noise, seed=3001)
    Om = inputs.omega(n, 25, seed=3002)
    compare(A, Om, 20, 5, 1, run_gpu(A, Om, 20, 5, 1, precision=prec), precision=prec)


@pytest.mark.slow
@pytest.mark.parametrize("kind,par,k,p,q", [("exp", 100.0, 12, 5, 2), ("poly", 1.76, 41, 5, 1)],
                         ids=["exp-ratio100-k12-q2", "poly1.76-k41-q1"])
def test_two_parts_at_large_size(kind, par, k, p, q):
    """Above m n = 2^27 the split form takes two BF16 parts: 16384^2 with a
    steep leading block (sigma_1 / sigma_k = 100, or the polynomial decay on
    which two parts missed at 705 x 1798) meets the plain tolerances."""
    import torch

    from paper_2110_01011_gb300 import rqlp
    n = 16384
    r = 1000
    sig = (np.exp(-np.arange(r) * np.log(par) / (k - 1)) if kind == "exp"
           else np.arange(1, r + 1, dtype=np.float64) ** (-par))
    A = inputs.low_rank_matrix_torch(n, n, sig, 1e-6, seed=9100 + k, rank=r, device="cuda")
    Om = inputs.omega_torch(n, k + p, seed=9200 + k, device="cuda")
    torch.cuda.synchronize()
    out = _gpu(A, Om, k, p, q, rqlp.PREC_BF16X3)
    A64, Om64 = A.double().cpu().numpy(), Om.double().cpu().numpy()
    del A, Om
    err = compare(A64, Om64, k, p, q, out, elem_atol=2e-4, precision=rqlp.PREC_BF16X3)
    print(kind, par, {kk: float(v) for kk, v in err.items()})
