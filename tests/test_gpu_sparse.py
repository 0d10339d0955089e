"""Rand-QLP of sparse A (CSR) on the device against the FP64 oracle run on the
densified matrix: seeded stand-ins with the sizes of the sparse test
matrices of section 5.1 (Table 1), whose data is not available here."""
import numpy as np
import pytest

from paper_2110_01011_gb300 import inputs
from parity_util import compare

pytestmark = pytest.mark.gpu


def _sparse(m, n, seed):
    import torch
    rp, ci, v = inputs.sparse_matrix(m, n, seed)
    dev = [torch.from_numpy(x).cuda() for x in (rp, ci, v)]
    return (rp, ci, v), dev


@pytest.mark.parametrize("m,n,k,p,q", [(inputs.SPARSE_SIZES[0],) * 2 + (20, 5, 1),
                                       (inputs.SPARSE_SIZES[1],) * 2 + (30, 10, 1),
                                       (inputs.SPARSE_SIZES[2],) * 2 + (40, 10, 2),
                                       (inputs.SPARSE_SIZES[3],) * 2 + (25, 5, 0),
                                       (inputs.SPARSE_SIZES[4],) * 2 + (50, 10, 1),
                                       (3000, 1200, 32, 8, 1), (900, 2500, 16, 4, 2)])
def test_sparse_matches_oracle(m, n, k, p, q):
    import torch

    from paper_2110_01011_gb300 import rqlp
    (rp, ci, v), (drp, dci, dv) = _sparse(m, n, seed=m + 3 * n)
    Om = inputs.omega(m, k + p, seed=m + n)
    Q, L, P, info, diag = rqlp.factor_sparse(drp, dci, dv, m, n, k, p, q, torch.from_numpy(Om).cuda())
    torch.cuda.synchronize()
    A = inputs.csr_to_dense(m, n, rp, ci, v)
    gpu = (Q.double().cpu().numpy(), L.double().cpu().numpy(), P.double().cpu().numpy(), info.cpu().numpy(),
           diag.cpu().numpy())
    err = compare(A, Om, k, p, q, gpu, elem_atol=5e-4, precision=0)
    print(m, n, {kk: float(vv) for kk, vv in err.items()})


def test_sparse_deterministic_and_matches_dense_path():
    """Two calls agree bitwise; the dense FP32 path on the densified matrix
    gives the same factors to FP32 rounding."""
    import torch

    from paper_2110_01011_gb300 import rqlp
    m, n, k, p, q = 2000, 1500, 24, 8, 1
    (rp, ci, v), (drp, dci, dv) = _sparse(m, n, seed=99)
    dO = torch.from_numpy(inputs.omega(m, k + p, seed=98)).cuda()
    a = rqlp.factor_sparse(drp, dci, dv, m, n, k, p, q, dO)
    b = rqlp.factor_sparse(drp, dci, dv, m, n, k, p, q, dO)
    torch.cuda.synchronize()
    for x, y in zip(a[:3], b[:3]):
        assert torch.equal(x, y)
    dA = torch.from_numpy(inputs.csr_to_dense(m, n, rp, ci, v).astype(np.float32)).cuda()
    Qd, Ld, Pd, _, _ = rqlp.factor(dA, k, p, q, dO)
    torch.cuda.synchronize()
    assert float((a[1] - Ld).abs().max()) <= 1e-5 * float(Ld.abs().max())


def test_bad_column_index_reported_and_skipped():
    import torch

    from paper_2110_01011_gb300 import rqlp
    m, n, k, p = 600, 400, 10, 5
    (rp, ci, v), _ = _sparse(m, n, seed=7)
    ci = ci.copy()
    ci[17] = n + 5            # out of range: skipped by the kernels, reported
    drp, dci, dv = (torch.from_numpy(x).cuda() for x in (rp, ci, v))
    dO = torch.from_numpy(inputs.omega(m, k + p, seed=8)).cuda()
    Q, L, P, info, diag = rqlp.factor_sparse(drp, dci, dv, m, n, k, p, 0, dO)
    torch.cuda.synchronize()
    assert int(info[0]) == 1   # RQLP_ERR_ARG
