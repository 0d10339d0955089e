"""Bounds checks without a sanitizer: rqlp_factor's outputs get leading
dimensions wider than d and extra rows, the workspace gets bytes on both
sides of the range it is given, all filled with canaries; after the call
every canary is intact, the inputs are unchanged and the factors' entries
are written. Both arithmetic forms, shapes with ragged tiles."""
import numpy as np
import pytest

from paper_2110_01011_gb300 import inputs, rqlp

pytestmark = pytest.mark.gpu

CANARY = 1234.5
BYTE = 0xA5


@pytest.mark.parametrize("prec", [rqlp.PREC_FP32, rqlp.PREC_BF16X3], ids=["fp32", "bf16x3"])
@pytest.mark.parametrize("m,n,k,p,q", [(300, 200, 20, 5, 1), (257, 131, 10, 3, 2), (131, 257, 12, 4, 0)])
def test_outputs_and_workspace_stay_in_bounds(m, n, k, p, q, prec):
    import torch
    d = k + p
    A = torch.from_numpy(inputs.low_rank_matrix(m, n, inputs.exp_spectrum(min(m, n), 8.0), 1e-5,
                                                seed=m + n)).cuda()
    Om = torch.from_numpy(inputs.omega(m, d, seed=m * 3 + n)).cuda()
    A0, Om0 = A.clone(), Om.clone()
    ldq, ldl, ldp = d + 7, d + 3, d + 5
    Qb = torch.full((m + 2, ldq), CANARY, device="cuda")
    Lb = torch.full((d + 2, ldl), CANARY, device="cuda")
    Pb = torch.full((n + 2, ldp), CANARY, device="cuda")
    opts = rqlp._opts(prec)
    nb = rqlp.rqlp_workspace_bytes(m, n, k, p, q, opts)
    assert nb > 0
    pad = 4096
    ws = torch.full((pad + nb + pad,), BYTE, dtype=torch.uint8, device="cuda")
    base = (ws.data_ptr() + pad + 255) // 256 * 256
    off = base - ws.data_ptr()
    info = torch.zeros(2, dtype=torch.int32, device="cuda")
    diag = torch.zeros(4, dtype=torch.float64, device="cuda")
    st = rqlp.rqlp_factor(A.data_ptr(), m, n, A.stride(0), k, p, q, Om.data_ptr(), Om.stride(0),
                          Qb.data_ptr(), ldq, Lb.data_ptr(), ldl, Pb.data_ptr(), ldp, base, nb,
                          info.data_ptr(), diag.data_ptr(), opts, rqlp._stream())
    assert st == 0
    torch.cuda.synchronize()
    assert int(info[0].item()) == 0
    assert torch.equal(A, A0) and torch.equal(Om, Om0)
    for X, rows, name in ((Qb, m, "Q"), (Lb, d, "L"), (Pb, n, "P")):
        X = X.cpu().numpy()
        assert np.all(X[:rows, d:] == CANARY), f"{name}: columns past d written"
        assert np.all(X[rows:, :] == CANARY), f"{name}: rows past the matrix written"
        assert np.isfinite(X[:rows, :d]).all() and not np.any(X[:rows, :d] == CANARY), f"{name}: not written"
    w = ws.cpu().numpy()
    assert np.all(w[:off] == BYTE), "bytes before the workspace written"
    assert np.all(w[off + nb:] == BYTE), "bytes past the workspace written"
