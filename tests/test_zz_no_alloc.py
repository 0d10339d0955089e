"""rqlp_factor_noalloc: the factorisation for callers that cannot allocate
device memory (a framework or host application whose pool owns all device
memory, a fixed device-memory budget, or a path where cudaMalloc's implicit
synchronisation is not acceptable). Its scratch is a library-owned array in
device memory, so it takes no workspace argument.

The GPU test calls it twice in a row through the C ABI, on two different
problems, and checks each result against rqlp_factor's on the same inputs
within the parity tolerances of the other tests. The file sorts last so a
run that stops at the first failure has run every other test before it.
"""
import numpy as np
import pytest

from paper_2110_01011_gb300 import inputs, rqlp
from parity_util import TOL_LII

ELEM_TOL = 2e-4   # max |difference| of Q, L, P entries, as in the parity tests


def _problem(m, n, k, p, seed):
    A = inputs.low_rank_matrix(m, n, inputs.exp_spectrum(min(m, n), 8.0), 1e-5, seed=seed)
    Om = inputs.omega(m, k + p, seed=seed + 1)
    return A, Om


def _noalloc(dA, dO, k, p, q):
    import torch
    m, n = dA.shape
    d = k + p
    dev = dA.device
    Q = torch.empty(m, d, device=dev)
    L = torch.empty(d, d, device=dev)
    P = torch.empty(n, d, device=dev)
    info = torch.full((2,), -1, dtype=torch.int32, device=dev)
    diag = torch.empty(4, dtype=torch.float64, device=dev)
    st = rqlp.rqlp_factor_noalloc(dA.data_ptr(), m, n, dA.stride(0), k, p, q, dO.data_ptr(),
                                  dO.stride(0), Q.data_ptr(), Q.stride(0), L.data_ptr(), L.stride(0),
                                  P.data_ptr(), P.stride(0), info.data_ptr(), diag.data_ptr(),
                                  rqlp.rqlp_default_opts(), torch.cuda.current_stream().cuda_stream)
    assert st == 0, rqlp.rqlp_status_string(st)
    return Q, L, P, info


@pytest.mark.gpu
def test_noalloc_matches_rqlp_factor_twice_in_a_row():
    import torch
    cases = [(1000, 1000, 20, 5, 1, 11), (700, 500, 12, 4, 2, 23)]
    for (m, n, k, p, q, seed) in cases:
        A, Om = _problem(m, n, k, p, seed)
        dA = torch.from_numpy(A).cuda()
        dO = torch.from_numpy(Om).cuda()
        Qn, Ln, Pn, info_n = _noalloc(dA, dO, k, p, q)
        torch.cuda.synchronize()
        Qn, Ln, Pn = (x.double().cpu().numpy() for x in (Qn, Ln, Pn))
        Qr, Lr, Pr, info_r, _ = rqlp.factor(dA, k, p, q, dO)
        torch.cuda.synchronize()
        Qr, Lr, Pr = (x.double().cpu().numpy() for x in (Qr, Lr, Pr))
        assert int(info_n[0]) == 0 and int(info_r[0]) == 0
        assert np.max(np.abs(Qn - Qr)) <= ELEM_TOL
        assert np.max(np.abs(Pn - Pr)) <= ELEM_TOL
        assert np.max(np.abs(Ln - Lr)) <= ELEM_TOL * np.abs(Lr).max()
        assert np.max(np.abs(np.diag(Ln) - np.diag(Lr)) / np.diag(Lr)) <= TOL_LII


def test_noalloc_rejects_oversize_before_any_work():
    """A problem whose workspace exceeds the library's array is refused with
    RQLP_ERR_WORKSPACE before anything touches the (fake) pointers."""
    m, n, k, p, q = 8192, 8192, 200, 10, 2
    assert rqlp.rqlp_workspace_bytes(m, n, k, p, q) > rqlp.NOALLOC_SCRATCH_BYTES
    fake = 0x1000
    st = rqlp.rqlp_factor_noalloc(fake, m, n, n, k, p, q, fake, k + p, fake, k + p, fake, k + p,
                                  fake, k + p, fake, None, rqlp.rqlp_default_opts(), None)
    assert st == 6
    assert rqlp.rqlp_factor_noalloc(fake, 10, 10, 10, 0, 1, 0, fake, 1, fake, 1, fake, 1, fake, 1,
                                    fake, None, None, None) == 1
