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
    """A and Omega on the device. Rank 64 with sigma_i = exp(-i / 8) and a
    1e-5 noise floor: the largest FP32 case is ~37000^2, whose full-rank Haar
    factors would take many minutes to draw on the host."""
    import torch
    A = inputs.low_rank_matrix_torch(m, n, inputs.exp_spectrum(64, 8.0), 1e-5, seed=seed, rank=64)
    Om = torch.from_numpy(inputs.omega(m, k + p, seed=seed + 1)).cuda()
    return A, Om


def _noalloc(dA, dO, k, p, q, precision=rqlp.PREC_FP32):
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
                                  rqlp.Opts(precision=precision), torch.cuda.current_stream().cuda_stream)
    assert st == 0, rqlp.rqlp_status_string(st)
    return Q, L, P, info


def _largest_square_within_bound(k, p, q, precision):
    """The largest n (multiple of 64) whose n x n problem fits the library's
    array: the bound is read from include/rqlp.h, not from a second copy."""
    o = rqlp.Opts(precision=precision)
    n = 64
    while rqlp.rqlp_workspace_bytes(n + 64, n + 64, k, p, q, o) <= rqlp.header_define("RQLP_NOALLOC_SCRATCH_BYTES"):
        n += 64
    return n


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [rqlp.PREC_FP32, rqlp.PREC_BF16X3])
def test_noalloc_matches_rqlp_factor_twice_in_a_row(precision):
    """Two calls in a row on different problems (the second one as large as
    the array allows), each against rqlp_factor with a caller workspace."""
    import torch
    nmax = _largest_square_within_bound(12, 4, 2, precision)
    cases = [(600, 500, 16, 4, 1, 11), (nmax, nmax, 12, 4, 2, 23)]
    for (m, n, k, p, q, seed) in cases:
        dA, dO = _problem(m, n, k, p, seed)
        Qn, Ln, Pn, info_n = _noalloc(dA, dO, k, p, q, precision)
        torch.cuda.synchronize()
        Qn, Ln, Pn = (x.double().cpu().numpy() for x in (Qn, Ln, Pn))
        Qr, Lr, Pr, info_r, _ = rqlp.factor(dA, k, p, q, dO, precision=precision)
        torch.cuda.synchronize()
        Qr, Lr, Pr = (x.double().cpu().numpy() for x in (Qr, Lr, Pr))
        assert int(info_n[0]) == 0 and int(info_r[0]) == 0
        assert np.max(np.abs(Qn - Qr)) <= ELEM_TOL
        assert np.max(np.abs(Pn - Pr)) <= ELEM_TOL
        assert np.max(np.abs(Ln - Lr)) <= ELEM_TOL * np.abs(Lr).max()
        assert np.max(np.abs(np.diag(Ln) - np.diag(Lr)) / np.diag(Lr)) <= TOL_LII


def test_noalloc_bound_comes_from_the_header():
    """The binding's copy of the array size is the header's value, and the
    sizes used above straddle it."""
    bound = rqlp.header_define("RQLP_NOALLOC_SCRATCH_BYTES")
    assert rqlp.NOALLOC_SCRATCH_BYTES == bound
    for prec in (rqlp.PREC_FP32, rqlp.PREC_BF16X3):
        n = _largest_square_within_bound(12, 4, 2, prec)
        o = rqlp.Opts(precision=prec)
        assert rqlp.rqlp_workspace_bytes(n, n, 12, 4, 2, o) <= bound < rqlp.rqlp_workspace_bytes(n + 64, n + 64, 12, 4, 2, o)


def test_noalloc_rejects_oversize_before_any_work():
    """A problem whose workspace exceeds the library's array is refused with
    RQLP_ERR_WORKSPACE before anything touches the (fake) pointers."""
    m, n, k, p, q = 8192, 8192, 200, 10, 2
    assert rqlp.rqlp_workspace_bytes(m, n, k, p, q) > rqlp.header_define("RQLP_NOALLOC_SCRATCH_BYTES")
    fake = 0x1000
    st = rqlp.rqlp_factor_noalloc(fake, m, n, n, k, p, q, fake, k + p, fake, k + p, fake, k + p,
                                  fake, k + p, fake, None, rqlp.rqlp_default_opts(), None)
    assert st == 6
    assert rqlp.rqlp_factor_noalloc(fake, 10, 10, 10, 0, 1, 0, fake, 1, fake, 1, fake, 1, fake, 1,
                                    fake, None, None, None) == 1
