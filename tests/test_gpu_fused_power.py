"""Power passes fused as A^T (A P~) over L2-sized row panels of A, with
Z = A P~ left un-orthonormalised (reading C3: the qf of the product does not
depend on a triangular right factor), against the FP64 oracle, which
orthonormalises after every product."""
import numpy as np
import pytest

from paper_2110_01011_gb300 import inputs
from parity_util import compare, run_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m,n,k,p,q,rate", [(8192, 8192, 40, 10, 2, 30.0), (6000, 4000, 64, 8, 3, 40.0),
                                            (3001, 2777, 20, 5, 1, 10.0), (9000, 3000, 100, 10, 2, 50.0)])
@pytest.mark.parametrize("prec", [0, 1], ids=["fp32", "bf16x3"])
def test_fused_power_matches_oracle(m, n, k, p, q, rate, prec):
    A = inputs.low_rank_matrix(m, n, inputs.exp_spectrum(min(m, n), rate), 1e-5, seed=m + 11 * n)
    Om = inputs.omega(m, k + p, seed=m + n + 1)
    err = compare(A, Om, k, p, q, run_gpu(A, Om, k, p, q, precision=prec, fused=True), elem_atol=5e-4,
                  precision=prec)
    print(m, n, ["fp32", "bf16x3"][prec], {kk: float(v) for kk, v in err.items()})
