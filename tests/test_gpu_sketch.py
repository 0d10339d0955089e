"""GPU parity of one pass over A (Algorithm 1 steps 3-4; the power passes):
Y = A^T X and Z = A X through rqlp_sketch, FP32 and BF16x3, against the
FP64 product (the oracle's step is the same library matmul in float64).

Tolerance: elementwise |Y - Y_ref| <= tol * (|A|^T |X|) with tol = 4e-6 for
FP32 (accumulation over K in FP32) and 1e-4 for BF16x3 (hi/lo split keeps
~16 significant bits per operand, the dropped A_lo X_lo term is 2^-18
relative, FP32 accumulation in tensor memory)."""
import numpy as np
import pytest

from paper_2110_01011_gb300 import inputs, rqlp

pytestmark = pytest.mark.gpu

# d = 160 and 161 sit on either side of the tensor-core pass's switch from
# K = 64 to K = 32 per pipeline stage (three K = 64 stages fit up to d = 160).
# In FP32, outputs of >= 1024 rows and >= 96 columns over K >= 1024 take the
# wide tile, 128 x 112 where that pads d less than 128 x 128 does (d = 100,
# 130, 160, 161, 210) and 128 x 128 otherwise (d = 128, 240): 1025 x 1031 with
# d = 130 has odd row strides (scalar loads), ragged tiles in both directions
# and split K; 3000 x 2000 with d = 100 the 128-bit loads. In BF16x3, A^T X of
# 9000 x 500 (four output tiles, ~38 CTAs each) and of 4100 x 300 sum their
# split tiles in a separate kernel after the pass.
SHAPES = [(300, 200, 13), (129, 257, 16), (1000, 777, 25), (777, 1000, 37),
          (2500, 1300, 210), (4100, 300, 64), (640, 512, 256), (97, 53, 1),
          (1500, 900, 160), (900, 1500, 161), (1025, 1031, 130), (3000, 2000, 100),
          (2048, 1100, 128), (1200, 1300, 240), (9000, 500, 205)]


def _run(A, X, trans, prec):
    import torch
    dA = torch.from_numpy(A).cuda()
    dX = torch.from_numpy(X).cuda()
    Y, _ = rqlp.sketch(dA, dX, trans, precision=prec)
    torch.cuda.synchronize()
    return Y.double().cpu().numpy()


@pytest.mark.parametrize("prec,tol", [(rqlp.PREC_FP32, 4e-6), (rqlp.PREC_BF16X3, 1e-4)])
@pytest.mark.parametrize("m,n,d", SHAPES)
@pytest.mark.parametrize("trans", [1, 0])
def test_pass(m, n, d, trans, prec, tol):
    g = inputs.rng(m * 31 + n * 7 + d)
    A = g.standard_normal((m, n)).astype(np.float32)
    X = g.standard_normal((m if trans else n, d)).astype(np.float32)
    A64, X64 = A.astype(np.float64), X.astype(np.float64)
    ref = A64.T @ X64 if trans else A64 @ X64
    bound = (np.abs(A64).T @ np.abs(X64)) if trans else (np.abs(A64) @ np.abs(X64))
    Y = _run(A, X, trans, prec)
    err = np.abs(Y - ref) / bound
    assert err.max() <= tol, (err.max(), np.unravel_index(err.argmax(), err.shape))


@pytest.mark.parametrize("trans", [1, 0])
def test_bf16_exact_x_uses_two_products(trans):
    """X exactly representable in BF16 (a rounded Omega): the low part is zero,
    the middle product is skipped, and the result is unchanged."""
    m, n, d = 1500, 900, 40
    g = inputs.rng(5)
    A = g.standard_normal((m, n)).astype(np.float32)
    X = inputs.round_to_bf16(g.standard_normal((m if trans else n, d)).astype(np.float32))
    A64, X64 = A.astype(np.float64), X.astype(np.float64)
    ref = A64.T @ X64 if trans else A64 @ X64
    bound = (np.abs(A64).T @ np.abs(X64)) if trans else (np.abs(A64) @ np.abs(X64))
    Y = _run(A, X, trans, rqlp.PREC_BF16X3)
    assert (np.abs(Y - ref) / bound).max() <= 1e-4


def test_bf16x3_typical_error_is_split_level():
    """Median relative error of BF16x3 sits near 2^-17, far below plain BF16 (2^-9)."""
    m, n, d = 2000, 2000, 64
    g = inputs.rng(9)
    A = g.standard_normal((m, n)).astype(np.float32)
    X = g.standard_normal((m, d)).astype(np.float32)
    ref = A.astype(np.float64).T @ X.astype(np.float64)
    bound = np.abs(A.astype(np.float64)).T @ np.abs(X.astype(np.float64))
    Y = _run(A, X, 1, rqlp.PREC_BF16X3)
    med = np.median(np.abs(Y - ref) / bound)
    assert med < 2e-6, med
