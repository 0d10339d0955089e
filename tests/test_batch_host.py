"""Host-side rules of the batch plan (no GPU): workspace sizing and argument
validation run on the host only."""
import pytest

from paper_2110_01011_gb300 import rqlp


def _prob(m, n, k, p, ld_extra=0):
    fake = 1 << 20   # never dereferenced by the sizing call
    d = k + p
    return rqlp.Problem(fake, m, n, n + ld_extra, fake, d, k, p, fake, d, fake, d, fake, d)


def _arr(ps):
    a = (rqlp.Problem * len(ps))()
    for i, p in enumerate(ps):
        a[i] = p
    return a


def test_sizing_grows_with_problems():
    one = rqlp.rqlp_batch_workspace_bytes(1, _arr([_prob(300, 200, 20, 5)]), 1)
    two = rqlp.rqlp_batch_workspace_bytes(2, _arr([_prob(300, 200, 20, 5), _prob(500, 100, 50, 5)]), 1)
    assert 0 < one < two
    # per-problem buffers: Y, Pt (n x ld), Z (m x ld), T1 (max x ld) at least
    assert one >= 4 * (200 + 300 + 200 + 300) * 28


@pytest.mark.parametrize("bad", [
    _prob(30, 20, 18, 5),          # d > min(m, n)
    _prob(300, 300, 125, 5),       # d > RQLP_BATCH_MAX_D
    _prob(300, 200, 0, 5),         # k < 1
    _prob(300, 200, 10, -1),       # p < 0
    _prob(300, 200, 10, 5, -1),    # lda < n
])
def test_invalid_problem_sizes_to_zero(bad):
    assert rqlp.rqlp_batch_workspace_bytes(2, _arr([_prob(300, 200, 20, 5), bad]), 1) == 0


def test_invalid_batch_arguments():
    a = _arr([_prob(300, 200, 20, 5)])
    assert rqlp.rqlp_batch_workspace_bytes(0, a, 1) == 0
    assert rqlp.rqlp_batch_workspace_bytes(1, a, -1) == 0
    assert rqlp.rqlp_batch_workspace_bytes(1, a, 1, rqlp._opts(7)) == 0          # unknown precision


@pytest.mark.parametrize("parts", [2, 3])
def test_split_form_workspace_holds_the_parts(parts):
    """The BF16x3 batch adds A's BF16 parts (64-column panels), the pass
    operand's parts and the tensor maps (8, or 12 with a third part) to the
    FP32 batch's workspace; without bf16_parts the batch takes three."""
    a = _arr([_prob(300, 200, 20, 5), _prob(500, 100, 40, 5)])
    fp32 = rqlp.rqlp_batch_workspace_bytes(2, a, 1)
    split = rqlp.rqlp_batch_workspace_bytes(2, a, 1, rqlp._opts(rqlp.PREC_BF16X3, parts=parts))
    halves = parts * 2 * (300 * 256 + 500 * 128)             # A_hi, A_lo[, A_lo2], BF16
    xt = parts * 2 * (25 * 304 + 45 * 504)                  # X parts^T, d x round8(max(m, n))
    maps = 2 * (8 if parts == 2 else 12) * 128
    assert split - fp32 >= halves + xt + maps
    assert split - fp32 <= halves + xt + maps + 64 * 1024     # + the grouped passes' plan tables
    if parts == 3:
        assert rqlp.rqlp_batch_workspace_bytes(2, a, 1, rqlp._opts(rqlp.PREC_BF16X3)) == split


def test_stall_hook_only_for_split_batches():
    a = _arr([_prob(300, 200, 20, 5)])
    o = rqlp._opts(rqlp.PREC_BF16X3)
    o.test_stall = 1
    assert rqlp.rqlp_batch_workspace_bytes(1, a, 1, o) > 0
    o.test_stall = 2
    assert rqlp.rqlp_batch_workspace_bytes(1, a, 1, o) == 0
    o = rqlp._opts(rqlp.PREC_FP32)
    o.test_stall = 1
    assert rqlp.rqlp_batch_workspace_bytes(1, a, 1, o) == 0


def test_batch_option_rules():
    """The paper-literal step 5 is a single-matrix option; BF16 parts belong to
    the BF16x3 form (2 or 3)."""
    a = _arr([_prob(300, 200, 20, 5)])
    assert rqlp.rqlp_batch_workspace_bytes(1, a, 1, rqlp._opts(literal=True)) == 0
    assert rqlp.rqlp_batch_workspace_bytes(1, a, 1, rqlp._opts(rqlp.PREC_BF16X3, parts=2)) > 0
    assert rqlp.rqlp_batch_workspace_bytes(1, a, 1, rqlp._opts(rqlp.PREC_BF16X3, parts=3)) > 0
    assert rqlp.rqlp_batch_workspace_bytes(1, a, 1, rqlp._opts(rqlp.PREC_BF16X3, parts=1)) == 0
    assert rqlp.rqlp_batch_workspace_bytes(1, a, 1, rqlp._opts(rqlp.PREC_FP32, parts=2)) == 0
