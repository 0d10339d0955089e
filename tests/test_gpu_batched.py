"""GPU parity of the batched form: every problem of a batch against the FP64
oracle on the same seeded inputs, through the batch plan's graph launch and
plain launches, before and after autotuning, in FP32 and in BF16x3 (the
passes over A as grouped tensor-core passes)."""
import numpy as np
import pytest

from paper_2110_01011_gb300 import inputs
from parity_util import compare

pytestmark = pytest.mark.gpu


def _problems(count, seed, q_rate=3.0, dmax=69, sizes=((40, 500), (40, 400))):
    g = inputs.rng(seed)
    out = []
    while len(out) < count:
        m = int(g.integers(*sizes[0]))
        n = int(g.integers(*sizes[1]))
        k = int(g.integers(1, 65))
        p = int(g.choice([0, 3, 5]))
        if k + p > min(m, n) or k + p > dmax:
            continue
        sig = inputs.exp_spectrum(min(m, n), rate=max(4.0, (k + p) / q_rate))
        s = 1000 * len(out) + seed
        A = inputs.low_rank_matrix(m, n, sig, 1e-5, seed=s)
        Om = inputs.omega(m, k + p, seed=s + 1)
        out.append((A, Om, k, p))
    return out


PRECS = [0, 1]   # rqlp.PREC_FP32, rqlp.PREC_BF16X3


def _batch(probs, q, small_fp64=False, precision=0, test_stall=False):
    import torch

    from paper_2110_01011_gb300 import rqlp
    As = [torch.from_numpy(np.ascontiguousarray(A)).cuda() for A, _, _, _ in probs]
    Os = [torch.from_numpy(np.ascontiguousarray(O)).cuda() for _, O, _, _ in probs]
    b = rqlp.Batch(As, Os, [k for _, _, k, _ in probs], [p for _, _, _, p in probs], q, small_fp64=small_fp64,
                   precision=precision, test_stall=test_stall)
    return b


def _results(b, i):
    import torch
    torch.cuda.synchronize()
    return (b.Q[i].double().cpu().numpy(), b.L[i].double().cpu().numpy(), b.P[i].double().cpu().numpy(),
            b.info[i].cpu().numpy(), b.diag[i].cpu().numpy())


# BF16x3 passes: each product carries ~2^-16 of |A| |X| (16 bits per operand),
# so an |L_ii| near sigma_i takes up to ~2 * 2^-16 * sigma_1 / sigma_i of its
# own size (measured on the single-problem path too: 2.7e-4 at k = 12, p = 0,
# q = 2, sigma_1 / sigma_k = 15.6, where FP32 gives 9e-6).
LII_SCALE = {0: None, 1: 2 * 2.0 ** -16}


def _check_all(b, probs, q, precision=0):
    for i, (A, Om, k, p) in enumerate(probs):
        compare(A, Om, k, p, q, _results(b, i), elem_atol=5e-4, precision=precision,
                lii_cond_scale=LII_SCALE[precision])


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("q", [0, 1, 2])
def test_batch_matches_oracle(q, prec):
    probs = _problems(18, seed=100 + q)
    assert any(k + p <= 32 for _, _, k, p in probs) and any(k + p > 32 for _, _, k, p in probs)
    b = _batch(probs, q, precision=prec)
    b.launch()
    _check_all(b, probs, q, prec)
    b.close()


@pytest.mark.parametrize("prec", PRECS)
def test_graph_replay_and_plain_launches_agree_bitwise(prec):
    probs = _problems(10, seed=7)
    b = _batch(probs, 1, precision=prec)
    b.launch()
    first = [_results(b, i) for i in range(len(probs))]
    b.launch()                      # replay
    second = [_results(b, i) for i in range(len(probs))]
    b.run()                         # the same kernels launched one by one
    third = [_results(b, i) for i in range(len(probs))]
    for x, y, z in zip(first, second, third):
        for u, v, w in zip(x, y, z):
            assert np.array_equal(u, v) and np.array_equal(u, w)
    b.close()


def test_autotune_then_launch():
    probs = _problems(16, seed=21)
    b = _batch(probs, 1)
    tune = b.autotune(reps=2)
    assert len(tune) == 10 and all(0 <= c < 12 for c in tune)
    b.launch()
    _check_all(b, probs, 1)
    b.close()


@pytest.mark.parametrize("prec", PRECS)
def test_edge_problems(prec):
    """d = 1, d = k (p = 0), square d = min(m, n), the widest d = 128, one batch."""
    g = []
    for (m, n, k, p, s) in [(50, 30, 1, 0, 1), (64, 64, 60, 4, 2), (300, 200, 120, 8, 3), (90, 200, 32, 0, 4),
                            (77, 91, 33, 0, 5)]:
        sig = inputs.exp_spectrum(min(m, n), rate=max(4.0, (k + p) / 3))
        g.append((inputs.low_rank_matrix(m, n, sig, 1e-5, seed=s), inputs.omega(m, k + p, seed=s + 9), k, p))
    b = _batch(g, 1, precision=prec)
    b.launch()
    _check_all(b, g, 1, prec)
    b.close()


def test_single_problem_and_small_fp64():
    probs = _problems(1, seed=5)
    b = _batch(probs, 1, small_fp64=True)
    b.launch()
    _check_all(b, probs, 1)
    b.close()


@pytest.mark.parametrize("prec", PRECS)
def test_status_rows_follow_caller_order(prec):
    """A non-finite problem and a rank-deficient one among healthy ones: only
    their own info / diag rows show it (problems are reordered internally)."""
    probs = _problems(6, seed=31)
    m, n = 120, 90
    bad = inputs.low_rank_matrix(m, n, inputs.exp_spectrum(n, 10.0), 0.0, seed=3)
    bad[5, 7] = np.nan
    probs[2] = (bad, inputs.omega(m, 40, seed=4), 35, 5)
    low = inputs.low_rank_matrix(m, n, np.linspace(1.0, 0.5, 4), 0.0, seed=5)
    probs[4] = (low, inputs.omega(m, 10, seed=6), 8, 2)
    b = _batch(probs, 0, precision=prec)
    b.launch()
    import torch
    torch.cuda.synchronize()
    info = b.info.cpu().numpy()
    diag = b.diag.cpu().numpy()
    assert info[2, 0] == 4                      # RQLP_ERR_NONFINITE
    assert info[4, 0] in (0, 3) and diag[4, 3] >= 1
    for i in (0, 1, 3, 5):
        assert info[i, 0] == 0 and diag[i, 3] == 0
        compare(*probs[i][:2], probs[i][2], probs[i][3], 0, _results(b, i), elem_atol=5e-4, precision=prec,
                lii_cond_scale=LII_SCALE[prec])
    b.close()


def test_split_form_large_problems():
    """BF16x3 batch with problems whose K spans more than one accumulation
    chunk of the grouped pass (m = 4500 > 4096) and ragged tiles."""
    g = []
    for (m, n, k, p, s) in [(4500, 300, 40, 5, 11), (300, 4200, 20, 5, 12), (1111, 777, 64, 5, 13)]:
        sig = inputs.exp_spectrum(min(m, n), rate=max(4.0, (k + p) / 3))
        g.append((inputs.low_rank_matrix(m, n, sig, 1e-5, seed=s), inputs.omega(m, k + p, seed=s + 9), k, p))
    b = _batch(g, 1, precision=1)
    b.launch()
    _check_all(b, g, 1, 1)
    b.close()


def test_withheld_stage_times_out_and_the_context_survives():
    """Fault injection without a GPU fault: CTA 0 of the first grouped pass
    withholds its first stage (the test hook), its bounded waits run out
    (~2 s each), the first problem's status row reports RQLP_ERR_TIMEOUT, the
    kernel frees what it holds and returns; a normal batch afterwards is
    correct."""
    import torch
    probs = _problems(3, seed=41)
    b = _batch(probs, 1, precision=1, test_stall=True)
    b.launch()
    torch.cuda.synchronize()
    assert int(b.info[0, 0].item()) == 5          # RQLP_ERR_TIMEOUT
    b.close()
    b = _batch(probs, 1, precision=1)
    b.launch()
    _check_all(b, probs, 1, 1)
    b.close()
