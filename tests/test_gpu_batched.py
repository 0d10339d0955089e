"""GPU parity of the batched form: every problem of a batch against the FP64
oracle on the same seeded inputs, through the batch plan's graph launch and
plain launches, before and after autotuning, in FP32 and in BF16x3 (the
passes over A as grouped tensor-core passes)."""
import numpy as np
import pytest

from paper_2110_01011_gb300 import inputs
from parity_util import compare

pytestmark = pytest.mark.gpu


def _problems(count, seed, q_rate=3.0, dmax=69, sizes=((40, 500), (40, 400)), ps=(0, 3, 5)):
    g = inputs.rng(seed)
    out = []
    while len(out) < count:
        m = int(g.integers(*sizes[0]))
        n = int(g.integers(*sizes[1]))
        k = int(g.integers(1, 65))
        p = int(g.choice(list(ps)))
        if k + p > min(m, n) or k + p > dmax:
            continue
        sig = inputs.exp_spectrum(min(m, n), rate=max(4.0, (k + p) / q_rate))
        s = 1000 * len(out) + seed
        A = inputs.low_rank_matrix(m, n, sig, 1e-5, seed=s)
        Om = inputs.omega(m, k + p, seed=s + 1)
        out.append((A, Om, k, p))
    return out


PRECS = [0, 1]   # rqlp.PREC_FP32, rqlp.PREC_BF16X3


def _batch(probs, q, small_fp64=False, precision=0, test_stall=False, parts=0):
    import torch

    from paper_2110_01011_gb300 import rqlp
    As = [torch.from_numpy(np.ascontiguousarray(A)).cuda() for A, _, _, _ in probs]
    Os = [torch.from_numpy(np.ascontiguousarray(O)).cuda() for _, O, _, _ in probs]
    b = rqlp.Batch(As, Os, [k for _, _, k, _ in probs], [p for _, _, _, p in probs], q, small_fp64=small_fp64,
                   precision=precision, test_stall=test_stall, parts=parts)
    return b


def _results(b, i):
    import torch
    torch.cuda.synchronize()
    return (b.Q[i].double().cpu().numpy(), b.L[i].double().cpu().numpy(), b.P[i].double().cpu().numpy(),
            b.info[i].cpu().numpy(), b.diag[i].cpu().numpy())


def _check_all(b, probs, q, precision=0):
    for i, (A, Om, k, p) in enumerate(probs):
        compare(A, Om, k, p, q, _results(b, i), elem_atol=5e-4, precision=precision)


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
        compare(*probs[i][:2], probs[i][2], probs[i][3], 0, _results(b, i), elem_atol=5e-4, precision=prec)
    b.close()


@pytest.mark.parametrize("parts", [0, 2])
def test_split_form_large_problems(parts):
    """BF16x3 batch with problems whose K spans more than one accumulation
    chunk of the grouped pass (m = 4500 > 4096) and ragged tiles, in three
    parts (the default) and in two on request."""
    g = []
    for (m, n, k, p, s) in [(4500, 300, 40, 5, 11), (300, 4200, 20, 5, 12), (1111, 777, 64, 5, 13)]:
        sig = inputs.exp_spectrum(min(m, n), rate=max(4.0, (k + p) / 3))
        g.append((inputs.low_rank_matrix(m, n, sig, 1e-5, seed=s), inputs.omega(m, k + p, seed=s + 9), k, p))
    b = _batch(g, 1, precision=1, parts=parts)
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
    probs = _problems(3, seed=41, ps=(5, 8))   # p >= 5: the passes run on the tensor cores
    b = _batch(probs, 1, precision=1, test_stall=True)
    b.launch()
    torch.cuda.synchronize()
    assert int(b.info[0, 0].item()) == 5          # RQLP_ERR_TIMEOUT
    b.close()
    b = _batch(probs, 1, precision=1)
    b.launch()
    _check_all(b, probs, 1, 1)
    b.close()


def _ill_conditioned(kind, ratio, m, n, k, p, seed):
    """sigma_1 / sigma_k = ratio, exponential or polynomial decay, noise 1e-6."""
    r = min(m, n)
    if kind == "exp":
        sig = np.exp(-np.arange(r) * np.log(ratio) / (k - 1))
    else:
        sig = np.arange(1, r + 1, dtype=np.float64) ** (-np.log(ratio) / np.log(k))
    return inputs.low_rank_matrix(m, n, sig, 1e-6, seed=seed), inputs.omega(m, k + p, seed=seed + 1)


@pytest.mark.parametrize("prec", PRECS)
def test_ill_conditioned_leading_blocks(prec):
    """The class the two-part split once missed: k = 12, p = 0, q = 2,
    sigma_1 / sigma_k from 15.6 to 100 (and p = 5 beside it), one batch, the
    plain 1e-4 |L_ii| bound in both precisions (BF16x3 in three parts)."""
    probs = []
    s = 500
    for kind in ("exp", "poly"):
        for ratio in (15.6, 50.0, 100.0):
            for p in (0, 5):
                s += 2
                m, n = 300 + 17 * (s % 7), 200 + 13 * (s % 5)
                A, Om = _ill_conditioned(kind, ratio, m, n, 12, p, s)
                probs.append((A, Om, 12, p))
    b = _batch(probs, 2, precision=prec)
    b.launch()
    _check_all(b, probs, 2, prec)
    b.close()
