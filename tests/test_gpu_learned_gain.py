"""What the trained (q, p) network gains over the method without it.

Held-out matrices (a seed the training never used; the training set's
recipe, n in [384, 1536]) are labelled by running the method: one
width-(k + 20) chain gives the excess rank-k error of all 15 (q, p). At
requests the fixed q = 2, p = 10 mostly misses (1e-2), the network's picks
reach the request far more often; at a loose request (1e-1) they reach it
as often as the fixed pair at a clearly lower cost (2q + 2)(k + p), the
flops of the passes over A. The network and its selection run on the
device (rqlp_mlp_forward and the library's selection rule, which
tests/test_learn_host.py pins to the FP64 reference).
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def held_out():
    from paper_2110_01011_gb300 import learn
    if not os.path.exists(learn.WEIGHTS):
        pytest.skip("no trained weights in the package")
    feats, ks, tabs, _ = learn.build_dataset(120, seed=31337, device="cuda", log_every=0, n_range=(384, 1536))
    params = learn.load_weights().astype(np.float64)
    return learn.evaluate(params, feats, tabs, ks, targets=(1e-2, 3e-2, 1e-1))


def test_gain_where_the_fixed_pair_misses(held_out):
    r = {e["target"]: e for e in held_out}[1e-2]
    print(r)
    assert r["learned_success"] >= r["default_success"] + 0.4
    assert r["learned_success"] >= 0.75 * r["feasible"]


def test_gain_in_cost_at_a_loose_request(held_out):
    r = {e["target"]: e for e in held_out}[1e-1]
    print(r)
    assert r["learned_success"] >= 0.95 and r["default_success"] >= 0.95
    assert r["learned_cost"] <= 0.8 * r["default_cost"]


def test_no_loss_between(held_out):
    r = {e["target"]: e for e in held_out}[3e-2]
    print(r)
    assert r["learned_success"] >= r["default_success"] - 0.1
    assert r["learned_cost"] <= 1.25 * r["default_cost"]
