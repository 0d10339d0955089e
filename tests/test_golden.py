"""The FP64 oracle against its recorded outputs (tests/golden/, written by
tests/golden/make_golden.py from the oracle alone): a regression record, so
that a change to the oracle's arithmetic shows up here and has to be
justified by the passage of the paper it follows. The recorded values also
satisfy the residual identity ||A||_F^2 = ||L||_F^2 + ||A - Q L P^T||_F^2
(Q and P orthonormal, L = Q^T A P)."""
import json
import os

import numpy as np
import pytest

from oracle import rqlp_oracle as orc
from paper_2110_01011_gb300 import inputs

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
REC = json.load(open(os.path.join(HERE, "rqlp_oracle_small.json")))


def _inputs(c):
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    A = inputs.low_rank_matrix(c["m"], c["n"], mg.spectrum(c["spectrum"], min(c["m"], c["n"])), c["noise"],
                               seed=c["seed"])
    Om = inputs.omega(c["m"], c["k"] + c["p"], seed=c["seed"] + 1)
    return A.astype(np.float64), Om.astype(np.float64)


@pytest.mark.parametrize("i", range(len(REC["cases"])))
def test_oracle_reproduces_record(i):
    c = REC["cases"][i]
    A, Om = _inputs(c)
    r = orc.rand_qlp(A, Om, c["q"])
    ld = np.array(c["L_diag"])
    assert np.allclose(np.diag(r.L), ld, rtol=1e-9, atol=1e-12 * np.abs(ld).max())
    assert np.isclose(np.linalg.norm(r.L), c["L_fro"], rtol=1e-10)
    assert np.isclose(orc.residual_fro(A, r.Q, r.L, r.P), c["residual_fro"], rtol=1e-7, atol=1e-12)


@pytest.mark.parametrize("i", range(len(REC["cases"])))
def test_record_satisfies_residual_identity(i):
    c = REC["cases"][i]
    A, _ = _inputs(c)
    a2 = np.linalg.norm(A) ** 2
    assert abs(c["L_fro"] ** 2 + c["residual_fro"] ** 2 - a2) <= 1e-10 * a2
