"""Writes tests/golden/rqlp_oracle_small.json: the FP64 oracle's Rand-QLP of
three small seeded problems (Algorithm 1, truncated to d = k + p columns, q
power passes), as a regression record of the oracle's arithmetic.

Calls only the oracle and the seeded input generators. The paper prints no
worked example with values, so this file records the oracle, not the
paper; the oracle itself is pinned by tests/test_oracle_pins.py (closed
forms, invariants, brute force). Regenerate only when a change to the
oracle's arithmetic is justified by the passage of the paper it follows:

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import rqlp_oracle as orc  # noqa: E402
from paper_2110_01011_gb300 import inputs  # noqa: E402

# (m, n, k, p, q, spectrum, noise, seed)
CASES = [
    (12, 9, 3, 2, 1, "exp", 1e-3, 11),
    (20, 30, 5, 0, 2, "step", 0.0, 12),
    (40, 25, 8, 4, 0, "poly", 1e-4, 13),
]


def spectrum(kind, n):
    if kind == "exp":
        return inputs.exp_spectrum(n, rate=3.0)
    if kind == "step":
        return inputs.step_spectrum(n, k=4, tail=0.1)
    return inputs.poly_spectrum(n, alpha=1.5)


def case(m, n, k, p, q, kind, noise, seed):
    A = inputs.low_rank_matrix(m, n, spectrum(kind, min(m, n)), noise, seed=seed)
    Om = inputs.omega(m, k + p, seed=seed + 1)
    r = orc.rand_qlp(A.astype(np.float64), Om.astype(np.float64), q)
    return {
        "m": m, "n": n, "k": k, "p": p, "q": q, "spectrum": kind, "noise": noise, "seed": seed,
        "L_diag": [float(x) for x in np.diag(r.L)],
        "L_fro": float(np.linalg.norm(r.L)),
        "residual_fro": float(orc.residual_fro(A.astype(np.float64), r.Q, r.L, r.P)),
    }


def main():
    out = {"source": "oracle/rqlp_oracle.py rand_qlp on inputs.low_rank_matrix / inputs.omega",
           "cases": [case(*c) for c in CASES]}
    with open(os.path.join(HERE, "rqlp_oracle_small.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
