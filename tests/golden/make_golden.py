"""Writes the stored oracle results under tests/golden/ (regression fixtures
of the FP64 oracle; the paper prints no worked example that could serve).

Calls only the oracle and the seeded input recipe.  Run from the repository
root:  python tests/golden/make_golden.py
A change of a stored value is a change of the oracle's arithmetic and names,
in its commit message, the passage of the paper that justifies it."""

import json
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import rd as orc  # noqa: E402
from paper_1907_07774_gb300 import synth  # noqa: E402

# the gradient case: 16^3, nt = 4, 2^3 Gaussians of width 2 pi / 8
CASE = {"n": [16, 16, 16], "nt": 4, "m": 2, "sigma": 2 * math.pi / 8, "seed": 1000, "label_seed": 7,
        "rtol": 1e-13, "fft": "recursive"}


def compute(case=CASE):
    prob = synth.calibration_problem(n=tuple(case["n"]), nt=case["nt"], m=case["m"], sigma=case["sigma"],
                                     seed=case["seed"])
    M = orc.model_from_problem(prob, rtol=case["rtol"], maxit=1000, kind=case["fft"])
    c_true, _ = M.forward(prob.p_true, prob.k_f_true, prob.rho_f_true)
    d = synth.labels(c_true, synth.ellipsoid_mask(prob.n), case["label_seed"])
    c1, _ = M.forward(prob.p, prob.k_f, prob.rho_f)
    J, g = M.gradient(prob.p, prob.k_f, prob.rho_f, d)[:2]
    return {
        "case": case,
        "c1_sum": float(c1.sum()),
        "c1_sumsq": float((c1 * c1).sum()),
        "c1_max": float(c1.max()),
        "labels_sum": float(d.sum()),
        "misfit": float(J),
        "gradient": [float(x) for x in g],
    }


if __name__ == "__main__":
    out = os.path.join(HERE, "oracle_gradient_16.json")
    with open(out, "w") as f:
        json.dump(compute(), f, indent=1)
        f.write("\n")
    print("wrote", out)
