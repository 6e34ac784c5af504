"""The stored oracle results (tests/golden/) against the oracle as it is now
(CPU), and the CUDA path against the stored values (GPU)."""

import json
import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_golden  # noqa: E402

GOLDEN = os.path.join(HERE, "golden", "oracle_gradient_16.json")


def _stored():
    with open(GOLDEN) as f:
        return json.load(f)


def _rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_oracle_reproduces_the_stored_gradient_case():
    want = _stored()
    got = make_golden.compute(want["case"])
    assert got["labels_sum"] == want["labels_sum"]
    for k in ("c1_sum", "c1_sumsq", "c1_max", "misfit"):
        assert abs(got[k] - want[k]) <= 1e-11 * abs(want[k]), k
    assert _rel(got["gradient"], want["gradient"]) <= 1e-11


@pytest.mark.gpu
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 2e-4)])
def test_cuda_gradient_matches_the_stored_oracle_values(prec, tol):
    pytest.importorskip("torch")
    from oracle import rd as orc
    from paper_1907_07774_gb300 import rd as R
    from paper_1907_07774_gb300 import synth

    want = _stored()
    case = want["case"]
    prob = synth.calibration_problem(n=tuple(case["n"]), nt=case["nt"], m=case["m"], sigma=case["sigma"],
                                     seed=case["seed"])
    # the labels come from the oracle's c_true(1), as in the stored case
    M = orc.model_from_problem(prob, rtol=case["rtol"], maxit=1000, kind="numpy")
    c_true, _ = M.forward(prob.p_true, prob.k_f_true, prob.rho_f_true)
    d = synth.labels(c_true, synth.ellipsoid_mask(prob.n), case["label_seed"])
    assert d.sum() == want["labels_sum"]
    ctx = R.context_for(prob, prec=prec, pcg_rtol=1e-12 if prec == "fp64" else 1e-6, pcg_maxit=1000)
    ctx.rd_set_data(d)
    c1 = np.zeros(prob.n)
    ctx.rd_forward(prob.p, prob.k_f, prob.rho_f, c1)
    assert abs(c1.sum() - want["c1_sum"]) <= tol * abs(want["c1_sum"])
    J, g = ctx.rd_gradient(prob.p, prob.k_f, prob.rho_f)
    assert abs(J - want["misfit"]) <= tol * abs(want["misfit"])
    assert _rel(g, want["gradient"]) <= tol
