"""The CUDA path against stored FP64 oracle runs at the grids where the
production kernels run (tests/golden/make_golden_full.py): 128^3 with 16
steps, and the benchmark grid 256^3 with 2 and with 32 steps.

Each case holds the oracle's labels, misfit, gradient (and, for two of them,
one Gauss-Newton Hessian-vector product), checksums of c(1) and alpha(0)
and three planes of c(1).  Tolerances are those of the rest of the parity
tests: relative L2 <= 1e-10 for the FP64 path (both sides solve to 1e-12)
and <= 2e-4 for the mixed path (FP32 fields, FP64 reductions, PCG rtol 1e-6).

The CPU test checks that every stored case is complete and self-consistent
(the labels reproduce the stored count, the planes match the checksums'
magnitude); re-running the oracle at these sizes takes hours, which is what
the stored values are for."""

import math
import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_golden_full as G  # noqa: E402

TOL = {"fp64": 1e-10, "mixed": 2e-4}
RTOL = {"fp64": 1e-12, "mixed": 1e-6}
CASES = [name for name in G.CASES if name.startswith("grad")]


def _have(name):
    return all(os.path.exists(p) for p in G.paths(name))


def rel(a, b):
    a, b = np.ravel(np.asarray(a, dtype=np.float64)), np.ravel(np.asarray(b, dtype=np.float64))
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("name", CASES)
def test_stored_case_is_complete(name):
    if not _have(name):
        pytest.skip(f"{name} not stored")
    want, arr = G.load(name)
    n = want["case"]["n"]
    assert arr["labels"].shape == (n, n, n)
    assert float(arr["labels"].sum()) == want["labels_sum"]
    assert set(np.unique(arr["labels"])) <= {0.0, 1.0}
    npar = want["case"]["m"] ** 3 + 2
    assert len(want["gradient"]) == npar and np.all(np.isfinite(want["gradient"]))
    if want["case"]["hessvec"]:
        assert len(want["hessvec"]) == npar
    for k in ("c1_plane0", "c1_plane1", "c1_plane2"):
        assert arr[k].shape == (n, n)
        # a plane's squares never exceed the whole field's
        assert float((arr[k] ** 2).sum()) <= want["c1"]["sumsq"] * (1 + 1e-12)
    assert want["misfit"] > 0 and min(want["pcg_iters_forward"]) >= 1


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", CASES)
def test_cuda_path_matches_the_stored_oracle_run(name, prec):
    torch = pytest.importorskip("torch")
    if not _have(name):
        pytest.skip(f"{name} not stored")
    from paper_1907_07774_gb300 import build
    from paper_1907_07774_gb300 import rd as R
    build.build()
    assert torch.cuda.is_available(), "GPU test"
    want, arr = G.load(name)
    case = want["case"]
    n = case["n"]
    tol = TOL[prec]
    prob = G.problem(case)
    ctx = R.context_for(prob, prec=prec, pcg_rtol=RTOL[prec], pcg_maxit=5000)
    ctx.rd_set_data(torch.from_numpy(arr["labels"]).cuda())
    w = torch.from_numpy(G.weight_field(n)).cuda()

    def check_sums(field, stored, what):
        s = float(field.sum())
        ss = float((field * field).sum())
        dw = float((field * w).sum())
        assert abs(s - stored["sum"]) <= tol * math.sqrt(stored["sumsq"] * n ** 3), (what, s, stored["sum"])
        assert abs(ss - stored["sumsq"]) <= 2.001 * tol * stored["sumsq"], (what, ss, stored["sumsq"])
        # |<u - u*, w>| <= ||u - u*|| ||w||
        bound = tol * math.sqrt(stored["sumsq"] * float((w * w).sum()))
        assert abs(dw - stored["dot_w"]) <= bound, (what, dw, stored["dot_w"])

    c1 = torch.zeros((n, n, n), dtype=torch.float64, device="cuda")
    J = ctx.rd_forward(prob.p, prob.k_f, prob.rho_f, c1)
    assert abs(J - want["misfit"]) <= tol * want["misfit"]
    check_sums(c1, want["c1"], "c(1)")
    h = n // 2
    for k, plane in (("c1_plane0", c1[h, :, :]), ("c1_plane1", c1[:, h, :]), ("c1_plane2", c1[:, :, h])):
        assert rel(plane.cpu().numpy(), arr[k]) <= tol, k
    alpha0 = torch.zeros_like(c1)
    g_adj = ctx.rd_adjoint(alpha0)
    check_sums(alpha0, want["alpha0"], "alpha(0)")
    if "alpha0_plane0" in arr:
        assert rel(alpha0[h, :, :].cpu().numpy(), arr["alpha0_plane0"]) <= tol
    assert rel(g_adj, want["gradient"]) <= tol
    del c1, alpha0
    Jg, g = ctx.rd_gradient(prob.p, prob.k_f, prob.rho_f)
    assert abs(Jg - want["misfit"]) <= tol * want["misfit"]
    assert rel(g, want["gradient"]) <= tol
    if case["hessvec"]:
        v = G.direction(len(prob.p) + 2)
        hv = ctx.rd_hessvec(prob.p, prob.k_f, prob.rho_f, v)
        assert rel(hv, want["hessvec"]) <= tol
