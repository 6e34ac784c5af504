"""The allocation-free preconditioner entry point (rd_apply_precond_static)
against the workspace-based one (rd_apply_precond), through the C ABI.

rd_apply_precond_static is for callers that cannot allocate device memory
where they need the preconditioner (device memory owned by another
framework's pool, or loops that must not pay cudaMalloc's implicit
synchronisation).  Its scratch is a fixed __device__ array shared by all
calls, so the test calls it twice in a row with different inputs and checks
both results.  This file is collected last on purpose."""

import math

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_static_scratch_preconditioner_matches_workspace_version_twice():
    from paper_1907_07774_gb300 import build
    from paper_1907_07774_gb300 import rd as R
    from paper_1907_07774_gb300 import synth

    build.build()
    assert torch.cuda.is_available(), "GPU test"
    n = (32, 16, 64)
    prob = synth.calibration_problem(n=n, nt=4, m=2, sigma=2 * math.pi / 8)
    ctx = R.context_for(prob, prec="fp64")
    k_f = 0.07
    kappa1 = prob.k_w[0] * prob.m_wm + prob.k_w[1] * prob.m_gm + prob.k_w[2] * prob.m_csf
    coef = 0.5 * (1.0 / prob.nt) * k_f * float(kappa1[kappa1 > 0].mean())   # the context's constant
    gen = torch.Generator(device="cuda").manual_seed(11)
    for _ in range(2):
        r = torch.randn(n, dtype=torch.float64, device="cuda", generator=gen)
        r_copy = r.clone()
        want = torch.zeros_like(r)
        ctx.rd_apply_precond(k_f, r, want)
        got = torch.full_like(r, float("nan"))
        assert R.rd_apply_precond_static(n, coef, r, got) == R.RD_OK
        torch.cuda.synchronize()
        err = float(torch.linalg.norm(got - want) / torch.linalg.norm(want))
        assert err <= 1e-12, err
        assert torch.equal(r, r_copy)


def test_static_scratch_preconditioner_rejects_unsupported_grid():
    from paper_1907_07774_gb300 import rd as R

    r = torch.zeros(8, dtype=torch.float64, device="cuda")
    z = torch.zeros_like(r)
    assert R.rd_apply_precond_static((512, 8, 8), 0.1, r, z) == 2     # RD_ERR_SHAPE
    assert R.rd_apply_precond_static((8, 8, 8), -1.0, r, z) == 1      # RD_ERR_ARG
