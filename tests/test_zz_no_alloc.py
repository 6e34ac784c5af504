"""The allocation-free preconditioner entry point (rd_apply_precond_static)
against the workspace-based one (rd_apply_precond), through the C ABI.

rd_apply_precond_static is for callers that cannot allocate device memory
where they need the preconditioner (device memory owned by another
framework's pool, or loops that must not pay cudaMalloc's implicit
synchronisation).  Its scratch is a fixed __device__ array shared by all
calls, so the test calls it twice in a row with different inputs and checks
both results.  This file is collected last on purpose."""

import math
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


# (96, 8, 64) and (8, 256, 16) run the radix-3 length and the largest length
# on different axes: the lengths whose twiddle slots are padded or filled to
# the array's fixed size
@pytest.mark.parametrize("n", [(32, 16, 64), (96, 8, 64), (8, 256, 16)])
def test_static_scratch_preconditioner_matches_workspace_version_twice(n):
    from paper_1907_07774_gb300 import build
    from paper_1907_07774_gb300 import rd as R
    from paper_1907_07774_gb300 import synth

    build.build()
    assert torch.cuda.is_available(), "GPU test"
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
    assert R.rd_apply_precond_static((8, 8, 8), math.inf, r, z) == 1  # RD_ERR_ARG
    assert R.rd_apply_precond_static((8, 8, 8), math.nan, r, z) == 1  # RD_ERR_ARG


_FIRST_CALL_ON_SIDE_STREAM = r"""
import math, sys, torch
sys.path.insert(0, sys.argv[1])
from paper_1907_07774_gb300 import rd as R
from paper_1907_07774_gb300 import synth
n = (16, 32, 8)
prob = synth.calibration_problem(n=n, nt=4, m=2, sigma=2 * math.pi / 8)
side = torch.cuda.Stream()          # a non-blocking stream
gen = torch.Generator(device="cuda").manual_seed(5)
r = torch.randn(n, dtype=torch.float64, device="cuda", generator=gen)
got = torch.full_like(r, float("nan"))
torch.cuda.synchronize()
k_f = 0.07
kappa1 = prob.k_w[0] * prob.m_wm + prob.k_w[1] * prob.m_gm + prob.k_w[2] * prob.m_csf
coef = 0.5 * (1.0 / prob.nt) * k_f * float(kappa1[kappa1 > 0].mean())
with torch.cuda.stream(side):
    assert R.rd_apply_precond_static(n, coef, r, got, stream=side) == R.RD_OK
side.synchronize()
ctx = R.context_for(prob, prec="fp64")
want = torch.zeros_like(r)
ctx.rd_apply_precond(k_f, r, want)
torch.cuda.synchronize()
err = float(torch.linalg.norm(got - want) / torch.linalg.norm(want))
assert err <= 1e-12, err
print("ok", err)
"""


def test_static_scratch_first_call_on_a_side_stream_in_a_fresh_process():
    """The first call on a device uploads the twiddle tables; it must be
    complete before the passes run on a caller's non-blocking stream."""
    from paper_1907_07774_gb300 import build

    build.build()
    out = subprocess.run([sys.executable, "-c", _FIRST_CALL_ON_SIDE_STREAM, ROOT], capture_output=True,
                         text=True, timeout=600)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.strip().startswith("ok")
