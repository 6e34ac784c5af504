"""Failure paths of the solver library, all provoked on the host side.

The paper's only safeguards are iteration caps on its solvers (Sec. 3.1,
3.2); the library adds status codes for non-convergence, non-finite values,
bad arguments and device-side waits that give up.  Every failure here is made
on the host: an iteration cap too small to converge, a NaN written into a
host array before it is handed over, a null or misaligned pointer, a
transaction that nothing completes (the bounded-wait self-test).  After each
failure the same context must still produce the oracle's result."""

import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import rd as orc
from paper_1907_07774_gb300 import rd as R
from paper_1907_07774_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-10, "mixed": 2e-4}
RTOL = {"fp64": 1e-12, "mixed": 1e-6}
RD_ERR_ARG, RD_ERR_NOCONV, RD_ERR_NONFINITE, RD_ERR_STATE = 1, 5, 6, 7


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1907_07774_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


@pytest.fixture(scope="module")
def case():
    prob = synth.calibration_problem(n=(16, 16, 32), nt=4, m=2, sigma=2 * math.pi / 8)
    M = orc.model_from_problem(prob, rtol=1e-13, maxit=1000, kind="numpy")
    c_true, _ = M.forward(prob.p_true, prob.k_f_true, prob.rho_f_true)
    d = synth.labels(c_true, synth.ellipsoid_mask(prob.n), prob.seed + 7)
    J, g, c1, _ = M.gradient(prob.p, prob.k_f, prob.rho_f, d)
    return prob, d, J, g, c1


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def check_recovered(ctx, case, prec):
    prob, d, J_or, g_or, _ = case
    J, g = ctx.rd_gradient(prob.p, prob.k_f, prob.rho_f)
    assert abs(J - J_or) <= TOL[prec] * abs(J_or)
    assert rel(g, g_or) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_iteration_cap_reports_noconv_and_keeps_the_iterate(prec, case):
    prob, d, J_or, g_or, c1_or = case
    ctx = R.context_for(prob, prec=prec, pcg_rtol=RTOL[prec], pcg_maxit=1)
    ctx.rd_set_data(d)
    c1 = np.full(prob.n, np.nan)
    with pytest.raises(R.RDError, match="RD_ERR_NOCONV"):
        ctx.rd_forward(prob.p, prob.k_f, prob.rho_f, c1)
    # the iterate after the capped solves is written: finite and near c(1)
    assert np.isfinite(c1).all()
    assert rel(c1, c1_or) < 0.5
    assert "pcg_maxit" in ctx.rd_last_error()
    assert ctx.rd_forward(prob.p, prob.k_f, prob.rho_f, c1, allow_noconv=True) is not None
    assert ctx.rd_last_pcg_iters() == ctx.rd_last_pcg_solves()      # one iteration per solve
    J, g = ctx.rd_gradient(prob.p, prob.k_f, prob.rho_f, allow_noconv=True)
    assert np.isfinite(J) and np.isfinite(g).all()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_nan_in_tissue_map_reports_nonfinite_then_context_recovers(prec, case):
    prob, d, *_ = case
    ctx = R.context_for(prob, prec=prec, pcg_rtol=RTOL[prec], pcg_maxit=1000)
    ctx.rd_set_data(d)
    check_recovered(ctx, case, prec)      # graphs built and warm before the fault
    bad = prob.m_wm.copy()
    bad[8, 8, 16] = np.nan                # inside the brain region
    ctx.rd_set_tissue(bad, prob.m_gm, prob.m_csf)
    with pytest.raises(R.RDError, match="RD_ERR_NONFINITE"):
        ctx.rd_gradient(prob.p, prob.k_f, prob.rho_f)
    ctx.rd_set_tissue(prob.m_wm, prob.m_gm, prob.m_csf)
    check_recovered(ctx, case, prec)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_nan_in_data_reports_nonfinite_then_context_recovers(prec, case):
    prob, d, *_ = case
    ctx = R.context_for(prob, prec=prec, pcg_rtol=RTOL[prec], pcg_maxit=1000)
    bad = d.copy()
    bad[8, 8, 16] = np.nan
    ctx.rd_set_data(torch.from_numpy(bad).cuda())      # device copy of the host array
    with pytest.raises(R.RDError, match="RD_ERR_NONFINITE"):
        ctx.rd_gradient(prob.p, prob.k_f, prob.rho_f)
    ctx.rd_set_data(d)
    check_recovered(ctx, case, prec)


def test_non_finite_parameters_are_rejected_on_the_host(case):
    """A NaN Gaussian weight would be skipped by the basis synthesis (terms
    below its cut-off are dropped), so the host arrays are checked first."""
    prob, d, *_ = case
    ctx = R.context_for(prob, prec="fp64", pcg_rtol=1e-12, pcg_maxit=1000)
    ctx.rd_set_data(d)
    p = prob.p.copy()
    p[0] = np.nan
    with pytest.raises(R.RDError, match="RD_ERR_ARG"):
        ctx.rd_gradient(p, prob.k_f, prob.rho_f)
    with pytest.raises(R.RDError, match="RD_ERR_ARG"):
        ctx.rd_forward(p, prob.k_f, prob.rho_f)
    v = np.zeros(len(p) + 2)
    v[-1] = np.inf
    with pytest.raises(R.RDError, match="RD_ERR_ARG"):
        ctx.rd_hessvec(prob.p, prob.k_f, prob.rho_f, v)
    with pytest.raises(R.RDError, match="RD_ERR_ARG"):
        ctx.rd_gradient(prob.p, math.inf, prob.rho_f)
    check_recovered(ctx, case, "fp64")


def test_null_and_misaligned_pointers_are_rejected_before_any_launch(case):
    prob, d, *_ = case
    ctx = R.context_for(prob, prec="fp64", pcg_rtol=1e-12, pcg_maxit=1000)
    L = R.lib()
    buf = torch.zeros(prob.n[0] * prob.n[1] * prob.n[2] + 1, dtype=torch.float64, device="cuda")
    good = buf.data_ptr()
    odd = good + 4                        # a device address not aligned to FP64
    assert L.rd_set_tissue(ctx.h, None, good, good) == RD_ERR_ARG
    assert L.rd_set_tissue(ctx.h, odd, good, good) == RD_ERR_ARG
    assert L.rd_set_data(ctx.h, odd) == RD_ERR_ARG
    assert L.rd_apply_operator(ctx.h, 0.05, odd, good) == RD_ERR_ARG
    assert L.rd_apply_precond(ctx.h, 0.05, good, odd) == RD_ERR_ARG
    assert L.rd_apply_precond(ctx.h, math.inf, good, good) == RD_ERR_ARG
    J = np.zeros(1)
    pv = np.ascontiguousarray(prob.p)
    assert L.rd_forward(ctx.h, pv.ctypes.data, 0.05, 6.0, odd, J.ctypes.data_as(R._c_double_p)) == RD_ERR_ARG
    assert L.rd_forward(ctx.h, pv.ctypes.data, math.nan, 6.0, None,
                        J.ctypes.data_as(R._c_double_p)) == RD_ERR_ARG
    assert L.rd_adjoint(ctx.h, odd) == RD_ERR_ARG
    # a gradient before rd_set_data is a state error, not a launch
    g = np.zeros(len(prob.p) + 2)
    assert L.rd_gradient(ctx.h, pv.ctypes.data, 0.05, 6.0, J.ctypes.data_as(R._c_double_p),
                         g.ctypes.data) == RD_ERR_STATE
    ctx.rd_set_data(d)
    check_recovered(ctx, case, "fp64")


def test_bounded_wait_gives_up_and_reports_timeout_then_context_works(case):
    """The mbarrier wait of the TMA passes with a transaction that no copy
    completes: it gives up after its poll limit and reports the timeout code;
    with a copy in flight it completes.  The context stays usable."""
    status = torch.full((1,), 99, dtype=torch.int32, device="cuda")
    src = torch.arange(4, dtype=torch.int32, device="cuda") + 17
    assert R.rd_selftest_bounded_wait(1 << 14, 0, None, status) == R.RD_OK
    torch.cuda.synchronize()
    assert int(status.item()) == 7        # kStTimeout, reported as "a TMA wait timed out"
    status.fill_(99)
    assert R.rd_selftest_bounded_wait(1 << 20, 1, src, status) == R.RD_OK
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert R.rd_selftest_bounded_wait(0, 0, None, status) == RD_ERR_ARG
    assert R.rd_selftest_bounded_wait(100, 1, None, status) == RD_ERR_ARG
    prob, d, *_ = case
    ctx = R.context_for(prob, prec="mixed", pcg_rtol=1e-6, pcg_maxit=1000)
    ctx.rd_set_data(d)
    check_recovered(ctx, case, "mixed")
