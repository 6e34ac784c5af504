"""CUDA path (through the C ABI) against the FP64 oracle, element by element.

Tolerances: relative L2 <= 1e-10 for the FP64 path (both sides solve the
CN systems to 1e-12) and <= 2e-4 for the mixed path (FP32 fields, FP64
reductions), on c(1), fields and gradients.
"""

import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import rd as orc
from paper_1907_07774_gb300 import rd as R
from paper_1907_07774_gb300 import synth

pytestmark = pytest.mark.gpu
TWO_PI = 2.0 * math.pi
TOL = {"fp64": 1e-10, "mixed": 2e-4}
RTOL = {"fp64": 1e-12, "mixed": 1e-6}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1907_07774_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def coords(n):
    x = synth.grid_coords(n)
    return (x[0][:, None, None], x[1][None, :, None], x[2][None, None, :])


def small_problem(n, nt, m=2, sigma=TWO_PI / 8, seed=1000):
    return synth.calibration_problem(n=n, nt=nt, m=m, sigma=sigma, seed=seed)


def oracle_for(prob, **kw):
    return orc.model_from_problem(prob, rtol=1e-13, maxit=1000, kind="numpy", **kw)


def gpu_for(prob, prec, **kw):
    return R.context_for(prob, prec=prec, pcg_rtol=RTOL[prec], pcg_maxit=1000, **kw)


# --------------------------------------------------------------- kernels
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("n", [(16, 32, 64), (256, 8, 16), (8, 128, 8), (96, 16, 32), (16, 96, 96)])
def test_operator_single_mode_closed_form(prec, n):
    x0, x1, x2 = coords(n)
    k = (1, 2, 3)
    u = np.cos(k[0] * x0 + k[1] * x1 + k[2] * x2) * np.ones(n)
    one, zero = np.ones(n), np.zeros(n)
    ctx = R.Context(n, 4, 1, prec=prec, k_w=(1, 0, 0), rho_w=(1, 0, 0))
    ctx.rd_set_tissue(one, zero, zero)
    out = np.zeros(n)
    ctx.rd_apply_operator(0.3, u, out)
    want = -0.3 * 14 * u
    # round-off of a spectral second derivative grows with the largest
    # resolved |k|^2: bound 16 eps k_f sum_a (n_a / 2)^2 max|u|
    eps = {"fp64": 2.2e-16, "mixed": 1.2e-7}[prec]
    bound = 16 * eps * 0.3 * sum((m / 2) ** 2 for m in n) * np.abs(u).max()
    assert np.abs(out - want).max() <= bound


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("n", [(16, 16, 16), (8, 16, 32), (32, 32, 32), (96, 8, 32), (16, 96, 96)])
def test_operator_and_preconditioner_match_oracle(prec, n):
    prob = small_problem(n, 4)
    M = oracle_for(prob)
    ctx = gpu_for(prob, prec)
    rng = np.random.default_rng(3)
    u = rng.standard_normal(n)
    k_f = 0.07
    out = np.zeros(n)
    ctx.rd_apply_operator(k_f, u, out)
    assert rel(out, M.A(u, k_f)) <= TOL[prec]
    z = np.zeros(n)
    ctx.rd_apply_precond(k_f, u, z)
    want = M.sp.precond(u, M.s * k_f * orc.kbar_positive(M.kappa1))
    assert rel(z, want) <= TOL[prec]


def test_operator_and_preconditioner_at_256_match_oracle():
    """The benchmark grid (256^3, its tissue maps and k_f): one operator
    application and one preconditioner application through the kernels the
    benchmark runs (TMA row and strided passes at L = 256), in both
    precisions, against the oracle on a field with smooth and rough parts."""
    prob = synth.calibration_problem(n=256, nt=32, m=5)
    M = orc.model_from_problem(prob, kind="numpy")
    rng = np.random.default_rng(11)
    u = M.phi(prob.p) + 0.1 * rng.standard_normal(prob.n)
    want_a = M.A(u, prob.k_f)
    want_z = M.sp.precond(u, M.s * prob.k_f * orc.kbar_positive(M.kappa1))
    for prec in ("fp64", "mixed"):
        ctx = gpu_for(prob, prec)
        out = np.zeros(prob.n)
        ctx.rd_apply_operator(prob.k_f, u, out)
        assert rel(out, want_a) <= TOL[prec], prec
        z = np.zeros(prob.n)
        ctx.rd_apply_precond(prob.k_f, u, z)
        assert rel(z, want_z) <= TOL[prec], prec
        del ctx


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_operator_where_kappa_vanishes_on_whole_tiles(prec):
    """The TMA operator passes visit only the tiles where kappa is not
    identically zero: kappa zero on a slab and on the whole box (no tile left),
    and nonzero only on one column of voxels, against the oracle."""
    n = (64, 32, 64)
    x0, x1, x2 = coords(n)
    rng = np.random.default_rng(5)
    u = rng.standard_normal(n)
    smooth = (1.2 + np.cos(x0) * np.sin(2 * x1) * np.cos(x2)) * np.ones(n)
    cases = {"slab": smooth * (np.abs(x0 - np.pi) < 1.0),
             "zero": np.zeros(n),
             "column": np.where((np.abs(x1 - np.pi) < 0.1) & (np.abs(x2 - 1.0) < 0.1), smooth, 0.0)}
    zero = np.zeros(n)
    for name, m in cases.items():
        ctx = R.Context(n, 4, 1, prec=prec, k_w=(1, 0, 0), rho_w=(1, 0, 0))
        ctx.rd_set_tissue(m, zero, zero)
        out = np.full(n, np.nan)
        ctx.rd_apply_operator(0.3, u, out)
        want = orc.Spectral(n, "numpy").A(u, 0.3 * m)
        if name == "zero":
            assert np.all(out == 0.0), name
        else:
            assert rel(out, want) <= TOL[prec], name


# ---------------------------------------------------------------- solves
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("n,nt", [((16, 16, 16), 4), ((8, 16, 32), 3), ((8, 8, 8), 2), ((32, 96, 16), 3)])
def test_forward_matches_oracle(prec, n, nt):
    prob = small_problem(n, nt)
    M = oracle_for(prob)
    c_or, _ = M.forward(prob.p_true, prob.k_f_true, prob.rho_f_true)
    ctx = gpu_for(prob, prec)
    c1 = np.zeros(n)
    ctx.rd_forward(prob.p_true, prob.k_f_true, prob.rho_f_true, c1)
    assert rel(c1, c_or) <= TOL[prec]
    # device output buffer
    c1d = torch.zeros(n, dtype=torch.float64, device="cuda")
    ctx.rd_forward(prob.p_true, prob.k_f_true, prob.rho_f_true, c1d)
    assert rel(c1d.cpu().numpy(), c_or) <= TOL[prec]


def _grad_case(n=(16, 16, 16), nt=4):
    prob = small_problem(n, nt)
    M = oracle_for(prob)
    c_true, _ = M.forward(prob.p_true, prob.k_f_true, prob.rho_f_true)
    d = synth.labels(c_true, synth.ellipsoid_mask(prob.n), 7)
    return prob, M, d


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("n", [(16, 16, 16), (96, 16, 32)])
def test_gradient_matches_oracle(prec, n):
    prob, M, d = _grad_case(n=n)
    J_or, g_or, _, a0_or = M.gradient(prob.p, prob.k_f, prob.rho_f, d)
    ctx = gpu_for(prob, prec)
    ctx.rd_set_data(d)
    J, g = ctx.rd_gradient(prob.p, prob.k_f, prob.rho_f)
    assert abs(J - J_or) <= TOL[prec] * abs(J_or)
    assert rel(g, g_or) <= TOL[prec]
    # rd_forward + rd_adjoint gives the same gradient and alpha(0)
    ctx.rd_forward(prob.p, prob.k_f, prob.rho_f)
    a0 = np.zeros(prob.n)
    g2 = ctx.rd_adjoint(a0)
    assert rel(g2, g_or) <= TOL[prec]
    assert rel(a0, a0_or) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_hessvec_matches_oracle(prec):
    prob, M, d = _grad_case()
    v = synth.random_directions(1, len(prob.p) + 2, 21)[0]
    hv_or = M.hessvec(prob.p, prob.k_f, prob.rho_f, v)
    ctx = gpu_for(prob, prec)
    hv = ctx.rd_hessvec(prob.p, prob.k_f, prob.rho_f, v)
    assert rel(hv, hv_or) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_checkpoint_recompute_is_bitwise_identical(prec):
    """A recomputed segment repeats the forward run bit for bit: the state
    solves' extrapolated guesses restart at every segment start, so a
    store-all run that restarts them at the same period gives the same bits."""
    prob, M, d = _grad_case(nt=8)
    out = []
    for stride in (0, 3):
        ctx = gpu_for(prob, prec, ckpt_stride=stride, guess_restart=3)
        ctx.rd_set_data(d)
        out.append(ctx.rd_gradient(prob.p, prob.k_f, prob.rho_f))
        v = np.linspace(-1, 1, len(prob.p) + 2)
        out.append(ctx.rd_hessvec(prob.p, prob.k_f, prob.rho_f, v))
    assert out[0][0] == out[2][0] and np.array_equal(out[0][1], out[2][1])
    assert np.array_equal(out[1], out[3])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_state_solve_guesses_save_iterations_not_accuracy(prec):
    """The extrapolated guesses of the state solves (rd_config.guess_restart
    0) against zero starts (-1) at 64^3, nt = 16: fewer PCG iterations in the
    forward sweep, and c(1) and the gradient agree with the oracle to the
    same tolerance either way."""
    prob = synth.calibration_problem(n=64, nt=16, m=4)
    M = orc.model_from_problem(prob, rtol=1e-13, maxit=2000, kind="numpy")
    c_true, _ = M.forward(prob.p_true, prob.k_f_true, prob.rho_f_true)
    d = synth.labels(c_true, synth.ellipsoid_mask(prob.n), prob.seed + 7)
    J_or, g_or, c1_or, _ = M.gradient(prob.p, prob.k_f, prob.rho_f, d)
    iters = {}
    for gr in (-1, 0):
        ctx = gpu_for(prob, prec, guess_restart=gr)
        ctx.rd_set_data(d)
        c1 = np.zeros(prob.n)
        ctx.rd_forward(prob.p, prob.k_f, prob.rho_f, c1)
        iters[gr] = ctx.rd_last_pcg_iters()
        assert rel(c1, c1_or) <= TOL[prec]
        J, g = ctx.rd_gradient(prob.p, prob.k_f, prob.rho_f)
        assert abs(J - J_or) <= TOL[prec] * abs(J_or) and rel(g, g_or) <= TOL[prec]
    assert iters[0] < iters[-1], iters


def test_graph_and_host_driven_solves_are_bitwise_identical():
    """PCG solves run as CUDA graphs with a device-side loop once a context
    is warm; with launch timing on they run host-driven.  Same bits."""
    prob, M, d = _grad_case(nt=6)
    ctx = gpu_for(prob, "mixed")
    ctx.rd_set_data(d)
    ctx.rd_gradient(prob.p, prob.k_f, prob.rho_f)          # warm: graph built
    J1, g1 = ctx.rd_gradient(prob.p, prob.k_f, prob.rho_f)
    it1 = ctx.rd_last_pcg_iters()
    assert ctx.rd_last_graph_solves() == ctx.rd_last_pcg_solves() > 0
    R.rd_profile_enable(True)
    try:
        J2, g2 = ctx.rd_gradient(prob.p, prob.k_f, prob.rho_f)
        it2 = ctx.rd_last_pcg_iters()
        prof = R.rd_profile_read()
    finally:
        R.rd_profile_enable(False)
    assert J1 == J2 and np.array_equal(g1, g2) and it1 == it2 > 0
    assert prof["pcg_opx"][1] == it2


def test_beta_p_regularisation_terms():
    prob, M, d = _grad_case()
    M.beta_p = 1e-2
    J_or, g_or, _, _ = M.gradient(prob.p, prob.k_f, prob.rho_f, d)
    ctx = gpu_for(prob, "fp64", beta_p=1e-2)
    ctx.rd_set_data(d)
    J, g = ctx.rd_gradient(prob.p, prob.k_f, prob.rho_f)
    assert abs(J - J_or) <= 1e-10 * J_or and rel(g, g_or) <= 1e-10


def _anatomy_data(prob, seed=41):
    rng = np.random.default_rng(seed)
    return [np.clip(mi + 0.1 * rng.standard_normal(prob.n), 0, 1) * (mi > 0)
            for mi in (prob.m_wm, prob.m_gm, prob.m_csf)]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_moving_atlas_gradient_and_hessvec_match_oracle(prec):
    """Objective D_c + D_m: misfit, adjoint final condition, alpha(0),
    gradient and the 1 + sum m_i^2 weighted Gauss-Newton product."""
    prob, M, d = _grad_case()
    md = _anatomy_data(prob)
    M.set_anatomy_data(md)
    J_or, g_or, _, a0_or = M.gradient(prob.p, prob.k_f, prob.rho_f, d)
    v = synth.random_directions(1, len(prob.p) + 2, 21)[0]
    hv_or = M.hessvec(prob.p, prob.k_f, prob.rho_f, v)
    ctx = gpu_for(prob, prec, moving_atlas=True)
    ctx.rd_set_data(d)
    J0, g0 = ctx.rd_gradient(prob.p, prob.k_f, prob.rho_f)      # before m_D: tumor misfit only
    ctx.rd_set_anatomy_data(*md)
    J, g = ctx.rd_gradient(prob.p, prob.k_f, prob.rho_f)
    assert J > J0
    assert abs(J - J_or) <= TOL[prec] * abs(J_or)
    assert rel(g, g_or) <= TOL[prec]
    a0 = np.zeros(prob.n)
    ctx.rd_forward(prob.p, prob.k_f, prob.rho_f)
    ctx.rd_adjoint(a0)
    assert rel(a0, a0_or) <= TOL[prec]
    hv = ctx.rd_hessvec(prob.p, prob.k_f, prob.rho_f, v)
    assert rel(hv, hv_or) <= TOL[prec]


def test_moving_atlas_needs_its_config_flag():
    prob, M, d = _grad_case()
    ctx = gpu_for(prob, "fp64")
    with pytest.raises(RuntimeError):
        ctx.rd_set_anatomy_data(*_anatomy_data(prob))


def test_batch_graph_sees_anatomy_data_set_after_capture():
    prob, M, d = _grad_case()
    md = _anatomy_data(prob)
    ctxs = [gpu_for(prob, "mixed", moving_atlas=True) for _ in range(2)]
    for c in ctxs:
        c.rd_set_data(d)
    th = [(prob.p, prob.k_f, prob.rho_f)] * 2
    J0, _ = R.rd_batch_gradient(ctxs, th)
    ctxs[1].rd_set_anatomy_data(*md)
    J1, g1 = R.rd_batch_gradient(ctxs, th)
    Js, gs = ctxs[1].rd_gradient(prob.p, prob.k_f, prob.rho_f)
    assert J1[0] == J0[0] and J1[1] > J0[1]
    assert J1[1] == Js and np.array_equal(g1[1], gs)


KW3, RW3 = (1.0, 0.1, 0.3), (1.0, 0.2, 0.05)   # every tissue class weighted


def _coupling_case(nt=4):
    prob, _, d = _grad_case(nt=nt)
    M = orc.Model(prob.n, prob.m_wm, prob.m_gm, prob.m_csf, prob.centers, prob.sigma, prob.nt,
                  k_w=KW3, rho_w=RW3, rtol=1e-13, maxit=1000, kind="numpy")
    return prob, M, d


def _coupling_ctx(prob, prec, **kw):
    ctx = R.Context(prob.n, prob.nt, len(prob.p), prec=prec, pcg_rtol=RTOL[prec], pcg_maxit=1000,
                    k_w=KW3, rho_w=RW3, coupling=True, **kw)
    ctx.rd_set_tissue(prob.m_wm, prob.m_gm, prob.m_csf)
    ctx.rd_set_basis(prob.centers, prob.sigma)
    return ctx


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_coupling_field_matches_oracle(prec):
    prob, M, d = _coupling_case()
    q_or = M.coupling(prob.p, prob.k_f, prob.rho_f, d)
    ctx = _coupling_ctx(prob, prec)
    ctx.rd_set_data(d)
    with pytest.raises(RuntimeError):
        ctx.rd_coupling_field()                       # no gradient yet
    ctx.rd_gradient(prob.p, prob.k_f, prob.rho_f)
    q = ctx.rd_coupling_field()
    for i in range(3):
        assert rel(q[i], q_or[i]) <= TOL[prec], i
    # a Hessian-vector product at the same parameters leaves q alone
    v = synth.random_directions(1, len(prob.p) + 2, 22)[0]
    ctx.rd_hessvec(prob.p, prob.k_f, prob.rho_f, v)
    q2 = ctx.rd_coupling_field()
    assert all(np.array_equal(a, b) for a, b in zip(q, q2))
    # device outputs
    qd = [torch.zeros(prob.n, dtype=torch.float64, device="cuda") for _ in range(3)]
    ctx.rd_coupling_field(*qd)
    assert all(np.array_equal(a, b.cpu().numpy()) for a, b in zip(q, qd))
    # a new forward solve invalidates it
    ctx.rd_forward(prob.p, 1.1 * prob.k_f, prob.rho_f)
    with pytest.raises(RuntimeError):
        ctx.rd_coupling_field()


def test_coupling_field_needs_its_config_flag():
    prob, M, d = _grad_case()
    ctx = gpu_for(prob, "fp64")
    ctx.rd_set_data(d)
    ctx.rd_gradient(prob.p, prob.k_f, prob.rho_f)
    with pytest.raises(RuntimeError):
        ctx.rd_coupling_field()


def test_coupling_field_checkpointed_and_batched_are_bitwise_identical():
    prob, M, d = _coupling_case(nt=8)
    out = []
    for stride in (0, 3):
        ctx = _coupling_ctx(prob, "mixed", ckpt_stride=stride, guess_restart=3)
        ctx.rd_set_data(d)
        ctx.rd_gradient(prob.p, prob.k_f, prob.rho_f)
        out.append(ctx.rd_coupling_field())
    ctxs = [_coupling_ctx(prob, "mixed", guess_restart=3) for _ in range(2)]
    for c in ctxs:
        c.rd_set_data(d)
    R.rd_batch_gradient(ctxs, [(prob.p, prob.k_f, prob.rho_f), (prob.p, 0.5 * prob.k_f, prob.rho_f)])
    out.append(ctxs[0].rd_coupling_field())
    for q in out[1:]:
        assert all(np.array_equal(a, b) for a, b in zip(out[0], q))


# ------------------------------------------------------- paper workloads
def test_forward_problem_64_fp64_matches_oracle():
    """64^3, nt = 16 forward recipe (8 Gaussians, sigma = 2 pi / 64)."""
    prob = synth.forward_problem(n=64, nt=16)
    M = orc.model_from_problem(prob, rtol=1e-12, kind="numpy")
    c_or, _ = M.forward(prob.p, prob.k_f, prob.rho_f)
    ctx = R.context_for(prob, prec="fp64", pcg_rtol=1e-12, pcg_maxit=1000)
    c1 = np.zeros(prob.n)
    ctx.rd_forward(prob.p, prob.k_f, prob.rho_f, c1)
    assert rel(c1, c_or) <= 1e-10
    mix = R.context_for(prob, prec="mixed")
    c1m = np.zeros(prob.n)
    mix.rd_forward(prob.p, prob.k_f, prob.rho_f, c1m)
    assert rel(c1m, c_or) <= 2e-4


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_gradient_64_matches_oracle(prec):
    """64^3 gradient and Hessian-vector product against the oracle (the
    TMA-staged strided passes run at this size in both precisions)."""
    prob = synth.calibration_problem(n=64, nt=4, m=3, sigma=TWO_PI / 32)
    M = oracle_for(prob)
    c_true, _ = M.forward(prob.p_true, prob.k_f_true, prob.rho_f_true)
    d = synth.labels(c_true, synth.ellipsoid_mask(prob.n), 17)
    J_or, g_or, _, _ = M.gradient(prob.p, prob.k_f, prob.rho_f, d)
    ctx = gpu_for(prob, prec)
    ctx.rd_set_data(d)
    J, g = ctx.rd_gradient(prob.p, prob.k_f, prob.rho_f)
    assert abs(J - J_or) <= TOL[prec] * abs(J_or)
    assert rel(g, g_or) <= TOL[prec]
    v = synth.random_directions(1, len(prob.p) + 2, 23)[0]
    assert rel(ctx.rd_hessvec(prob.p, prob.k_f, prob.rho_f, v), M.hessvec(prob.p, prob.k_f, prob.rho_f, v)) <= TOL[prec]


def _calibration_data(prob, ctx):
    c_true = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    ctx.rd_forward(prob.p_true, prob.k_f_true, prob.rho_f_true, c_true)
    d = synth.labels(c_true.cpu().numpy(), synth.ellipsoid_mask(prob.n), prob.seed + 7)
    return d


def test_gradient_128_central_differences_fp64():
    """128^3, nt = 16, 64 Gaussians: the FP64 gradient against central
    differences (eps = 1e-6) of the FP64 misfit on 10 seeded directions."""
    prob = synth.calibration_problem(n=128, nt=16, m=4)
    ctx = R.context_for(prob, prec="fp64", pcg_rtol=1e-12, pcg_maxit=1000)
    ctx.rd_set_data(_calibration_data(prob, ctx))
    th = np.concatenate([prob.p, [prob.k_f, prob.rho_f]])
    J0, g = ctx.rd_gradient(prob.p, prob.k_f, prob.rho_f)
    errs = []
    for v in synth.random_directions(10, len(th), 5):
        eps = 1e-6
        jp = ctx.rd_forward((th + eps * v)[:-2], *(th + eps * v)[-2:])
        jm = ctx.rd_forward((th - eps * v)[:-2], *(th - eps * v)[-2:])
        fd = (jp - jm) / (2 * eps)
        errs.append(abs(fd - g @ v) / max(abs(fd), 1e-12))
    assert max(errs) < 1e-5, errs
    mix = R.context_for(prob, prec="mixed")
    mix.rd_set_data(_calibration_data(prob, ctx))
    Jm, gm = mix.rd_gradient(prob.p, prob.k_f, prob.rho_f)
    assert rel(gm, g) <= 2e-4 and abs(Jm - J0) <= 2e-4 * J0


def test_gradient_128_mixed_repeats_bit_for_bit_with_fields_in_l2():
    """At 128^3 every FP32 field (8 MB) stays in the 129 MB L2, so a TMA
    reload of a tile buffer completes quickly after the block's threads have
    read the buffer; the reads are ordered before the reload by a proxy
    fence.  Without it the direction kernel, which reuses its two buffers
    within a tile, read a reloaded value now and then and a PCG solve did
    not converge.  Repeated gradients must agree bit for bit, take the same
    PCG iterations and converge."""
    prob = synth.calibration_problem(n=128, nt=16, m=4)
    ctx = R.context_for(prob, prec="mixed", pcg_rtol=1e-6, pcg_maxit=500)
    ctx.rd_set_data(_calibration_data(prob, ctx))
    J0, g0 = ctx.rd_gradient(prob.p, prob.k_f, prob.rho_f)
    it0 = ctx.rd_last_pcg_iters()
    assert ctx.rd_last_graph_solves() > 0
    for _ in range(4):
        J, g = ctx.rd_gradient(prob.p, prob.k_f, prob.rho_f)
        assert J == J0 and np.array_equal(g, g0)
        assert ctx.rd_last_pcg_iters() == it0


def test_gradient_256_mixed_against_fp64_and_hessian_symmetry():
    """256^3, nt = 32, 125 Gaussians (the benchmark workload): the mixed
    gradient against the FP64 gradient of the same GPU, and symmetry of the
    mixed Gauss-Newton Hessian."""
    prob = synth.calibration_problem(n=256, nt=32, m=5)
    ref = R.context_for(prob, prec="fp64", pcg_rtol=1e-10, pcg_maxit=1000)
    d = _calibration_data(prob, ref)
    ref.rd_set_data(d)
    J64, g64 = ref.rd_gradient(prob.p, prob.k_f, prob.rho_f)
    mix = R.context_for(prob, prec="mixed", ckpt_stride=6)
    mix.rd_set_data(d)
    Jm, gm = mix.rd_gradient(prob.p, prob.k_f, prob.rho_f)
    assert abs(Jm - J64) <= 2e-4 * J64
    assert rel(gm, g64) <= 2e-4
    v, w = synth.random_directions(2, len(prob.p) + 2, 9)
    hv = mix.rd_hessvec(prob.p, prob.k_f, prob.rho_f, v)
    hw = mix.rd_hessvec(prob.p, prob.k_f, prob.rho_f, w)
    assert abs(v @ hw - w @ hv) <= 1e-3 * abs(v @ hw)


# ------------------------------------------- autograd and Gauss-Newton loop
def test_autograd_function_backward_is_the_adjoint_gradient():
    from paper_1907_07774_gb300.autograd import misfit

    prob, M, d = _grad_case()
    J_or, g_or, _, _ = M.gradient(prob.p, prob.k_f, prob.rho_f, d)
    ctx = gpu_for(prob, "fp64")
    ctx.rd_set_data(d)
    p = torch.tensor(prob.p, dtype=torch.float64, device="cuda", requires_grad=True)
    kf = torch.tensor(prob.k_f, dtype=torch.float64, requires_grad=True)
    rf = torch.tensor(prob.rho_f, dtype=torch.float64, requires_grad=True)
    J = misfit(p, kf, rf, ctx)
    (2.0 * J).backward()
    g = np.concatenate([p.grad.cpu().numpy(), [kf.grad.item(), rf.grad.item()]])
    assert abs(J.item() - J_or) <= 1e-10 * J_or
    assert rel(g, 2.0 * g_or) <= 1e-10
    # another solve between forward and backward does not change the result
    J2 = misfit(p.detach().requires_grad_(True), kf, rf, ctx)
    ctx.rd_forward(prob.p_true, prob.k_f_true, prob.rho_f_true)
    kf.grad = None
    J2.backward()
    assert abs(kf.grad.item() - g_or[-2]) <= 1e-10 * abs(g_or[-2])


def test_gauss_newton_reduces_misfit_on_gpu():
    from paper_1907_07774_gb300 import gn

    prob = synth.calibration_problem(n=32, nt=8, m=3, sigma=TWO_PI / 16)
    ctx = gpu_for(prob, "mixed", beta_p=1e-4)
    c_true = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    ctx.rd_forward(prob.p_true, prob.k_f_true, prob.rho_f_true, c_true)
    ctx.rd_set_data(c_true)           # noise-free data: truth is a minimiser
    th0 = np.concatenate([prob.p, [prob.k_f, prob.rho_f]])
    J0, g0 = ctx.rd_gradient(prob.p, prob.k_f, prob.rho_f)
    res = gn.gauss_newton(ctx, th0, iters=4, cg_maxit=10)
    Js = [h["misfit"] for h in res.history]
    assert len(Js) >= 2 and Js[0] < J0 and all(b <= a for a, b in zip(Js, Js[1:]))
    assert Js[-1] < 0.5 * J0


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_gauss_newton_recovers_growth_parameters_from_noise_free_data(prec):
    """Sec. 3.1/3.2 on data the model can fit exactly: the oracle's c_true(1)
    at 64^3, unthresholded.  With the initial condition at the truth the
    Gauss-Newton loop recovers (k_f, rho_f) from (0.02, 6) to the truth
    (0.05, 10); on all parameters at once it lowers the misfit by orders of
    magnitude (the initial condition itself is not identifiable from c(1):
    many weight vectors of the overlapping Gaussians give nearly the same
    state, the ill-posedness the paper notes)."""
    from paper_1907_07774_gb300 import gn

    prob = synth.calibration_problem(n=64, nt=8, m=4, sigma=TWO_PI / 32)
    M = oracle_for(prob)
    c_true, _ = M.forward(prob.p_true, prob.k_f_true, prob.rho_f_true)
    ctx = gpu_for(prob, prec)
    ctx.rd_set_data(c_true)
    npar = len(prob.p)
    th0 = np.concatenate([prob.p_true, [prob.k_f, prob.rho_f]])
    res = gn.gauss_newton(ctx, th0, iters=8, cg_maxit=10, forcing=1e-3, fixed=tuple(range(npar)))
    assert np.array_equal(res.theta[:npar], prob.p_true)
    assert abs(res.theta[-2] - prob.k_f_true) <= 1e-3 * prob.k_f_true
    assert abs(res.theta[-1] - prob.rho_f_true) <= 1e-3 * prob.rho_f_true
    th0 = np.concatenate([prob.p, [prob.k_f, prob.rho_f]])
    J0 = ctx.rd_forward(prob.p, prob.k_f, prob.rho_f)
    res = gn.gauss_newton(ctx, th0, iters=6, cg_maxit=20, forcing=1e-3)
    assert res.misfit < 1e-2 * J0


def test_batch_gradient_of_uneven_problems_matches_single_gradients():
    """One graph launch for several contexts of different grid sizes equals
    the per-context rd_gradient results, on two calls in a row."""
    shapes = [((16, 16, 16), 4, "mixed"), ((32, 16, 16), 3, "mixed"), ((96, 16, 32), 2, "mixed"),
              ((16, 16, 16), 3, "fp64")]
    ctxs, probs = [], []
    for i, (n, nt, prec) in enumerate(shapes):
        prob = small_problem(n, nt, seed=3000 + i)
        M = oracle_for(prob)
        c_true, _ = M.forward(prob.p_true, prob.k_f_true, prob.rho_f_true)
        ctx = gpu_for(prob, prec)
        ctx.rd_set_data(synth.labels(c_true, synth.ellipsoid_mask(prob.n), i))
        ctxs.append(ctx)
        probs.append(prob)
    for scale in (1.0, 1.3):
        thetas = [(pr.p * scale, pr.k_f * scale, pr.rho_f / scale) for pr in probs]
        want = [c.rd_gradient(*t) for c, t in zip(ctxs, thetas)]
        Js, gs = R.rd_batch_gradient(ctxs, thetas)
        for (Jw, gw), J, g, c in zip(want, Js, gs, ctxs):
            assert J == Jw and np.array_equal(g, gw)
            assert c.rd_last_graph_solves() == c.rd_last_pcg_solves() > 0


def test_autotuned_grid_sizes_keep_parity():
    prob, M, d = _grad_case(n=(32, 32, 32))
    J_or, g_or, _, _ = M.gradient(prob.p, prob.k_f, prob.rho_f, d)
    ctx = gpu_for(prob, "mixed")
    ctx.rd_set_data(d)
    try:
        caps = ctx.rd_autotune(reps=2)
        assert set(caps) >= {"op_axis01", "pcg_opx", "dht_plain", "dht_sym", "dht_update"}
        assert all(shape in ("tma", "pencil") and blocks >= 0 for blocks, shape in caps.values())
        J, g = ctx.rd_gradient(prob.p, prob.k_f, prob.rho_f)
        assert rel(g, g_or) <= TOL["mixed"] and abs(J - J_or) <= TOL["mixed"] * J_or
    finally:
        R.rd_autotune_clear()


def test_preconditioner_scale_changes_convergence_not_the_result():
    prob, M, d = _grad_case(nt=4)
    J_or, g_or, _, _ = M.gradient(prob.p, prob.k_f, prob.rho_f, d)
    ctx = gpu_for(prob, "fp64")
    ctx.rd_set_data(d)
    ctx.rd_gradient(prob.p, prob.k_f, prob.rho_f)
    it1 = ctx.rd_last_pcg_iters()
    for scale in (0.3, 3.0):
        ctx.rd_set_precond_scale(scale)
        J, g = ctx.rd_gradient(prob.p, prob.k_f, prob.rho_f)
        assert abs(J - J_or) <= 1e-10 * abs(J_or) and rel(g, g_or) <= 1e-10
        assert ctx.rd_last_pcg_iters() != it1
    ctx.rd_set_precond_scale(1.0)
    ctx.rd_set_tissue(prob.m_wm, prob.m_gm, prob.m_csf)
    ctx.rd_gradient(prob.p, prob.k_f, prob.rho_f)
    assert ctx.rd_last_pcg_iters() == it1
    with pytest.raises(RuntimeError):
        ctx.rd_set_precond_scale(0.0)
