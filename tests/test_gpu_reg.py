"""Registration path (include/rg.h) through the C ABI against the FP64
oracle (oracle/reg.py), element by element on the same seeded inputs.

Tolerances: relative L2 <= 1e-10 for the FP64 path and <= 2e-4 for the
mixed path (FP32 fields, FP64 reductions): both sides run the same
semi-Lagrangian scheme, so the difference is rounding only."""

import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import reg as G
from paper_1907_07774_gb300 import rg as RG
from paper_1907_07774_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-10, "mixed": 2e-4}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1907_07774_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def rel(a, b):
    a = np.concatenate([np.ravel(x) for x in a]) if isinstance(a, (list, tuple)) else np.ravel(a)
    b = np.concatenate([np.ravel(x) for x in b]) if isinstance(b, (list, tuple)) else np.ravel(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def oracle_for(prob):
    return G.Registration(prob.n, prob.m_atlas, prob.m_patient, prob.c1, prob.q, prob.nt, prob.beta_v)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("n", [(16, 16, 16), (8, 32, 16), (16, 96, 16)])
def test_projection_and_preconditioner_match_oracle(prec, n):
    g = G.Grid(n)
    rng = np.random.default_rng(7)
    w = [rng.standard_normal(n) for _ in range(3)]
    ctx = RG.RegContext(n, 2, prec=prec, beta_v=0.3)
    kw = ctx.rg_project(w)
    assert rel(kw, g.leray(w)) <= TOL[prec]
    R = G.Registration(n, [np.zeros(n)] * 3, [np.zeros(n)] * 3, np.zeros(n), None, 2, beta_v=0.3)
    z = ctx.rg_apply_precond(w)
    assert rel(z, R.precond(w)) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("n,nt", [((16, 16, 16), 4), ((8, 32, 16), 3), ((16, 96, 16), 2)])
def test_forward_matches_oracle(prec, n, nt):
    prob = synth.registration_problem(n=n, nt=nt, seed=4100)
    R = oracle_for(prob)
    lv = R.forward(prob.v)
    J_or = R.objective(prob.v, lv)
    ctx = RG.context_for(prob, prec)
    m1 = [np.zeros(n) for _ in range(3)]
    J = ctx.rg_forward(prob.v, m1)
    assert rel(m1, lv[-1]) <= TOL[prec]
    assert abs(J - J_or) <= TOL[prec] * abs(J_or)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_gradient_and_hessvec_match_oracle(prec):
    prob = synth.registration_problem(n=16, nt=4, seed=4200)
    R = oracle_for(prob)
    J_or, g_or = R.gradient(prob.v)
    hv_or = R.hessvec(prob.v, prob.directions[0])
    ctx = RG.context_for(prob, prec)
    J, g = ctx.rg_gradient(prob.v)
    assert abs(J - J_or) <= TOL[prec] * abs(J_or)
    assert rel(g, g_or) <= TOL[prec]
    hv = ctx.rg_hessvec(prob.v, prob.directions[0])
    assert rel(hv, hv_or) <= TOL[prec]


def test_device_buffers_and_no_coupling_field():
    prob = synth.registration_problem(n=(16, 16, 32), nt=2, seed=4300)
    R = G.Registration(prob.n, prob.m_atlas, prob.m_patient, prob.c1, None, prob.nt, prob.beta_v)
    J_or, g_or = R.gradient(prob.v)
    ctx = RG.RegContext(prob.n, prob.nt, prec="fp64", beta_v=prob.beta_v)
    dev = lambda xs: [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in xs]
    ctx.rg_set_images(dev(prob.m_atlas), dev(prob.m_patient), dev([prob.c1])[0], None)
    gd = [torch.zeros(prob.n, dtype=torch.float64, device="cuda") for _ in range(3)]
    J, _ = ctx.rg_gradient(dev(prob.v), gd)
    assert abs(J - J_or) <= 1e-10 * abs(J_or)
    assert rel([x.cpu().numpy() for x in gd], g_or) <= 1e-10


def test_whole_cell_transport_is_an_exact_shift_on_the_gpu():
    n, nt = (16, 16, 16), 4
    h = [2 * math.pi / k for k in n]
    cells = (1, -2, 1)
    v = [np.full(n, cells[a] * h[a] * nt) for a in range(3)]
    rng = np.random.default_rng(9)
    mA = [rng.standard_normal(n) for _ in range(3)]
    ctx = RG.RegContext(n, nt, prec="fp64", beta_v=1.0)
    ctx.rg_set_images(mA, mA, np.zeros(n), None)
    m1 = [np.zeros(n) for _ in range(3)]
    ctx.rg_forward(v, m1)
    tot = tuple(nt * c for c in cells)
    for i in range(3):
        assert np.abs(m1[i] - np.roll(mA[i], shift=tot, axis=(0, 1, 2))).max() < 1e-12


def test_gradient_is_divergence_free_and_projection_idempotent():
    prob = synth.registration_problem(n=32, nt=2, seed=4400)
    ctx = RG.context_for(prob, "fp64")
    _, g = ctx.rg_gradient(prob.v)
    grid = G.Grid(prob.n)
    assert np.abs(grid.div(g)).max() < 1e-9 * max(np.abs(x).max() for x in g)
    kg = ctx.rg_project(g)
    assert rel(kg, g) < 1e-12


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_gauss_newton_on_the_gpu_reduces_the_misfit(prec):
    """Patient = atlas transported (on the GPU) by a known divergence-free
    velocity; Gauss-Newton-Krylov from v = 0 brings the objective down."""
    from paper_1907_07774_gb300 import reg_gn
    n, nt = (32, 32, 32), 2
    prob = synth.registration_problem(n=n, nt=nt, seed=4600, disp_amp=0.0, q_amp=0.0, beta_v=1e-3)
    gen = RG.RegContext(n, nt, prec="fp64", beta_v=1e-3)
    gen.rg_set_images(prob.m_atlas, prob.m_atlas, np.zeros(n), None)
    mP = [np.zeros(n) for _ in range(3)]
    gen.rg_forward(prob.v, mP)
    ctx = RG.RegContext(n, nt, prec=prec, beta_v=1e-3)
    ctx.rg_set_images(prob.m_atlas, mP, np.zeros(n), None)
    zero = [np.zeros(n) for _ in range(3)]
    J0 = ctx.rg_forward(zero)
    h3 = (2 * math.pi) ** 3 / np.prod(n)
    res = reg_gn.gauss_newton(ctx, zero, h3, iters=4, cg_maxit=8)
    objs = [J0] + [h["objective"] for h in res.history]
    assert len(objs) >= 3 and all(b < a for a, b in zip(objs, objs[1:]))
    assert res.objective < 0.2 * J0
