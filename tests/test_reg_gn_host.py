"""Host logic of the registration Gauss-Newton-Krylov solve, driven by the
FP64 oracle (CPU): PCG against a dense solve, and misfit reduction on a
small problem whose patient anatomy is the atlas transported by a known
divergence-free velocity."""

import math

import numpy as np

from oracle import reg as G
from paper_1907_07774_gb300 import reg_gn
from paper_1907_07774_gb300 import synth


class OracleSolver:
    """The oracle behind the rg_* call names the solver uses."""

    def __init__(self, R):
        self.R = R

    def rg_gradient(self, v):
        return self.R.gradient(v)

    def rg_hessvec(self, v, vt):
        return self.R.hessvec(v, vt)

    def rg_apply_precond(self, r):
        return self.R.precond(r)

    def rg_forward(self, v):
        return self.R.objective(v)


def test_pcg_matches_a_dense_solve():
    rng = np.random.default_rng(1)
    n = 12
    A = rng.standard_normal((n, n))
    A = A @ A.T + n * np.eye(n)
    Mi = np.diag(1.0 / np.diag(A))
    b = [rng.standard_normal(4), rng.standard_normal(4), rng.standard_normal(4)]
    flat = lambda xs: np.concatenate(xs)
    split = lambda y: [y[0:4], y[4:8], y[8:12]]
    x, used = reg_gn.pcg(lambda p: split(A @ flat(p)), lambda r: split(Mi @ flat(r)), b, 1.0, 1e-12, 50)
    assert np.allclose(flat(x), np.linalg.solve(A, flat(b)), rtol=1e-9, atol=1e-10)
    assert used <= n


def test_gauss_newton_recovers_most_of_a_known_transport():
    n, nt = (16, 16, 16), 2
    prob = synth.registration_problem(n=n, nt=nt, seed=4500, disp_amp=0.0, q_amp=0.0, beta_v=1e-3)
    # patient = atlas transported by the problem's test velocity, no tumor
    truth = G.Registration(n, prob.m_atlas, prob.m_atlas, np.zeros(n), None, nt, 1e-3)
    mP = truth.forward(prob.v)[-1]
    R = G.Registration(n, prob.m_atlas, mP, np.zeros(n), None, nt, 1e-3)
    zero = [np.zeros(n) for _ in range(3)]
    J0 = R.objective(zero)
    res = reg_gn.gauss_newton(OracleSolver(R), zero, R.g.h3, iters=4, cg_maxit=8)
    assert len(res.history) >= 2
    objs = [J0] + [h["objective"] for h in res.history]
    assert all(b < a for a, b in zip(objs, objs[1:]))
    assert res.objective < 0.2 * J0
    # the recovered velocity points the way of the true one
    cosang = sum(float(np.vdot(a, b)) for a, b in zip(res.v, prob.v)) / math.sqrt(
        sum(float(np.vdot(a, a)) for a in res.v) * sum(float(np.vdot(b, b)) for b in prob.v))
    assert cosang > 0.7


def test_beta_continuation_schedule():
    from paper_1907_07774_gb300.picard import beta_schedule
    s = beta_schedule(1e-1, 1e-3, final_repeats=2)
    assert np.allclose(s, [1e-1, 1e-2, 1e-3, 1e-3])
    assert beta_schedule(1e-3, 1e-3, final_repeats=2) == [1e-3, 1e-3]
