"""Host logic of the Gauss-Newton-Krylov loop on small analytic problems
(CPU only; the solver is a stand-in exposing the same calls)."""

import numpy as np

from paper_1907_07774_gb300 import gn


class LeastSquares:
    """J = 1/2 |r(theta)|^2 with Jacobian-based GN products."""

    def __init__(self, r, jac, npar):
        self.r, self.jac, self.np = r, jac, npar
        self.last = None

    def rd_forward(self, p, k_f, rho_f):
        th = np.concatenate([p, [k_f, rho_f]])
        self.last = th
        return 0.5 * float(self.r(th) @ self.r(th))

    def rd_adjoint(self):
        th = self.last
        return self.jac(th).T @ self.r(th)

    def rd_gradient(self, p, k_f, rho_f):
        J = self.rd_forward(p, k_f, rho_f)
        return J, self.rd_adjoint()

    def rd_hessvec(self, p, k_f, rho_f, v):
        th = np.concatenate([p, [k_f, rho_f]])
        Jm = self.jac(th)
        return Jm.T @ (Jm @ v)


def test_cg_solves_spd_system_exactly():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((6, 6))
    H = A @ A.T + 6 * np.eye(6)
    b = rng.standard_normal(6)
    x, used = gn.cg(lambda v: H @ v, b, 50, 1e-14)
    assert np.allclose(H @ x, b, atol=1e-10) and used <= 7


def test_linear_least_squares_converges_to_the_lstsq_solution():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((20, 5))
    want = np.array([0.3, -0.2, 0.5, 0.05, 7.0])        # k_f slot (index 3) positive
    b = A @ want + 1e-3 * rng.standard_normal(20)
    want = np.linalg.lstsq(A, b, rcond=None)[0]
    prob = LeastSquares(lambda th: A @ th - b, lambda th: A, 3)
    th0 = np.array([0.1, 0.2, 0.3, 0.4, 0.5])
    res = gn.gauss_newton(prob, th0, iters=20, cg_maxit=20)
    assert np.allclose(res.theta, want, atol=1e-8)


def test_nonlinear_fit_decreases_monotonically():
    t = np.linspace(0, 1, 40)
    truth = np.array([1.5, 0.8, 2.0, 0.3])   # a e^{-b t} + c t + d  (last two play k_f, rho_f)

    def model(th):
        return th[0] * np.exp(-th[1] * t) + th[2] * t + th[3]

    def jac(th):
        e = np.exp(-th[1] * t)
        return np.stack([e, -th[0] * t * e, t, np.ones_like(t)], axis=1)

    data = model(truth)
    prob = LeastSquares(lambda th: model(th) - data, jac, 2)
    res = gn.gauss_newton(prob, np.array([1.0, 0.3, 1.0, 0.5]), iters=25, cg_maxit=10)
    Js = [h["misfit"] for h in res.history]
    J0 = 0.5 * float(np.sum((model(np.array([1.0, 0.3, 1.0, 0.5])) - data) ** 2))
    assert Js[0] < J0 and all(b <= a for a, b in zip(Js, Js[1:]))
    assert Js[-1] < 1e-4 * J0


def test_line_search_keeps_k_f_nonnegative():
    # the unconstrained minimiser has k_f < 0; every accepted iterate stays feasible
    prob = LeastSquares(lambda th: np.array([th[0] - 1.0, th[1] + 2.0, th[2] - 3.0]),
                        lambda th: np.eye(3), 1)
    res = gn.gauss_newton(prob, np.array([0.0, 0.5, 0.0]), iters=5, cg_maxit=5)
    assert res.theta[1] >= 0.0


class _NonFinite(RuntimeError):
    status = 6


def test_non_finite_trial_solves_are_rejected_steps():
    """A full Newton step that makes the solve blow up (as a negative
    initial concentration does) is halved instead of ending the run."""
    rng = np.random.default_rng(2)
    A = rng.standard_normal((20, 5))
    want = np.array([0.3, -0.2, 0.5, 0.05, 7.0])
    b = A @ want
    base = LeastSquares(lambda th: A @ th - b, lambda th: A, 3)
    th0 = np.array([0.1, 0.2, 0.3, 0.4, 0.5])

    class Fragile(LeastSquares):
        calls = 0

        def rd_forward(self, p, k_f, rho_f):
            Fragile.calls += 1
            if Fragile.calls == 2:          # the first line-search trial
                raise _NonFinite("non-finite value in a PCG solve")
            return super().rd_forward(p, k_f, rho_f)

    prob = Fragile(base.r, base.jac, 3)
    J0 = base.rd_forward(th0[:3], th0[3], th0[4])
    res = gn.gauss_newton(prob, th0, iters=30, cg_maxit=20)
    assert res.history[0]["step"] == 0.5 and res.history[0]["line_search"] == 2
    assert res.misfit < 1e-6 * J0


def test_fixed_parameter_stays_and_the_rest_solves_the_reduced_problem():
    """With rho_f held (the paper's protocol: invert for p and k_f at a fixed
    proliferation rate) the loop leaves it untouched and converges to the
    least-squares solution over the other parameters."""
    rng = np.random.default_rng(4)
    A = rng.standard_normal((30, 5))
    b = rng.standard_normal(30)
    prob = LeastSquares(lambda th: A @ th - b, lambda th: A, 3)
    th0 = np.array([0.1, 0.2, 0.3, 0.4, 2.5])
    res = gn.gauss_newton(prob, th0, iters=30, cg_maxit=20, fixed=(4,))
    assert res.theta[4] == 2.5
    free = A[:, :4]
    want = np.linalg.lstsq(free, b - A[:, 4] * 2.5, rcond=None)[0]
    if want[3] >= 0:                                      # k_f bound inactive
        assert np.allclose(res.theta[:4], want, atol=1e-8)
