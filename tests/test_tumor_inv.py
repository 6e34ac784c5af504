"""Host logic of the tumor inversion solver (l1 GIST phase with the Hoyer
beta search, weighted-l2 L-BFGS phase with the More-Thuente line search),
pinned by closed forms: the Lasso optimality conditions, the prox of the
l1 norm, dense BFGS updates, the strong Wolfe conditions, a ridge solution
and scipy's L-BFGS-B optimum."""

import math

import numpy as np
import pytest

from paper_1907_07774_gb300 import tumor_inv as T


class FakeSolver:
    """Stands in for a context: D(p, k_f) = 1/2 |G p + k_f u + k_f^2 v - b|^2
    with the rd_forward / rd_gradient / rd_adjoint calls of the library."""

    def __init__(self, G, b, u=None, v=None):
        self.G, self.b = np.asarray(G, float), np.asarray(b, float)
        self.np = self.G.shape[1]
        m = self.G.shape[0]
        self.u = np.zeros(m) if u is None else np.asarray(u, float)
        self.v = np.zeros(m) if v is None else np.asarray(v, float)
        self.last = None
        self.forwards = 0

    def _res(self, p, k_f):
        return self.G @ p + k_f * self.u + k_f * k_f * self.v - self.b

    def rd_forward(self, p, k_f, rho_f):
        self.forwards += 1
        p = np.asarray(p, float)
        self.last = (p.copy(), float(k_f))
        r = self._res(p, k_f)
        return 0.5 * float(r @ r)

    def rd_adjoint(self):
        p, k_f = self.last
        r = self._res(p, k_f)
        return np.concatenate([self.G.T @ r, [float(r @ (self.u + 2 * k_f * self.v)), 0.0]])

    def rd_gradient(self, p, k_f, rho_f):
        J = self.rd_forward(p, k_f, rho_f)
        return J, self.rd_adjoint()


def _sparse_problem(m=60, n=40, k=3, seed=0, noise=0.01):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((m, n)) / math.sqrt(m)
    x = np.zeros(n)
    x[rng.choice(n, k, replace=False)] = rng.uniform(1, 2, k) * rng.choice([-1, 1], k)
    b = G @ x + noise * rng.standard_normal(m)
    return G, b, x


# ------------------------------------------------------------- closed forms
def test_hoyer_closed_forms():
    n = 17
    e = np.zeros(n)
    e[4] = -3.0
    assert T.hoyer(e) == 1.0
    assert T.hoyer(np.ones(n)) == pytest.approx(0.0, abs=1e-15)
    for k in (2, 5, 11):
        p = np.zeros(n)
        p[:k] = 2.5
        assert T.hoyer(p) == pytest.approx((n - k) / (n - 1), rel=1e-14)
    p = np.random.default_rng(1).standard_normal(n)
    assert T.hoyer(7.0 * p) == pytest.approx(T.hoyer(p), rel=1e-14)
    assert T.hoyer(np.zeros(n)) == 1.0


def test_soft_threshold_is_the_prox_of_the_l1_norm():
    """argmin_p 1/2 (p - x)^2 + t |p|, by brute force on a fine grid."""
    rng = np.random.default_rng(2)
    grid = np.linspace(-5, 5, 200001)
    for x, t in zip(rng.uniform(-4, 4, 20), rng.uniform(0, 2, 20)):
        brute = grid[np.argmin(0.5 * (grid - x) ** 2 + t * np.abs(grid))]
        assert abs(T.soft_threshold(np.array([x]), t)[0] - brute) <= 1e-4


def test_l2_weights_threshold():
    p = np.array([0.0, 0.05, -0.2, 1.0, -0.09, 0.1])
    w = T.l2_weights(p, 0.1, 5.0, 0.5)
    assert np.array_equal(w, [5.0, 5.0, 0.5, 0.5, 5.0, 0.5])


# ---------------------------------------------------------------- GIST
def test_gist_reaches_the_lasso_optimum():
    """First-order conditions of min 1/2 |G p - b|^2 + beta |p|_1:
    g_i = -beta sign(p_i) on the support, |g_i| <= beta off it."""
    G, b, _ = _sparse_problem()
    s = FakeSolver(G, b)
    beta = 0.05
    r = T.gist(s, np.zeros(s.np), 0.0, 0.0, beta, tau_j=1e-22, maxit=5000, nonneg=False)
    _, g = s.rd_gradient(r.p, 0.0, 0.0)
    g = g[:s.np]
    on = r.p != 0.0
    assert on.any() and (~on).any()
    assert np.max(np.abs(g[on] + beta * np.sign(r.p[on]))) <= 1e-6
    assert np.max(np.abs(g[~on])) <= beta * (1 + 1e-6)
    objs = [h["objective"] for h in r.history]
    assert all(b_ <= a_ + 1e-15 for a_, b_ in zip(objs, objs[1:]))


def test_gist_nonnegative_reaches_its_optimality_conditions():
    """min 1/2 |G p - b|^2 + beta |p|_1 s.t. p >= 0:
    g_i = -beta where p_i > 0, g_i >= -beta where p_i = 0."""
    G, b, _ = _sparse_problem(seed=12)
    s = FakeSolver(G, b)
    beta = 0.02
    r = T.gist(s, np.zeros(s.np), 0.0, 0.0, beta, tau_j=1e-22, maxit=5000)
    assert np.all(r.p >= 0.0)
    _, g = s.rd_gradient(r.p, 0.0, 0.0)
    g = g[:s.np]
    on = r.p > 0.0
    assert on.any()
    assert np.max(np.abs(g[on] + beta)) <= 1e-6
    assert np.min(g[~on]) >= -beta * (1 + 1e-6)
    assert np.array_equal(T.soft_threshold(np.array([-2.0, 0.5, 3.0]), 1.0, nonneg=True), [0.0, 0.0, 2.0])


def test_gist_with_beta_above_the_gradient_bound_stays_at_zero():
    """For beta >= |grad D(0)|_inf the zero vector is optimal."""
    G, b, _ = _sparse_problem(seed=3)
    s = FakeSolver(G, b)
    _, g0 = s.rd_gradient(np.zeros(s.np), 0.0, 0.0)
    r = T.gist(s, np.zeros(s.np), 0.0, 0.0, 1.0001 * np.max(np.abs(g0[:s.np])), maxit=20)
    assert not np.any(r.p)


def test_beta_search_finds_a_sparse_solution_and_brackets_the_target():
    G, b, x = _sparse_problem(m=80, n=60, k=2, seed=4, noise=0.05)
    s = FakeSolver(G, b)
    res = T.beta_search(s, np.zeros(s.np), 0.0, 0.0, target=0.95, steps=10,
                        tau_j=1e-16, maxit=2000, nonneg=False)
    assert np.any(res.p) and res.sparsity >= 0.95
    sparse = [t["beta"] for t in res.tried if t["nnz"] > 0 and t["sparsity"] >= 0.95]
    assert res.beta == min(sparse)
    # every tried beta below the result was too dense
    assert all(t["sparsity"] < 0.95 for t in res.tried if t["beta"] < res.beta)
    # the two largest entries are the true support
    assert set(np.argsort(-np.abs(res.p))[:2]) == set(np.flatnonzero(x))


# ------------------------------------------------------------ line search
def _check_wolfe(phi, f0, g0, r, ftol, gtol):
    f, g = phi(r.stp)
    assert f <= f0 + ftol * r.stp * g0
    assert abs(g) <= gtol * abs(g0)


def _line(f, df, x0, d):
    return lambda a: (f(x0 + a * d), float(df(x0 + a * d) @ d))


def _softplus(z):
    return max(z, 0.0) + math.log1p(math.exp(-abs(z)))


def _sigmoid(z):
    return 1 / (1 + math.exp(-z)) if z >= 0 else math.exp(z) / (1 + math.exp(z))


def _rosen(x):
    return float(np.sum(100.0 * (x[1:] - x[:-1] ** 2) ** 2 + (1 - x[:-1]) ** 2))


def _rosen_grad(x):
    g = np.zeros_like(x)
    g[:-1] = -400.0 * x[:-1] * (x[1:] - x[:-1] ** 2) - 2 * (1 - x[:-1])
    g[1:] += 200.0 * (x[1:] - x[:-1] ** 2)
    return g


@pytest.mark.parametrize("gtol", [0.9, 0.1, 0.01])
@pytest.mark.parametrize("stp0", [1e-3, 1.0, 1e3])
def test_more_thuente_returns_strong_wolfe_steps(gtol, stp0):
    x0 = np.array([-1.2, 1.0, 0.5])
    phis = [
        lambda a: ((a - 2.0) ** 2 - 4.0, 2.0 * (a - 2.0)),
        lambda a: (-a * math.exp(-a), (a - 1.0) * math.exp(-a)),
        lambda a: (0.1 * math.sin(5 * a) - a + 0.3 * a * a, 0.5 * math.cos(5 * a) - 1.0 + 0.6 * a),
        _line(_rosen, _rosen_grad, x0, -_rosen_grad(x0)),
        lambda a: (_softplus(3 - 4 * a) + 0.05 * a * a, -4 * _sigmoid(3 - 4 * a) + 0.1 * a),
    ]
    for phi in phis:
        f0, g0 = phi(0.0)
        r = T.more_thuente(phi, f0, g0, stp=stp0, ftol=1e-4, gtol=gtol, xtol=1e-12, maxfev=60)
        assert r.status == "wolfe", (r, gtol, stp0)
        _check_wolfe(phi, f0, g0, r, 1e-4, gtol)
        # with a coarse interval tolerance the search may stop early, but
        # always at a point of sufficient decrease
        r = T.more_thuente(phi, f0, g0, stp=stp0, ftol=1e-4, gtol=gtol, xtol=0.1, maxfev=60)
        assert r.status in ("wolfe", "xtol") and r.f <= f0 + 1e-4 * r.stp * g0


def test_more_thuente_stops_at_stpmax_on_an_unbounded_line():
    r = T.more_thuente(lambda a: (-a, -1.0), 0.0, -1.0, stp=1.0, stpmax=5.0)
    assert r.status == "stpmax" and r.stp == 5.0


# ---------------------------------------------------------------- L-BFGS
def test_two_loop_recursion_equals_dense_bfgs_updates():
    rng = np.random.default_rng(5)
    n = 8
    A = rng.standard_normal((n, n))
    A = A @ A.T + n * np.eye(n)
    S = [rng.standard_normal(n) for _ in range(5)]
    Y = [A @ s for s in S]
    g = rng.standard_normal(n)
    gamma = float(S[-1] @ Y[-1]) / float(Y[-1] @ Y[-1])
    H = gamma * np.eye(n)
    for s, y in zip(S, Y):
        r = 1.0 / float(y @ s)
        V = np.eye(n) - r * np.outer(y, s)
        H = V.T @ H @ V + r * np.outer(s, s)
    assert np.allclose(T.lbfgs_direction(g, S, Y), -H @ g, rtol=1e-12, atol=1e-12)
    assert np.array_equal(T.lbfgs_direction(g, [], []), -g)


def test_lbfgs_matches_scipy_on_rosenbrock():
    scipy_opt = pytest.importorskip("scipy.optimize")
    x0 = np.array([-1.2, 1.0, -0.5, 0.8, 1.3, -0.7])
    r = T.lbfgs(lambda x: (_rosen(x), _rosen_grad(x)), x0, m=10, maxit=500, gtol_rel=1e-10)
    ref = scipy_opt.minimize(_rosen, x0, jac=_rosen_grad, method="L-BFGS-B",
                             options={"gtol": 1e-12, "ftol": 1e-15, "maxiter": 2000})
    assert r.converged
    assert np.allclose(r.x, ref.x, atol=1e-6) and np.allclose(r.x, 1.0, atol=1e-6)
    fs = [h["f"] for h in r.history]
    assert all(b <= a for a, b in zip(fs, fs[1:]))


def test_lbfgs_respects_a_lower_bound():
    fg = lambda x: ((x[0] + 1) ** 2 + (x[1] - 2) ** 2 + 0.5 * x[0] * x[1],
                    np.array([2 * (x[0] + 1) + 0.5 * x[1], 2 * (x[1] - 2) + 0.5 * x[0]]))
    r = T.lbfgs(fg, np.array([3.0, 0.0]), lower=np.array([0.0, -np.inf]), maxit=50, gtol_rel=1e-9)
    assert r.converged
    assert r.x[0] == pytest.approx(0.0, abs=1e-12)
    assert r.x[1] == pytest.approx(2.0, abs=1e-6)


def test_weighted_l2_phase_reaches_the_ridge_solution():
    """Linear model in (p, k_f): the optimum of
    1/2 |G p + k_f u - b|^2 + beta/2 sum w p^2 solves a normal system."""
    G, b, x = _sparse_problem(m=50, n=12, k=3, seed=6)
    rng = np.random.default_rng(7)
    u = rng.standard_normal(50)
    kf_true = 0.3
    b = b + kf_true * u
    s = FakeSolver(G, b, u=u)
    w = T.l2_weights(x, 0.1, 10.0, 0.1)
    beta = 0.02
    res, scale = T.weighted_l2(s, np.zeros(12), 0.05, 0.0, beta, w, opttol=1e-10, maxit=400, nonneg=False)
    th = res.x * scale
    M = np.column_stack([G, u])
    reg = np.diag(np.concatenate([beta * w, [0.0]]))
    want = np.linalg.solve(M.T @ M + reg, M.T @ b)
    assert res.converged
    assert np.allclose(th[:13], want, atol=1e-7)


def test_weighted_l2_keeps_k_f_nonnegative():
    G, b, _ = _sparse_problem(m=40, n=10, k=2, seed=8)
    u = np.random.default_rng(9).standard_normal(40)
    s = FakeSolver(G, b - 0.5 * u, u=u)        # the unconstrained k_f would be -0.5
    res, scale = T.weighted_l2(s, np.zeros(10), 0.1, 0.0, 1e-3, np.ones(10), opttol=1e-8, maxit=200,
                               nonneg=False)
    th = res.x * scale
    assert res.converged
    assert th[10] == 0.0 and res.g[10] > 0.0
    # on the face k_f = 0 the optimum is the ridge solution in p alone
    want = np.linalg.solve(G.T @ G + 1e-3 * np.eye(10), G.T @ (b - 0.5 * u))
    assert np.allclose(th[:10], want, atol=1e-6)


def test_tumor_inversion_runs_both_phases():
    G, b, x = _sparse_problem(m=80, n=30, k=2, seed=10, noise=0.02)
    rng = np.random.default_rng(11)
    u = 0.3 * rng.standard_normal(80)
    v = 0.1 * rng.standard_normal(80)
    s = FakeSolver(G, b + 0.2 * u + 0.04 * v, u=u, v=v)
    out = T.tumor_inversion(s, rho_f=0.0, k_f_l2=0.05, beta_steps=8, gist_kw={"tau_j": 1e-14, "maxit": 500},
                            tau_s=0.1, w_large=1.0, w_small=0.0, beta_l2=1e-3, opttol=1e-6, l2_maxit=300,
                            nonneg=False)
    assert out.sparsity >= 0.95
    assert out.l2.converged and out.k_f >= 0.0
    J0 = s.rd_forward(out.l1.p, 0.0, 0.0)
    assert out.misfit < J0
    assert abs(out.k_f - 0.2) < 0.1


class _NonFinite(RuntimeError):
    status = 6


class BlowUpSolver(FakeSolver):
    """Fails like the library's RD_ERR_NONFINITE beyond k_f = 0.4."""

    def rd_forward(self, p, k_f, rho_f):
        if k_f > 0.4:
            raise _NonFinite("non-finite value in a PCG solve")
        return super().rd_forward(p, k_f, rho_f)


def test_nonfinite_trials_shorten_the_step_instead_of_failing():
    G, b, _ = _sparse_problem(m=40, n=8, k=2, seed=13)
    u = np.random.default_rng(14).standard_normal(40)
    s = BlowUpSolver(G, b + 0.3 * u, u=u)
    res, scale = T.weighted_l2(s, np.zeros(8), 0.01, 0.0, 1e-4, np.ones(8), opttol=1e-8, maxit=300,
                               k_f_scale=1.0, nonneg=False)
    th = res.x * scale
    assert res.converged and abs(th[8] - 0.3) < 0.05
    # GIST treats a failing trial as a rejected step and halves alpha
    class BigP(FakeSolver):
        def rd_forward(self, p, k_f, rho_f):
            if np.max(np.abs(p)) > 0.5:
                raise _NonFinite("non-finite value in a PCG solve")
            return super().rd_forward(p, k_f, rho_f)

    s2 = BigP(G, b)
    r = T.gist(s2, np.zeros(8), 0.0, 0.0, 0.01, alpha0=1e3, maxit=5, nonneg=False)
    assert r.history and r.history[0]["alpha"] < 1e3 and np.max(np.abs(r.p)) <= 0.5


def test_lbfgs_keeps_p_nonnegative_by_default():
    G, b, x = _sparse_problem(m=60, n=10, k=3, seed=15)
    s = FakeSolver(G, b)
    res, scale = T.weighted_l2(s, np.abs(x), 0.0, 0.0, 1e-3, np.ones(10), opttol=1e-7, maxit=300)
    th = res.x * scale
    assert res.converged and np.all(th[:10] >= 0.0)
    # projected-gradient optimality on the face p >= 0
    g = res.g / scale
    free = th[:10] > 0
    assert np.max(np.abs(g[:10][free])) <= 1e-6 * np.linalg.norm(G.T @ b)
    assert np.all(g[:10][~free] >= -1e-9)


def test_auto_k_f_scaling_moves_a_weakly_coupled_diffusivity():
    """When dJ/dk_f is tiny next to dJ/dp, the automatic scale lets the
    first quasi-Newton steps move k_f: within a few iterations it gets much
    closer to the ridge optimum than with the fixed scale."""
    G, b, x = _sparse_problem(m=50, n=12, k=3, seed=16)
    u = 1e-3 * np.random.default_rng(17).standard_normal(50)
    kf_true = 40.0
    s = FakeSolver(G, b + kf_true * u, u=u)
    w = np.ones(12)
    beta = 1e-3
    M = np.column_stack([G, u])
    want = np.linalg.solve(M.T @ M + np.diag(np.concatenate([beta * w, [0.0]])), M.T @ (b + kf_true * u))
    errs = {}
    for ks in (None, "auto"):
        res, scale = T.weighted_l2(s, np.zeros(12), 1.0, 0.0, beta, w, opttol=1e-12, maxit=6, nonneg=False,
                                   k_f_scale=ks)
        errs[ks] = abs((res.x * scale)[12] - want[12])
    assert errs["auto"] < 0.1 * errs[None], errs
