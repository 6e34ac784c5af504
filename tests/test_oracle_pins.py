"""Pins of the FP64 oracle against things other than itself: closed forms,
textbook special cases, brute force and finite differences (CPU only)."""

import math

import numpy as np
import pytest

from oracle import fft as F
from oracle import rd
from paper_1907_07774_gb300 import synth

TWO_PI = 2.0 * math.pi


def coords(n):
    x = synth.grid_coords(n)
    return (x[0][:, None, None], x[1][None, :, None], x[2][None, None, :])


# ---------------------------------------------------------------- transforms
def test_dense_dft_of_plane_wave_is_a_delta():
    n = 8
    j = np.arange(n)
    for m in range(n):
        x = np.exp(2j * np.pi * m * j / n)
        X = F.dft_dense(x, 0)
        want = np.zeros(n, complex)
        want[m] = n                  # forward sign exp(-2 pi i n k / N)
        assert np.abs(X - want).max() < 1e-12


@pytest.mark.parametrize("shape", [(8, 8, 8), (12, 6, 9), (16, 4, 2)])
def test_recursive_fft_matches_dense_dft(shape):
    rng = np.random.default_rng(1)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    a = F.fftn(x, kind="recursive")
    b = F.fftn(x, kind="dense")
    assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max() * 10
    ai = F.fftn(a, inverse=True, kind="recursive")
    assert np.abs(ai - x).max() < 1e-13


def test_recursive_fft_matches_library_and_parseval():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((16, 32, 8)) + 1j * rng.standard_normal((16, 32, 8))
    a = F.fftn(x)
    assert np.abs(a - np.fft.fftn(x)).max() < 1e-11
    assert abs(np.sum(abs(a) ** 2) / x.size - np.sum(abs(x) ** 2)) < 1e-9 * np.sum(abs(x) ** 2)


# ------------------------------------------------------------------ operator
def test_operator_on_single_mode_with_constant_kappa():
    n = (16, 16, 16)
    sp = rd.Spectral(n)
    x0, x1, x2 = coords(n)
    k = (1, 2, 3)
    u = np.cos(k[0] * x0 + k[1] * x1 + k[2] * x2)
    au = sp.A(u, 0.7 * np.ones(n))
    assert np.abs(au + 0.7 * 14 * u).max() < 1e-12


def test_operator_variable_kappa_closed_form():
    """Band-limited u and kappa: the spectral operator is exact, so it must
    equal grad(kappa).grad(u) + kappa lap(u) written out by hand."""
    n = (16, 12, 20)
    sp = rd.Spectral(n)
    x0, x1, x2 = coords(n)
    u = np.sin(x0) * np.cos(2 * x1) + np.cos(3 * x2 + x0)
    ux0 = np.cos(x0) * np.cos(2 * x1) - np.sin(3 * x2 + x0)
    ux1 = -2 * np.sin(x0) * np.sin(2 * x1)
    ux2 = -3 * np.sin(3 * x2 + x0)
    lap = -np.sin(x0) * np.cos(2 * x1) - np.cos(3 * x2 + x0) \
        - 4 * np.sin(x0) * np.cos(2 * x1) - 9 * np.cos(3 * x2 + x0)
    kap = 2.0 + np.cos(x0) + 0.5 * np.sin(x1 + x2)
    k0 = -np.sin(x0)
    k1 = 0.5 * np.cos(x1 + x2)
    k2 = 0.5 * np.cos(x1 + x2)
    want = k0 * ux0 + k1 * ux1 + k2 * ux2 + kap * lap
    got = sp.A(u, kap)
    assert np.abs(got - want).max() < 1e-11


def test_operator_symmetric_negative_semidefinite_mass_free():
    n = (8, 12, 16)
    sp = rd.Spectral(n)
    rng = np.random.default_rng(3)
    u, v = rng.standard_normal(n), rng.standard_normal(n)
    kap = rng.uniform(0.0, 1.0, n)
    au, av = sp.A(u, kap), sp.A(v, kap)
    assert abs(np.vdot(v, au) - np.vdot(av, u)) < 1e-12 * np.abs(au).sum()
    assert np.vdot(u, au) < 0
    assert abs(au.sum()) < 1e-10


def test_nyquist_mode_has_zero_derivative():
    n = (8, 8, 8)
    sp = rd.Spectral(n)
    x0, _, _ = coords(n)
    u = np.cos(4 * x0) * np.ones(n)
    assert max(np.abs(g).max() for g in sp.grad(u)) < 1e-13


def test_operator_brute_force_dense_solve():
    """PCG on (I - s A) against a dense solve of the matrix assembled column
    by column from the operator (brute force, 4x6x4 grid)."""
    n = (4, 6, 4)
    sp = rd.Spectral(n)
    rng = np.random.default_rng(4)
    kap = rng.uniform(0.0, 2.0, n)
    s = 0.3
    N = int(np.prod(n))
    M = np.zeros((N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        M[:, j] = e - s * sp.A(e.reshape(n), kap).ravel()
    assert np.abs(M - M.T).max() < 1e-12
    assert np.linalg.eigvalsh(M).min() >= 1.0 - 1e-12
    b = rng.standard_normal(n)
    want = np.linalg.solve(M, b.ravel()).reshape(n)
    got, it, rr = rd.pcg(lambda x: x - s * sp.A(x, kap),
                         lambda r: sp.precond(r, s * kap.mean()), b, b, 1e-14, 200)
    assert np.abs(got - want).max() < 1e-12


# ------------------------------------------------------------ time stepping
def _model(n, nt, kappa1=None, rho1=None, kind="recursive", **kw):
    prob = synth.calibration_problem(n=n, nt=nt, m=2, sigma=TWO_PI / 12)
    M = rd.model_from_problem(prob, kind=kind, **kw)
    if kappa1 is not None:
        M.kappa1 = kappa1
    if rho1 is not None:
        M.rho1 = rho1
    return M, prob


def test_cn_single_mode_amplification_and_one_pcg_iteration():
    n = (16, 16, 16)
    x0, x1, x2 = coords(n)
    M, _ = _model(n, nt=5, kappa1=np.ones(n), rho1=np.zeros(n))
    k = (2, 1, 3)
    u0 = 0.3 * np.cos(k[0] * x0 + k[1] * x1 + k[2] * x2)
    M.iters = []
    k_f = 0.02
    c1, _ = M.forward(np.zeros(8), k_f, 0.0, c0=u0)
    a = M.s * k_f * 14
    g = ((1 - a) / (1 + a)) ** 5
    assert np.abs(c1 - g * u0).max() < 1e-13
    assert all(i == 1 for i in M.iters)


def test_reaction_only_matches_logistic_closed_form():
    n = (8, 8, 8)
    rng = np.random.default_rng(5)
    rho1 = rng.uniform(0.0, 1.0, n)
    M, _ = _model(n, nt=7, rho1=rho1)
    c0 = rng.uniform(0.05, 0.95, n)
    c1, _ = M.forward(None, 0.0, 9.0, c0=c0)
    want = c0 / (c0 + (1 - c0) * np.exp(-9.0 * rho1))
    assert np.abs(c1 - want).max() < 1e-13


def test_constant_state_diffusion_inert():
    n = (8, 8, 8)
    M, _ = _model(n, nt=4, rho1=np.ones(n))
    c0 = 0.2 * np.ones(n)
    c1, _ = M.forward(None, 0.07, 3.0, c0=c0)
    want = 0.2 / (0.2 + 0.8 * math.exp(-3.0))
    assert np.abs(c1 - want).max() < 1e-13


def test_pure_diffusion_conserves_mass():
    n = (16, 16, 16)
    M, prob = _model(n, nt=6)
    c0 = M.phi(prob.p_true)
    c1, _ = M.forward(None, 0.1, 0.0, c0=c0)
    assert abs(c1.sum() - c0.sum()) < 1e-11 * c0.sum()


def test_smooth_state_stays_in_unit_interval():
    """Resolved data (wide Gaussians, constant coefficients): 0 <= c <= 1.
    With the ellipsoid mask kappa jumps at the brain surface and the
    spectral CN step undershoots slightly, so the invariant is only pinned
    for smooth coefficients."""
    n = (16, 16, 16)
    prob = synth.calibration_problem(n=n, nt=8, m=2, sigma=TWO_PI / 6)
    M = rd.model_from_problem(prob, kind="numpy")
    M.kappa1 = np.ones(n)
    M.rho1 = np.ones(n)
    c1, _ = M.forward(prob.p_true, 0.05, 5.0)
    assert c1.min() > -1e-10 and c1.max() < 1 + 1e-10


def test_logistic_derivative_matches_difference_quotient():
    c = np.linspace(0.01, 0.99, 50)
    rho, t, e = 7.0, 0.3, 1e-6
    fd = (rd.logistic(c + e, rho, t) - rd.logistic(c - e, rho, t)) / (2 * e)
    assert np.abs(fd - rd.logistic_dc(c, rho, t)).max() < 1e-8
    # the flow solves dL/dt = rho L (1 - L)
    fdt = (rd.logistic(c, rho, t + e) - rd.logistic(c, rho, t - e)) / (2 * e)
    L = rd.logistic(c, rho, t)
    assert np.abs(fdt - rho * L * (1 - L)).max() < 1e-7


# ------------------------------------------------------------ Gaussian basis
def test_gaussian_basis_peak_and_periodic_wrap():
    n = (16, 16, 16)
    h = TWO_PI / 16
    sig = 0.4
    cen = np.array([[3 * h, 8 * h, 0.0]])
    g = rd.gaussian_factors(n, cen, sig)
    G = rd.phi(np.ones(1), g)
    assert abs(G[3, 8, 0] - 1.0) < 1e-15
    assert abs(G[3, 8, 15] - math.exp(-h * h / (2 * sig * sig))) < 1e-15
    assert abs(G[3, 8, 1] - G[3, 8, 15]) < 1e-15
    assert abs(G[5, 7, 0] - math.exp(-(4 * h * h + h * h) / (2 * sig * sig))) < 1e-15
    u = np.random.default_rng(6).standard_normal(n)
    assert abs(rd.phi_t(u, g)[0] - np.sum(G * u)) < 1e-12


# --------------------------------------------------- adjoint and derivatives
@pytest.fixture(scope="module")
def small_problem():
    prob = synth.calibration_problem(n=16, nt=8, m=2, sigma=TWO_PI / 8)
    M = rd.model_from_problem(prob, kind="numpy", rtol=1e-13)
    c1, _ = M.forward(prob.p_true, prob.k_f_true, prob.rho_f_true)
    d = synth.labels(c1, synth.ellipsoid_mask(prob.n), 7)
    th = np.concatenate([prob.p, [prob.k_f, prob.rho_f]])
    return M, prob, d, th


def _J(M, d, th):
    c1, _ = M.forward(th[:-2], th[-2], th[-1])
    return M.misfit(c1, d, th[:-2])


def test_gradient_matches_central_differences(small_problem):
    M, prob, d, th = small_problem
    J, g, _, _ = M.gradient(th[:-2], th[-2], th[-1], d)
    dirs = list(synth.random_directions(3, len(th), 11))
    for i in (0, len(th) - 2, len(th) - 1):
        e = np.zeros(len(th))
        e[i] = 1.0
        dirs.append(e)
    for v in dirs:
        eps = 1e-6
        fd = (_J(M, d, th + eps * v) - _J(M, d, th - eps * v)) / (2 * eps)
        assert abs(fd - g @ v) <= 1e-6 * max(abs(fd), 1e-3 * np.linalg.norm(g))


def test_gradient_taylor_remainder_is_second_order(small_problem):
    M, prob, d, th = small_problem
    J0, g, _, _ = M.gradient(th[:-2], th[-2], th[-1], d)
    v = synth.random_directions(1, len(th), 12)[0]
    rem = []
    for eps in (1e-1, 5e-2, 2.5e-2, 1.25e-2):
        rem.append(abs(_J(M, d, th + eps * v) - J0 - eps * (g @ v)))
    ratios = [rem[i] / rem[i + 1] for i in range(3)]
    assert all(3.0 < r < 5.0 for r in ratios), ratios


def test_adjoint_dot_product(small_problem):
    """<w, J v>_{h^3} = v . J^T w with J = dc(1)/d(p, k_f, rho_f)."""
    M, prob, d, th = small_problem
    c1, traj = M.forward(th[:-2], th[-2], th[-1])
    v = synth.random_directions(1, len(th), 13)[0]
    w = np.random.default_rng(14).standard_normal(prob.n)
    jv = M.tangent(traj, v, th[-2], th[-1])
    a0, gk, gr = M.adjoint(traj, -w, th[-2], th[-1])
    jtw = np.concatenate([-M.h3 * M.phi_t(a0), [gk, gr]])
    lhs = M.h3 * float(np.sum(w * jv))
    assert abs(lhs - jtw @ v) < 1e-9 * abs(lhs)


def test_gauss_newton_hessian_symmetric_and_matches_gradient_differences(small_problem):
    M, prob, _, th = small_problem
    c1, _ = M.forward(th[:-2], th[-2], th[-1])
    d0 = c1.copy()   # zero residual: the GN Hessian is the exact Hessian
    v, w = synth.random_directions(2, len(th), 15)
    hv = M.hessvec(th[:-2], th[-2], th[-1], v)
    hw = M.hessvec(th[:-2], th[-2], th[-1], w)
    assert abs(v @ hw - w @ hv) < 1e-10 * abs(v @ hw)
    assert v @ hv > 0 and w @ hw > 0
    eps = 1e-5
    gp = M.gradient(th[:-2] + eps * v[:-2], th[-2] + eps * v[-2], th[-1] + eps * v[-1], d0)[1]
    gm = M.gradient(th[:-2] - eps * v[:-2], th[-2] - eps * v[-2], th[-1] - eps * v[-1], d0)[1]
    fd = (gp - gm) / (2 * eps)
    assert np.linalg.norm(fd - hv) < 1e-7 * np.linalg.norm(hv)


def test_misfit_quadrature_weight():
    M, prob = _model((8, 8, 8), nt=1)
    c = np.full(prob.n, 0.5)
    d = np.zeros(prob.n)
    assert abs(M.misfit(c, d, np.zeros(8)) - 0.5 * 0.25 * (TWO_PI ** 3)) < 1e-12


@pytest.fixture(scope="module")
def moving_atlas_problem(small_problem):
    M, prob, d, th = small_problem
    import copy
    Mm = copy.copy(M)
    rng = np.random.default_rng(41)
    Mm.set_anatomy_data([np.clip(mi + 0.1 * rng.standard_normal(prob.n), 0, 1) * (mi > 0) for mi in Mm.m])
    return Mm, prob, d, th


def test_moving_atlas_gradient_matches_central_differences(moving_atlas_problem):
    """D_c + D_m objective: the extra final condition m^T (m (1 - c) - m_D)."""
    M, prob, d, th = moving_atlas_problem
    J, g, _, _ = M.gradient(th[:-2], th[-2], th[-1], d)
    J0 = _J(M, d, th)
    assert abs(J - J0) < 1e-14 * J0
    for v in list(synth.random_directions(2, len(th), 42)) + [np.eye(len(th))[-2]]:
        eps = 1e-6
        fd = (_J(M, d, th + eps * v) - _J(M, d, th - eps * v)) / (2 * eps)
        assert abs(fd - g @ v) <= 1e-6 * max(abs(fd), 1e-3 * np.linalg.norm(g))


def test_moving_atlas_term_changes_objective_and_hessian(moving_atlas_problem, small_problem):
    M, prob, d, th = moving_atlas_problem
    M0 = small_problem[0]
    assert _J(M, d, th) > _J(M0, d, th)
    c1, _ = M.forward(th[:-2], th[-2], th[-1])
    d0 = c1.copy()
    # with zero tumor residual the remaining D_m residual keeps the GN Hessian
    # symmetric positive: check symmetry with the weight 1 + sum m_i^2
    v, w = synth.random_directions(2, len(th), 43)
    hv = M.hessvec(th[:-2], th[-2], th[-1], v)
    hw = M.hessvec(th[:-2], th[-2], th[-1], w)
    assert abs(v @ hw - w @ hv) < 1e-10 * abs(v @ hw) and v @ hv > 0


def test_moving_atlas_gauss_newton_hessian_is_exact_at_zero_residual(small_problem):
    """With d = c(1) and m_D = m (1 - c(1)) both residuals vanish, so the
    Gauss-Newton Hessian equals the true Hessian: H v must match central
    differences of the reduced gradient, which fixes the final weight
    1 + sum_i m_i^2 of the tangent c(1)."""
    import copy
    M0, prob, _, th = small_problem
    M = copy.copy(M0)
    c1, _ = M.forward(th[:-2], th[-2], th[-1])
    M.set_anatomy_data([mi * (1.0 - c1) for mi in M.m])
    d = c1.copy()
    v = synth.random_directions(1, len(th), 44)[0]
    hv = M.hessvec(th[:-2], th[-2], th[-1], v)
    eps = 1e-5
    gp = M.gradient(*(lambda t: (t[:-2], t[-2], t[-1]))(th + eps * v), d)[1]
    gm = M.gradient(*(lambda t: (t[:-2], t[-2], t[-1]))(th - eps * v), d)[1]
    fd = (gp - gm) / (2 * eps)
    assert np.linalg.norm(fd - hv) <= 1e-5 * np.linalg.norm(hv)
    # the plain tumor weight would miss the anatomy term
    M1 = copy.copy(M0)
    hv1 = M1.hessvec(th[:-2], th[-2], th[-1], v)
    assert np.linalg.norm(fd - hv1) > 1e-2 * np.linalg.norm(hv)


def _tissue_perturbation(n, seed):
    """Smooth seeded field: a few random periodic Gaussians."""
    rng = np.random.default_rng(seed)
    x = synth.grid_coords(n)
    out = np.zeros(n)
    for _ in range(3):
        c = rng.uniform(0, TWO_PI, 3)
        r2 = 0.0
        for a in range(3):
            dx = np.abs(x[a] - c[a])
            dx = np.minimum(dx, TWO_PI - dx)
            shape = [1, 1, 1]
            shape[a] = n[a]
            r2 = r2 + (dx ** 2).reshape(shape)
        out += rng.standard_normal() * np.exp(-r2 / (2 * 0.8 ** 2))
    return out


def test_coupling_field_is_the_derivative_through_the_coefficients(small_problem):
    """q(x) of the Picard step (Sec. 2.2): perturbing tissue class i inside
    the coefficients k and f only (Eq. coeff_tumor) by eps dm must change the
    objective by eps h^3 sum_x q_i dm at first order.  Checked per class, so a
    swapped weight index, a dropped diffusion or reaction term or a wrong sign
    each fails."""
    M, prob, d, th = small_problem
    p, k_f, rho_f = th[:-2], th[-2], th[-1]
    ms = [prob.m_wm, prob.m_gm, prob.m_csf]

    def J_with(i, dm):
        mm = [m.copy() for m in ms]
        mm[i] = mm[i] + dm
        Mi = rd.Model(prob.n, *mm, prob.centers, prob.sigma, prob.nt, k_w=(1.0, 0.1, 0.3),
                      rho_w=(1.0, 0.2, 0.05), kind="numpy", rtol=1e-13)
        c1, _ = Mi.forward(p, k_f, rho_f)
        return Mi.misfit(c1, d, p)

    # non-zero CSF weights so every class is exercised
    M3 = rd.Model(prob.n, *ms, prob.centers, prob.sigma, prob.nt, k_w=(1.0, 0.1, 0.3),
                  rho_w=(1.0, 0.2, 0.05), kind="numpy", rtol=1e-13)
    q = M3.coupling(p, k_f, rho_f, d)
    eps = 1e-4
    for i in range(3):
        dm = _tissue_perturbation(prob.n, 60 + i)
        fd = (J_with(i, eps * dm) - J_with(i, -eps * dm)) / (2 * eps)
        lin = M3.h3 * float(np.sum(q[i] * dm))
        assert abs(fd - lin) <= 1e-6 * abs(lin), (i, fd, lin)


def test_coupling_field_euler_identity(small_problem):
    """k and f are linear in m, so h^3 sum_x sum_i m_i q_i equals
    k_f dJ/dk_f + rho_f dJ/drho_f; with zero CSF weights q_CSF vanishes."""
    M, prob, d, th = small_problem
    p, k_f, rho_f = th[:-2], th[-2], th[-1]
    q = M.coupling(p, k_f, rho_f, d)
    _, g, _, _ = M.gradient(p, k_f, rho_f, d)
    lhs = M.h3 * sum(float(np.sum(mi * qi)) for mi, qi in zip(M.m, q))
    rhs = k_f * g[-2] + rho_f * g[-1]
    assert abs(lhs - rhs) <= 1e-12 * abs(rhs)
    assert np.all(q[2] == 0.0)


def test_threaded_library_fft_matches_the_recursive_fft():
    """The "scipy" kind (library transform on several threads, used to shorten
    long oracle runs) agrees with the oracle's own recursive FFT."""
    from oracle import fft as F
    rng = np.random.default_rng(9)
    x = rng.standard_normal((8, 12, 6)) + 1j * rng.standard_normal((8, 12, 6))
    old = F.SCIPY_WORKERS
    try:
        F.SCIPY_WORKERS = 2
        for inv in (False, True):
            want = F.fftn(x, inverse=inv, kind="recursive")
            got = F.fftn(x, inverse=inv, kind="scipy")
            assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()
    finally:
        F.SCIPY_WORKERS = old
