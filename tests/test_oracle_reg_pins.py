"""Pins of the registration oracle (oracle/reg.py) against closed forms and
limits, on the CPU.

The optimize-then-discretize gradient is the derivative of the discrete
objective only in the limit of fine grids, so the finite-difference pins
check convergence under refinement rather than a fixed tight tolerance."""

import math

import numpy as np

from oracle import reg as G
from paper_1907_07774_gb300 import synth

TWO_PI = 2.0 * math.pi


def _trig(n, seed, radius=1, amp=1.0):
    rng = np.random.default_rng(seed)
    return synth.TrigSum.random(rng, radius, amp=amp)(synth.coords_mesh(n))


def _divfree(n, seed, radius=1, amp=1.0):
    rng = np.random.default_rng(seed)
    pots = [synth.TrigSum.random(rng, radius, amp=amp) for _ in range(3)]
    return synth.curl_field(pots, synth.coords_mesh(n))


def _ip(g, a, b):
    return g.h3 * sum(float(np.sum(x * y)) for x, y in zip(a, b))


def _smooth_case(n, nt, seed=0, zero_res=False):
    """Smooth fields (wave vectors of norm 1) so that interpolation errors
    stay small: atlas/patient anatomy, tumor, q, a velocity, directions."""
    n3 = (n, n, n)
    g = G.Grid(n3)
    mA = [0.5 + 0.2 * _trig(n3, seed + i) for i in range(3)]
    c = 0.3 + 0.1 * _trig(n3, seed + 10)
    mP = [0.5 + 0.2 * _trig(n3, seed + 20 + i) for i in range(3)]
    q = [0.05 * _trig(n3, seed + 30 + i) for i in range(3)]
    v = _divfree(n3, seed + 40, amp=0.4)
    R = G.Registration(n3, mA, mP, c, q, nt, beta_v=1e-2)
    if zero_res:
        m1 = R.forward(v)[-1]
        R.mP = [(1.0 - c) * m for m in m1]
        R.q = [np.zeros(n3) for _ in range(3)]
    return R, v, _divfree(n3, seed + 50), _divfree(n3, seed + 60)


# ---------------------------------------------------------- interpolation
def test_lagrange_weights_reproduce_cubics():
    nodes = np.array([-1.0, 0.0, 1.0, 2.0])
    for f in np.linspace(0.0, 0.999, 17):
        w = np.array(G.lagrange_weights(f))
        for p in range(4):
            assert abs(float(w @ nodes ** p) - f ** p) < 1e-13


def test_interp_identity_shift_and_interior_cubics():
    n = (8, 10, 12)
    u = np.random.default_rng(1).standard_normal(n)
    I = G.index_grid(n)
    assert np.array_equal(G.interp(u, I), u)
    s = (1, -2, 3)
    got = G.interp(u, [I[a] + s[a] for a in range(3)])
    assert np.allclose(got, np.roll(u, shift=(-s[0], -s[1], -s[2]), axis=(0, 1, 2)), rtol=0, atol=1e-14)
    # a separable cubic polynomial in the index is reproduced away from the wrap
    poly = lambda t, c: c[0] + c[1] * t + c[2] * t ** 2 + c[3] * t ** 3
    cs = [(0.3, -1.0, 0.2, 0.05), (1.0, 0.5, -0.1, 0.01), (-0.2, 0.1, 0.03, -0.002)]
    P = poly(I[0], cs[0]) * poly(I[1], cs[1]) * poly(I[2], cs[2])
    rng = np.random.default_rng(2)
    X = [rng.uniform(1.0, k - 3.0, 50) for k in n]
    want = poly(X[0], cs[0]) * poly(X[1], cs[1]) * poly(X[2], cs[2])
    assert np.allclose(G.interp(P, X), want, rtol=1e-12, atol=1e-12)


# --------------------------------------------------------------- transport
def test_constant_velocity_with_whole_cell_steps_is_an_exact_shift():
    n, nt = (16, 16, 16), 4
    g = G.Grid(n)
    cells = (1, 2, -1)                         # cells per step
    v = [np.full(n, cells[a] * g.h[a] * nt) for a in range(3)]
    mA = [np.random.default_rng(i).standard_normal(n) for i in range(3)]
    R = G.Registration(n, mA, mA, np.zeros(n), None, nt, 1.0)
    m1 = R.forward(v)[-1]
    tot = tuple(nt * c for c in cells)
    for i in range(3):
        assert np.allclose(m1[i], np.roll(mA[i], shift=tot, axis=(0, 1, 2)), rtol=0, atol=1e-13)
    # the adjoint runs the other way
    lam = R.adjoint(v, mA)[0]
    for i in range(3):
        assert np.allclose(lam[i], np.roll(mA[i], shift=tuple(-t for t in tot), axis=(0, 1, 2)), atol=1e-13)


def test_constant_velocity_transport_converges_to_the_translated_field():
    """m(1)(x) = m_A(x - v) for constant v.  With cubic interpolation the
    error behaves like h^4 / dt; doubling the grid and the number of steps
    together divides it by about 2^3."""
    errs = []
    vel = (0.37, -0.21, 0.29)
    for n in (16, 32):
        n3 = (n, n, n)
        X = synth.coords_mesh(n3)
        f = lambda Y: np.exp(np.cos(Y[0]) + 0.5 * np.sin(Y[1]) * np.cos(Y[2]))
        v = [np.full(n3, vel[a]) for a in range(3)]
        R = G.Registration(n3, [f(X)] * 3, [f(X)] * 3, np.zeros(n3), None, n // 4, 1.0)
        m1 = R.forward(v)[-1][0]
        errs.append(np.abs(m1 - f([X[a] - vel[a] for a in range(3)])).max())
    assert errs[1] < 1e-2 and errs[0] / errs[1] > 6.0, errs


# ------------------------------------------------------------------- Leray
def test_leray_projection_properties():
    n = (16, 12, 20)
    g = G.Grid(n)
    rng = np.random.default_rng(3)
    w = [rng.standard_normal(n) for _ in range(3)]
    Kw = g.leray(w)
    assert np.abs(g.div(Kw)).max() < 1e-10
    KKw = g.leray(Kw)
    assert max(np.abs(a - b).max() for a, b in zip(KKw, Kw)) < 1e-12
    phi = rng.standard_normal(n)
    assert max(np.abs(x).max() for x in g.leray(g.grad(phi))) < 1e-10
    u = _divfree(n, 4, radius=3)
    assert max(np.abs(a - b).max() for a, b in zip(g.leray(u), u)) < 1e-12
    # self-adjoint
    z = [rng.standard_normal(n) for _ in range(3)]
    assert abs(_ip(g, g.leray(w), z) - _ip(g, w, g.leray(z))) < 1e-10 * abs(_ip(g, w, z) + 1.0)


def test_preconditioner_inverts_the_regularisation():
    n = (16, 16, 16)
    g = G.Grid(n)
    R = G.Registration(n, [np.zeros(n)] * 3, [np.zeros(n)] * 3, np.zeros(n), None, 2, beta_v=0.3)
    u = _divfree(n, 5, radius=3)
    Au = [0.3 * g.neg_lap(x) for x in u]
    z = R.precond(Au)
    assert max(np.abs(a - b).max() for a, b in zip(z, u)) < 1e-12
    one = [np.ones(n)] * 3                          # the zero mode is divided by beta
    assert np.allclose(R.precond(one)[0], 1.0 / 0.3)


# ------------------------------------------------------- gradient, Hessian
def _fd_rel(R, v, vt, eps=1e-5):
    J, gr = R.gradient(v)
    Jp = R.objective([v[a] + eps * vt[a] for a in range(3)])
    Jm = R.objective([v[a] - eps * vt[a] for a in range(3)])
    fd = (Jp - Jm) / (2 * eps)
    return abs(fd - _ip(R.g, gr, vt)) / abs(fd)


def test_gradient_converges_to_central_differences():
    """The reduced gradient matches central differences of the objective up
    to the discretisation's inconsistency (interpolation error ~ h^4 / dt),
    which falls steeply under grid refinement at a fixed number of steps."""
    e16 = _fd_rel(*_smooth_case(16, 4)[:3])
    e32 = _fd_rel(*_smooth_case(32, 4)[:3])
    assert e32 < 1e-3 and e16 / e32 > 8.0, (e16, e32)


def test_gauss_newton_hessian_at_zero_residual_and_symmetry():
    """At zero residual (m_P = (1 - c) m(1), q = 0) the Gauss-Newton product
    is the derivative of the gradient; it is positive, and symmetric up to
    the small discretisation error of the optimize-then-discretize scheme."""
    R, v, vt, vt2 = _smooth_case(16, 4, zero_res=True)
    eps = 1e-5
    gp = R.gradient([v[a] + eps * vt[a] for a in range(3)])[1]
    gm = R.gradient([v[a] - eps * vt[a] for a in range(3)])[1]
    fdg = [(p - m) / (2 * eps) for p, m in zip(gp, gm)]
    H = R.hessvec(v, vt)
    rel = math.sqrt(sum(float(np.sum((a - b) ** 2)) for a, b in zip(fdg, H))) / \
        math.sqrt(sum(float(np.sum(b * b)) for b in H))
    assert rel < 1e-2, rel
    sym = []
    for n in (16, 32):
        R, v, vt, vt2 = _smooth_case(n, 2)
        h1, h2 = R.hessvec(v, vt), R.hessvec(v, vt2)
        a, b = _ip(R.g, h1, vt2), _ip(R.g, h2, vt)
        sym.append(abs(a - b) / abs(a))
        assert _ip(R.g, h1, vt) > 0.0
    assert max(sym) < 1e-3, sym


def test_gradient_of_the_q_term_and_the_regularisation():
    """With v = 0 the state is m_A at all times: the gradient is
    K[int sum_i l_i grad m_A,i] with l constant in time, and the
    regularisation term vanishes; beta scales only the H^1 part."""
    R, v, vt, _ = _smooth_case(16, 2)
    zero = [np.zeros(R.n) for _ in range(3)]
    J0, g0 = R.gradient(zero)
    lam1 = R.final_adjoint(R.mA)
    b = [sum(lam1[i] * R.g.grad(R.mA[i])[a] for i in range(3)) for a in range(3)]
    want = R.g.leray(b)
    assert max(np.abs(x - y).max() for x, y in zip(g0, want)) < 1e-12
    # the reduced gradient lives in the divergence-free space
    _, gv = R.gradient(v)
    assert np.abs(R.g.div(gv)).max() < 1e-10 * max(np.abs(x).max() for x in gv)
    R2 = G.Registration(R.n, R.mA, R.mP, R.c, R.q, R.nt, beta_v=2 * R.beta)
    _, g1 = R.gradient(v)
    _, g2 = R2.gradient(v)
    diff = [y - x for x, y in zip(g1, g2)]
    reg = [R.beta * R.g.neg_lap(x) for x in v]
    assert max(np.abs(d - r).max() for d, r in zip(diff, reg)) < 1e-12
