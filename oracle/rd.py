"""FP64 CPU oracle of the tumor reaction-diffusion calibration hot path.

TEST INFRASTRUCTURE ONLY: tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this module; the product path never
does, and it shares no code with the CUDA implementation.

It computes, plainly and slowly, in FP64:

* the coefficients ``kappa = k_f sum_i k_i m_i`` and
  ``rho = rho_f sum_i rho_i m_i`` (Eq. ``coeff_tumor``);
* the initial condition ``c(0) = Phi p``, a sum of Gaussians (Eq.
  ``tumor:fwd-init``; Sec. 4.1 for width and lattice);
* the state equation ``dc/dt = div(kappa grad c) + rho c (1 - c)`` (Eq.
  ``tumor:fwd``) on the periodic box ``[0, 2 pi)^3`` with Fourier spectral
  derivatives (Sec. 3.3) and the second-order Strang splitting with an exact
  logistic reaction step and Crank-Nicolson diffusion (Sec. 3.3);
* the misfit ``D_c = 1/2 ||c(1) - d||^2_{L2}`` (Table 1);
* the discrete adjoint of that scheme (Eq. ``tumor:adj`` and
  ``tumor:adj-final`` with the final condition ``alpha(1) = d - c(1)``);
* the reduced gradient w.r.t. ``p`` (Eq. ``tumor:inv``), ``k_f`` (Eq.
  ``tumor:inv_diff``) and ``rho_f`` (derived the same way from Eq.
  ``coeff_tumor``);
* the Gauss-Newton Hessian-vector product ``J^T J v`` built from the tangent
  linear model and the same adjoint;
* the Moving-Atlas anatomy misfit ``D_m`` and its final-condition term
  (Eq. ``objective_tu``, ``tumor:adj-final``);
* the Picard coupling field ``q(x)`` handed to the registration step
  (Sec. 2.2).

Readings where the paper is silent:

* Strang order ``L(tau/2) CN(tau) L(tau/2)`` with ``L_t`` the exact logistic
  flow ``c e^{rho t} / (1 - c + c e^{rho t})``.
* CN: ``(I - tau/2 A) c** = (I + tau/2 A) c*`` solved by PCG with the
  spectral preconditioner ``1 / (1 + tau/2 * kbar * |k~|^2)``, kbar the
  mean of kappa over the voxels where it is positive (the brain region).
* ``i k`` is zeroed at the Nyquist index of every even axis (``k~``), which
  keeps ``A = div(kappa grad .)`` real, symmetric and negative semidefinite.
* Adjoint reaction sign: the adjoint of the logistic step is multiplication
  by ``dL_t/dc = e^{rho t} / (1 - c + c e^{rho t})^2``; the sign printed in
  Eq. ``tumor:adj`` is read as a typo (pinned by finite differences).
* Gaussians ``exp(-|x - x_i|^2 / (2 sigma^2))`` with the minimum-image
  distance per axis and peak value 1; no CSF zeroing unless requested.
* Misfit weight ``h^3`` (the L2(Omega) quadrature of ``D_c``).

Moving-Atlas objective (Eq. ``objective_tu``, optional): with anatomy data
``m_D`` set, the misfit adds ``D_m = 1/2 ||m (1 - c(1)) - m_D||^2`` summed
over the three labels, and the adjoint final condition adds
``m^T (m (1 - c(1)) - m_D)`` (Eq. ``tumor:adj-final``).
"""

from __future__ import annotations

import math

import numpy as np

from . import fft as _fft

TWO_PI = 2.0 * math.pi


# --------------------------------------------------------------------------
# spectral derivatives (Sec. 3.3)
# --------------------------------------------------------------------------
class Spectral:
    """Fourier pseudo-spectral derivatives on the periodic box [0, 2 pi)^3."""

    def __init__(self, n, kind="recursive"):
        self.n = tuple(int(k) for k in n)
        self.kind = kind
        self.h3 = float(np.prod([TWO_PI / k for k in self.n]))
        self.kd = []
        for a, m in enumerate(self.n):
            j = np.arange(m)
            k = np.where(j <= (m - 1) // 2, j, j - m).astype(np.float64)
            if m % 2 == 0:
                k[m // 2] = 0.0          # Nyquist: derivative symbol zeroed
            shape = [1, 1, 1]
            shape[a] = m
            self.kd.append(k.reshape(shape))
        self.ksq = self.kd[0] ** 2 + self.kd[1] ** 2 + self.kd[2] ** 2

    def F(self, u):
        return _fft.fftn(u, kind=self.kind)

    def Finv(self, U):
        return _fft.fftn(U, inverse=True, kind=self.kind)

    def grad(self, u):
        """``[d u / d x_a]`` for a = 0, 1, 2."""
        U = self.F(u)
        return [np.real(self.Finv(1j * self.kd[a] * U)) for a in range(3)]

    def div(self, hs):
        """``sum_a d h_a / d x_a``."""
        S = 1j * self.kd[0] * self.F(hs[0])
        S = S + 1j * self.kd[1] * self.F(hs[1])
        S = S + 1j * self.kd[2] * self.F(hs[2])
        return np.real(self.Finv(S))

    def A(self, u, kappa):
        """``div(kappa grad u)``: one forward transform, three inverse
        transforms for the gradient, three forward and one inverse for the
        divergence."""
        return self.div([kappa * g for g in self.grad(u)])

    def precond(self, r, coef):
        """``F^{-1} [ F r / (1 + coef |k~|^2) ]``."""
        return np.real(self.Finv(self.F(r) / (1.0 + coef * self.ksq)))


# --------------------------------------------------------------------------
# reaction (exact logistic flow, Sec. 3.3 "analytical solution")
# --------------------------------------------------------------------------
def logistic(c, rho, t):
    e = np.exp(rho * t)
    return c * e / (1.0 - c + c * e)


def logistic_dc(c, rho, t):
    e = np.exp(rho * t)
    return e / (1.0 - c + c * e) ** 2


# --------------------------------------------------------------------------
# preconditioned conjugate gradients
# --------------------------------------------------------------------------
def pcg(matvec, precond, b, x0, rtol, maxit):
    """Textbook PCG; stops when ``||r||_2 <= rtol ||b||_2`` or after
    ``maxit`` iterations.  Returns ``(x, iterations, ||r|| / ||b||)``."""
    x = np.array(x0, dtype=np.float64, copy=True)
    r = b - matvec(x)
    bn = float(np.linalg.norm(b))
    if bn == 0.0:
        return np.zeros_like(b), 0, 0.0
    z = precond(r)
    p = z.copy()
    rz = float(np.vdot(r, z))
    it = 0
    rn = float(np.linalg.norm(r))
    while rn > rtol * bn and it < maxit:
        q = matvec(p)
        alpha = rz / float(np.vdot(p, q))
        x += alpha * p
        r -= alpha * q
        it += 1
        rn = float(np.linalg.norm(r))
        if rn <= rtol * bn:
            break
        z = precond(r)
        rz_new = float(np.vdot(r, z))
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it, rn / bn


def kbar_positive(kappa1):
    """Preconditioner constant: the mean of kappa1 over the voxels where it
    is positive (0 if there are none)."""
    pos = kappa1[kappa1 > 0.0]
    return float(pos.mean()) if pos.size else 0.0


# --------------------------------------------------------------------------
# Gaussian basis Phi (Eq. tumor:fwd-init)
# --------------------------------------------------------------------------
def gaussian_factors(n, centers, sigma):
    """Per-axis factors ``g[i, a](x_a) = exp(-d_a^2 / (2 sigma^2))`` with
    ``d_a`` the minimum-image distance; ``G_i = g[i,0] g[i,1] g[i,2]``."""
    out = []
    for a, m in enumerate(n):
        x = np.arange(m) * (TWO_PI / m)
        d = x[None, :] - np.asarray(centers, dtype=np.float64)[:, a:a + 1]
        d = d - TWO_PI * np.round(d / TWO_PI)
        out.append(np.exp(-d * d / (2.0 * sigma * sigma)))
    return out


def phi(p, g):
    """``Phi p = sum_i p_i G_i``."""
    return np.einsum("i,ia,ib,ic->abc", np.asarray(p, dtype=np.float64),
                     g[0], g[1], g[2], optimize=True)


def phi_t(u, g):
    """``(Phi^T u)_i = sum_x G_i(x) u(x)`` (plain sum, no quadrature)."""
    t = np.einsum("abc,ic->iab", u, g[2], optimize=True)
    t = np.einsum("iab,ib->ia", t, g[1], optimize=True)
    return np.einsum("ia,ia->i", t, g[0], optimize=True)


# --------------------------------------------------------------------------
# the model
# --------------------------------------------------------------------------
class Model:
    """Forward, adjoint, gradient and Gauss-Newton Hessian-vector product of
    the discretised tumor model on one grid."""

    def __init__(self, n, m_wm, m_gm, m_csf, centers, sigma, nt,
                 k_w=(1.0, 0.1, 0.0), rho_w=(1.0, 0.2, 0.0), t_end=1.0,
                 rtol=1e-12, maxit=1000, beta_p=0.0, kind="recursive",
                 csf_zero=False):
        self.sp = Spectral(n, kind)
        self.n = self.sp.n
        self.h3 = self.sp.h3
        m = [np.asarray(x, dtype=np.float64) for x in (m_wm, m_gm, m_csf)]
        self.kappa1 = k_w[0] * m[0] + k_w[1] * m[1] + k_w[2] * m[2]
        self.rho1 = rho_w[0] * m[0] + rho_w[1] * m[1] + rho_w[2] * m[2]
        self.g = gaussian_factors(self.n, centers, sigma)
        self.csf = (m[2] < 0.5).astype(np.float64) if csf_zero else None
        self.m = m
        self.k_w = tuple(float(x) for x in k_w)
        self.rho_w = tuple(float(x) for x in rho_w)
        self.m_data = None
        self.nt = int(nt)
        self.tau = t_end / nt
        self.s = 0.5 * self.tau
        self.rtol = rtol
        self.maxit = maxit
        self.beta_p = beta_p
        self.iters = []

    # -- pieces ------------------------------------------------------------
    def A(self, u, k_f):
        return self.sp.A(u, k_f * self.kappa1)

    def phi(self, p):
        c = phi(p, self.g)
        return c if self.csf is None else c * self.csf

    def phi_t(self, u):
        return phi_t(u if self.csf is None else u * self.csf, self.g)

    def solve(self, b, x0, k_f):
        """``(I - s A) x = b`` by PCG with the spectral preconditioner."""
        s = self.s
        coef = s * k_f * kbar_positive(self.kappa1)
        x, it, _ = pcg(lambda v: v - s * self.A(v, k_f),
                       lambda r: self.sp.precond(r, coef),
                       b, x0, self.rtol, self.maxit)
        self.iters.append(it)
        return x

    # -- forward (Eq. tumor:fwd, Strang + CN) -------------------------------
    def forward(self, p, k_f, rho_f, c0=None):
        """Returns ``(c(1), trajectory)``; trajectory entry ``n`` holds
        ``(c_n, c*_n, c**_n, c_{n+1})``: the state, after the first half
        reaction, after the diffusion step, after the second half reaction."""
        rho = rho_f * self.rho1
        s = self.s
        c = self.phi(p) if c0 is None else np.array(c0, dtype=np.float64)
        traj = []
        for _ in range(self.nt):
            c_star = logistic(c, rho, s)
            b = c_star + s * self.A(c_star, k_f)
            c_ss = self.solve(b, c_star, k_f)
            c_next = logistic(c_ss, rho, s)
            traj.append((c, c_star, c_ss, c_next))
            c = c_next
        return c, traj

    def set_anatomy_data(self, m_d):
        """Patient anatomy labels ``m_D`` (three fields) for ``D_m``."""
        self.m_data = [np.asarray(x, dtype=np.float64) for x in m_d]

    def misfit(self, c1, d, p):
        r = c1 - d
        J = 0.5 * self.h3 * float(np.sum(r * r)) + 0.5 * self.beta_p * float(np.dot(p, p))
        if self.m_data is not None:
            for mi, mdi in zip(self.m, self.m_data):
                e = mi * (1.0 - c1) - mdi
                J += 0.5 * self.h3 * float(np.sum(e * e))
        return J

    def final_adjoint(self, c1, d):
        """``alpha(1) = d - c(1) [+ m^T (m (1 - c(1)) - m_D)]``."""
        a = d - c1
        if self.m_data is not None:
            for mi, mdi in zip(self.m, self.m_data):
                a = a + mi * (mi * (1.0 - c1) - mdi)
        return a

    def final_weight(self):
        """Second derivative of the misfit in c(1): 1 [+ sum_i m_i^2]."""
        w = 1.0
        if self.m_data is not None:
            w = w + sum(mi * mi for mi in self.m)
        return w

    # -- adjoint (Eq. tumor:adj, tumor:adj-final) and gradient assembly -----
    def adjoint(self, traj, alpha1, k_f, rho_f, fields=None):
        """Reverse sweep of the discrete adjoint from ``alpha(1)``.

        Returns ``(alpha(0), g_kf, g_rhof)`` where, with ``s = tau/2`` and
        ``abar`` the CN-transposed adjoint of each step,
        ``g_kf = sum_n s h^3 sum_x kappa1 grad(abar) . grad(c* + c**)``
        (trapezoidal form of Eq. ``tumor:inv_diff``) and
        ``g_rhof = -sum_half-steps h^3 sum_x alpha s rho1 L (1 - L)``.

        ``fields``: a dict that receives the same integrands before the sum
        over x, ``"k"`` = ``sum_n s grad(abar) . grad(c* + c**)`` and
        ``"rho"`` = ``-sum_half-steps s alpha L (1 - L)`` per voxel, so that
        ``g_kf = h^3 sum_x kappa1 fields["k"]`` and likewise for rho_f."""
        rho = rho_f * self.rho1
        s, h3 = self.s, self.h3
        alpha = np.array(alpha1, dtype=np.float64)
        g_kf = 0.0
        g_rho = 0.0
        qk = np.zeros(self.n)
        qr = np.zeros(self.n)
        for c, c_star, c_ss, c_next in reversed(traj):
            qr -= alpha * s * c_next * (1.0 - c_next)
            g_rho -= h3 * float(np.sum(alpha * s * self.rho1 * c_next * (1.0 - c_next)))
            alpha_ss = logistic_dc(c_ss, rho, s) * alpha
            abar = self.solve(alpha_ss, alpha_ss, k_f)
            ga = self.sp.grad(abar)
            gw = self.sp.grad(c_star + c_ss)
            dot = ga[0] * gw[0] + ga[1] * gw[1] + ga[2] * gw[2]
            qk += s * dot
            g_kf += s * h3 * float(np.sum(self.kappa1 * dot))
            alpha_star = abar + s * self.A(abar, k_f)
            qr -= alpha_star * s * c_star * (1.0 - c_star)
            g_rho -= h3 * float(np.sum(alpha_star * s * self.rho1 * c_star * (1.0 - c_star)))
            alpha = logistic_dc(c, rho, s) * alpha_star
        if fields is not None:
            fields["k"] = qk
            fields["rho"] = qr
        return alpha, g_kf, g_rho

    def gradient(self, p, k_f, rho_f, d):
        """Misfit and reduced gradient ``[g_p, g_kf, g_rhof]`` (Sec. 3.1:
        state solve, adjoint solve, then Eq. ``tumor:inv``/``inv_diff``)."""
        p = np.asarray(p, dtype=np.float64)
        c1, traj = self.forward(p, k_f, rho_f)
        J = self.misfit(c1, d, p)
        alpha0, g_kf, g_rho = self.adjoint(traj, self.final_adjoint(c1, d), k_f, rho_f)
        g_p = -self.h3 * self.phi_t(alpha0) + self.beta_p * p
        return J, np.concatenate([g_p, [g_kf, g_rho]]), c1, alpha0

    def coupling(self, p, k_f, rho_f, d):
        """Picard coupling field ``q = (q_WM, q_GM, q_CSF)`` of Sec. 2.2: the
        time integral of ``kbar grad c . grad alpha + rhobar c (1 - c) alpha``
        with ``kbar = k_f (k_WM, k_GM, k_CSF)`` and ``rhobar = rho_f (rho_WM,
        rho_GM, rho_CSF)``, taken with the quadrature of the discrete
        gradient and the sign of a derivative, so that a change of the tissue
        maps inside the coefficients (Eq. ``coeff_tumor``) changes the
        objective by ``h^3 sum_x q . dm`` at first order."""
        p = np.asarray(p, dtype=np.float64)
        c1, traj = self.forward(p, k_f, rho_f)
        fl = {}
        self.adjoint(traj, self.final_adjoint(c1, d), k_f, rho_f, fields=fl)
        return [k_f * self.k_w[i] * fl["k"] + rho_f * self.rho_w[i] * fl["rho"] for i in range(3)]

    # -- Gauss-Newton Hessian-vector product --------------------------------
    def tangent(self, traj, v, k_f, rho_f):
        """Tangent-linear model: ``dc(1)`` for the direction
        ``v = [v_p, v_kf, v_rhof]`` about the trajectory ``traj``."""
        npar = len(v) - 2
        v_p, v_k, v_r = np.asarray(v[:npar]), float(v[npar]), float(v[npar + 1])
        rho = rho_f * self.rho1
        s = self.s
        ch = self.phi(v_p)
        for c, c_star, c_ss, c_next in traj:
            ch_star = logistic_dc(c, rho, s) * ch \
                + v_r * s * self.rho1 * c_star * (1.0 - c_star)
            b = ch_star + s * self.A(ch_star, k_f) \
                + s * v_k * self.sp.A(c_star + c_ss, self.kappa1)
            ch_ss = self.solve(b, ch_star, k_f)
            ch = logistic_dc(c_ss, rho, s) * ch_ss \
                + v_r * s * self.rho1 * c_next * (1.0 - c_next)
        return ch

    def hessvec(self, p, k_f, rho_f, v, traj=None):
        """``H_GN v = J^T (h^3 W J v) + beta_p v_p`` with W the second
        derivative of the misfit in c(1) (1, plus sum m_i^2 with D_m)."""
        p = np.asarray(p, dtype=np.float64)
        v = np.asarray(v, dtype=np.float64)
        if traj is None:
            _, traj = self.forward(p, k_f, rho_f)
        ch1 = self.tangent(traj, v, k_f, rho_f)
        alpha0, g_kf, g_rho = self.adjoint(traj, -self.final_weight() * ch1, k_f, rho_f)
        npar = len(v) - 2
        hv_p = -self.h3 * self.phi_t(alpha0) + self.beta_p * v[:npar]
        return np.concatenate([hv_p, [g_kf, g_rho]])


def model_from_problem(prob, **kw):
    """Build a :class:`Model` from a synthetic problem description."""
    return Model(prob.n, prob.m_wm, prob.m_gm, prob.m_csf, prob.centers,
                 prob.sigma, prob.nt, k_w=prob.k_w, rho_w=prob.rho_w, **kw)
