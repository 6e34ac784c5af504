"""FP64 CPU oracle of the registration component of the Picard step.

TEST INFRASTRUCTURE ONLY: tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this module; the product path never
does, and it shares no code with the CUDA implementation.

What it computes (the modified registration problem of Sec. 2.2, Eq.
``objective_reg``, with the optimality conditions ``reg:state``,
``reg:adj``, ``reg:adj-final``, ``reg:inv`` of Sec. 2.1 and the numerics of
Sec. 3.2 and 3.3):

* the atlas anatomy ``m = (m_WM, m_GM, m_CSF)`` transported by a stationary
  velocity ``v``: ``dm/dt + grad(m) v = 0``, ``m(0) = m_A`` (Eq. ``reg:fwd``);
* the objective ``J(v) = D_m[m(1) (1 - c), m_P] + h^3 sum_x q . m(1)
  + beta_v / 2 |grad v|^2`` with ``D_m = 1/2 h^3 sum_i sum_x (m_i(1)
  (1 - c) - m_P,i)^2`` (c = c(1) and q from the tumor solve, held fixed);
* the adjoint ``-dl/dt - div(l v) = 0`` backwards from
  ``l(1) = -[(1 - c)(m(1)(1 - c) - m_P) + q]`` (Eq. ``reg:adj``,
  ``reg:adj-final`` with the Picard substitution of q);
* the reduced gradient ``g = beta_v (-Lap) v + K[int_0^1 sum_i l_i grad m_i
  dt]`` (Eq. ``reg:inv``; the H^1 seminorm of Eq. ``registr_reg``);
* the Gauss-Newton Hessian-vector product from the incremental state and
  adjoint equations;
* the spectral preconditioner ``(beta_v (-Lap))^-1`` (zero mode ``1 /
  beta_v``).

Readings where the paper defers to its references:

* ``div v = w`` is taken with ``w = 0`` (incompressible velocity), so K is
  the Leray projection ``K u = u - grad Lap^-1 div u`` onto divergence-free
  fields (the paper prints the sign of the second term as ``+``).
* Semi-Lagrangian time stepping with ``nt`` steps of ``dt = 1 / nt``: the
  characteristic foot ``X = x - dt/2 (v(x) + v(x - dt v(x)))`` (Heun / RK2
  for the stationary field), tricubic Lagrange interpolation on the periodic
  grid (nodes -1, 0, 1, 2 around the foot's cell, per axis).
* Adjoint: along the reversed characteristics ``X+ = x + dt/2 (v(x) + v(x +
  dt v(x)))``, Heun's rule for the source ``l div v``.
* Incremental state: ``dm~/dt + grad(m~) v = -grad(m) v~``, trapezoidal rule
  for the source along the characteristic; time integral of the body force
  by the trapezoidal rule over the nt + 1 time levels.
* Spatial derivatives spectral, with the Nyquist mode of first derivatives
  zeroed (as for the tumor operator).
"""

from __future__ import annotations

import numpy as np

TWO_PI = 2.0 * np.pi


# ------------------------------------------------------------ spectral ops
class Grid:
    """Periodic grid on [0, 2 pi)^3 with FFT-based derivatives."""

    def __init__(self, n):
        self.n = tuple(int(k) for k in n)
        self.h = tuple(TWO_PI / k for k in self.n)
        self.h3 = float(np.prod(self.h))
        self.k = []
        for a, m in enumerate(self.n):
            j = np.arange(m)
            k = np.where(j <= (m - 1) // 2, j, j - m).astype(np.float64)
            kd = k.copy()
            if m % 2 == 0:
                kd[m // 2] = 0.0      # first derivative: Nyquist symbol zeroed
            shape = [1, 1, 1]
            shape[a] = m
            self.k.append((kd.reshape(shape), k.reshape(shape)))
        # |k|^2 with the Nyquist kept (second derivatives, Poisson)
        self.ksq = sum(kk ** 2 for _, kk in self.k)

    def d(self, u, a):
        """Spectral first derivative along axis a."""
        return np.real(np.fft.ifftn(1j * self.k[a][0] * np.fft.fftn(u)))

    def grad(self, u):
        return [self.d(u, a) for a in range(3)]

    def div(self, w):
        return self.d(w[0], 0) + self.d(w[1], 1) + self.d(w[2], 2)

    def neg_lap(self, u):
        """-Lap u = sum_a -d_a d_a u with the first-derivative symbol on
        each axis (the H^1 seminorm's operator, consistent with grad)."""
        return -sum(self.d(self.d(u, a), a) for a in range(3))

    def inv_neg_lap(self, f, zero_mode=0.0):
        """Solve -Lap u = f with the same symbol sum_a k~_a^2; modes where the
        symbol vanishes get ``zero_mode * f``."""
        s = sum(kd ** 2 for kd, _ in self.k)
        F = np.fft.fftn(f)
        with np.errstate(divide="ignore", invalid="ignore"):
            U = np.where(s > 0, F / np.where(s > 0, s, 1.0), zero_mode * F)
        return np.real(np.fft.ifftn(U))

    def leray(self, w):
        """K w = w - grad Lap^-1 div w: the divergence-free part (built from
        the same first-derivative symbols, so div K w = 0 exactly)."""
        phi = self.inv_neg_lap(-self.div(w))     # Lap phi = div w
        gp = self.grad(phi)
        return [w[a] - gp[a] for a in range(3)]


# --------------------------------------------------- semi-Lagrangian pieces
def lagrange_weights(f):
    """Cubic Lagrange weights of the nodes -1, 0, 1, 2 at offset f in [0, 1)."""
    return [-f * (f - 1.0) * (f - 2.0) / 6.0,
            (f + 1.0) * (f - 1.0) * (f - 2.0) / 2.0,
            -(f + 1.0) * f * (f - 2.0) / 2.0,
            (f + 1.0) * f * (f - 1.0) / 6.0]


def interp(u, X):
    """Periodic tricubic Lagrange interpolation of the grid function u at
    the points X = (X0, X1, X2) given in index units (x_a / h_a)."""
    n = u.shape
    base, wts = [], []
    for a in range(3):
        fl = np.floor(X[a])
        base.append(fl.astype(np.int64))
        wts.append(lagrange_weights(X[a] - fl))
    out = np.zeros(X[0].shape)
    for o0 in range(4):
        i0 = (base[0] + o0 - 1) % n[0]
        for o1 in range(4):
            i1 = (base[1] + o1 - 1) % n[1]
            w01 = wts[0][o0] * wts[1][o1]
            for o2 in range(4):
                i2 = (base[2] + o2 - 1) % n[2]
                out += w01 * wts[2][o2] * u[i0, i1, i2]
    return out


def index_grid(n):
    return np.meshgrid(*[np.arange(k, dtype=np.float64) for k in n], indexing="ij")


def feet(grid, v, dt, sign=-1.0):
    """Characteristic feet in index units: x + sign dt/2 (v(x) + v(x + sign
    dt v(x))) (Heun's rule for the stationary velocity)."""
    I = index_grid(grid.n)
    hs = grid.h
    Y = [I[a] + sign * dt * v[a] / hs[a] for a in range(3)]
    vY = [interp(v[a], Y) for a in range(3)]
    return [I[a] + sign * 0.5 * dt * (v[a] + vY[a]) / hs[a] for a in range(3)]


# ------------------------------------------------------------ the problem
class Registration:
    """The registration sub-problem for fixed tumor c(1) and coupling q."""

    def __init__(self, n, m_atlas, m_patient, c1, q, nt, beta_v):
        self.g = Grid(n)
        self.n = self.g.n
        self.mA = [np.asarray(x, dtype=np.float64) for x in m_atlas]
        self.mP = [np.asarray(x, dtype=np.float64) for x in m_patient]
        self.c = np.asarray(c1, dtype=np.float64)
        self.q = [np.zeros(self.n) if q is None else np.asarray(x, dtype=np.float64) for x in (q or [None] * 3)]
        self.nt = int(nt)
        self.dt = 1.0 / self.nt
        self.beta = float(beta_v)

    # -- state ------------------------------------------------------------
    def forward(self, v):
        """m^0 = m_A, m^{j+1}(x) = m^j(X(x)); returns the nt + 1 levels."""
        X = feet(self.g, v, self.dt, -1.0)
        levels = [[m.copy() for m in self.mA]]
        for _ in range(self.nt):
            levels.append([interp(m, X) for m in levels[-1]])
        return levels

    def objective(self, v, levels=None):
        if levels is None:
            levels = self.forward(v)
        m1 = levels[-1]
        h3, w = self.g.h3, 1.0 - self.c
        J = 0.0
        for i in range(3):
            r = m1[i] * w - self.mP[i]
            J += 0.5 * h3 * float(np.sum(r * r)) + h3 * float(np.sum(self.q[i] * m1[i]))
        for a in range(3):
            ga = self.g.grad(v[a])
            J += 0.5 * self.beta * h3 * sum(float(np.sum(x * x)) for x in ga)
        return J

    def final_adjoint(self, m1):
        w = 1.0 - self.c
        return [-(w * (m1[i] * w - self.mP[i]) + self.q[i]) for i in range(3)]

    # -- adjoint ----------------------------------------------------------
    def adjoint(self, v, lam1):
        """-dl/dt - div(l v) = 0 from l(1) = lam1, backwards; returns the
        nt + 1 levels (index j = time j dt)."""
        dt = self.dt
        Xp = feet(self.g, v, dt, +1.0)
        D = self.g.div(v)
        DX = interp(D, Xp)
        lev = [None] * (self.nt + 1)
        lev[self.nt] = [x.copy() for x in lam1]
        for j in range(self.nt - 1, -1, -1):
            nxt = []
            for l in lev[j + 1]:
                lX = interp(l, Xp)
                pred = lX + dt * lX * DX
                nxt.append(lX + 0.5 * dt * (lX * DX + pred * D))
            lev[j] = nxt
        return lev

    def body_force(self, levels, lam):
        """int_0^1 sum_i l_i grad m_i dt, trapezoidal over the time levels."""
        b = [np.zeros(self.n) for _ in range(3)]
        for j in range(self.nt + 1):
            wj = self.dt * (0.5 if j in (0, self.nt) else 1.0)
            for i in range(3):
                gm = self.g.grad(levels[j][i])
                for a in range(3):
                    b[a] += wj * lam[j][i] * gm[a]
        return b

    def gradient(self, v):
        """Objective and reduced gradient ``beta (-Lap) v + K[b]``."""
        levels = self.forward(v)
        J = self.objective(v, levels)
        lam = self.adjoint(v, self.final_adjoint(levels[-1]))
        b = self.g.leray(self.body_force(levels, lam))
        return J, [self.beta * self.g.neg_lap(v[a]) + b[a] for a in range(3)]

    # -- Gauss-Newton -----------------------------------------------------
    def incremental_state(self, v, vt, levels):
        """dm~/dt + grad(m~) v = -grad(m) vt, m~(0) = 0; trapezoidal rule
        for the source along the characteristic."""
        X = feet(self.g, v, self.dt, -1.0)
        dt = self.dt

        def src(ms):
            out = []
            for m in ms:
                gm = self.g.grad(m)
                out.append(gm[0] * vt[0] + gm[1] * vt[1] + gm[2] * vt[2])
            return out

        mt = [np.zeros(self.n) for _ in range(3)]
        s_prev = src(levels[0])
        for j in range(self.nt):
            s_next = src(levels[j + 1])
            mt = [interp(mt[i], X) - 0.5 * dt * (interp(s_prev[i], X) + s_next[i]) for i in range(3)]
            s_prev = s_next
        return mt

    def hessvec(self, v, vt, levels=None):
        """``H vt = beta (-Lap) vt + K[int sum_i l~_i grad m_i dt]`` with
        ``l~(1) = -(1 - c)^2 m~(1)`` (Gauss-Newton: terms carrying l are
        dropped)."""
        if levels is None:
            levels = self.forward(v)
        mt1 = self.incremental_state(v, vt, levels)
        w2 = (1.0 - self.c) ** 2
        lt = self.adjoint(v, [-w2 * x for x in mt1])
        b = self.g.leray(self.body_force(levels, lt))
        return [self.beta * self.g.neg_lap(vt[a]) + b[a] for a in range(3)]

    def precond(self, r):
        """(beta (-Lap))^-1 per component; the zero mode is divided by beta."""
        return [self.g.inv_neg_lap(x, zero_mode=1.0) / self.beta for x in r]
