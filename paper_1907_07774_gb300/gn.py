"""Gauss-Newton-Krylov calibration of (p, k_f, rho_f).

Each outer iteration: the reduced gradient (``rd_gradient``), an inexact
Newton step from conjugate gradients on the Gauss-Newton Hessian
(``rd_hessvec``; forcing term ``eta = min(0.5, sqrt(|g| / |g_0|))`` after
Eisenstat-Walker, at most ``cg_maxit`` products), and a projected Armijo
backtracking line search on the misfit (``rd_forward``) that keeps
``k_f >= 0``; a trial whose solve turns non-finite counts as a rejected
step.  This is the inexact
Gauss-Newton-Krylov / PCG / Armijo scheme of Sec. 3.2 applied to the tumor
parameters.  The reduction scalars (CG inner products, step lengths,
sufficient-decrease tests) are FP64 on the host over the n_p + 2 parameters;
every field operation runs in the CUDA library.
"""

from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class GNResult:
    theta: np.ndarray
    misfit: float
    history: list = field(default_factory=list)


def cg(hv, b, maxit, rtol):
    """Plain CG on H x = b (H symmetric positive semidefinite), x0 = 0.
    Stops at |r| <= rtol |b|, after maxit products, or on non-positive
    curvature (returns the iterate so far, or b if that happens at once)."""
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = float(r @ r)
    bn = float(np.sqrt(rr))
    used = 0
    for _ in range(maxit):
        if np.sqrt(rr) <= rtol * bn:
            break
        q = hv(p)
        used += 1
        pq = float(p @ q)
        if pq <= 0.0:
            if used == 1:
                x = b.copy()
            break
        a = rr / pq
        x += a * p
        r -= a * q
        rr_new = float(r @ r)
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x, used


def project(theta):
    """Projection onto the admissible set k_f >= 0 (the diffusion scale of
    Eq. coeff_tumor cannot be negative)."""
    out = theta.copy()
    out[-2] = max(out[-2], 0.0)
    return out


def gauss_newton(solver, theta0, iters=10, cg_maxit=20, armijo_c=1e-4, max_backtracks=12, gtol=1e-6,
                 forcing=None, scale=None, callback=None, fixed=()):
    """Run ``iters`` Gauss-Newton iterations from ``theta0 = [p, k_f, rho_f]``
    with a context that has tissue, basis and data set.

    CG runs on the system rescaled by ``scale`` (default: 1 for p and the
    initial magnitudes of k_f and rho_f, whose natural units differ by orders
    of magnitude), i.e. on S H S with S = diag(scale).  ``forcing``: CG
    relative tolerance; None gives Eisenstat-Walker
    ``min(0.5, sqrt(|g| / |g_0|))``, a number fixes it (with ``cg_maxit``
    the Newton step then uses up to that many Hessian-vector products).
    ``fixed``: indices of parameters held at their start value (their scale
    is set to 0, so neither the gradient nor the step moves them); e.g.
    ``fixed=(n_p + 1,)`` keeps rho_f, as the paper does for its inversions
    (Sec. 1.2: inverting for every growth parameter at once is ill-posed)."""
    npar = solver.np
    theta = np.asarray(theta0, dtype=np.float64).copy()
    split = lambda th: (th[:npar], th[npar], th[npar + 1])
    if scale is None:
        scale = np.ones_like(theta)
        scale[npar] = max(abs(theta[npar]), 1e-3)
        scale[npar + 1] = max(abs(theta[npar + 1]), 1e-3)
    scale = np.asarray(scale, dtype=np.float64).copy()
    for i in fixed:
        scale[i] = 0.0
    J, g = solver.rd_gradient(*split(theta))
    g0 = float(np.linalg.norm(scale * g))
    hist = []
    for k in range(iters):
        t0 = time.perf_counter()
        gs = scale * g
        gn = float(np.linalg.norm(g[scale != 0.0]))
        if gn <= gtol or float(np.linalg.norm(gs)) <= 1e-12 * max(g0, 1e-300):
            break
        if forcing is None:
            eta = min(0.5, np.sqrt(float(np.linalg.norm(gs)) / g0)) if g0 > 0 else 0.5
        else:
            eta = float(forcing)
        ds, n_hv = cg(lambda v: scale * solver.rd_hessvec(*split(theta), scale * v), -gs, cg_maxit, eta)
        d = scale * ds
        slope = float(g @ d)
        if slope >= 0.0:
            d = -(scale != 0.0) * g
            slope = -gn * gn
        step, accepted, n_ls = 1.0, False, 0
        for _ in range(max_backtracks):
            trial = project(theta + step * d)
            n_ls += 1
            if np.all(np.isfinite(trial)):
                try:
                    Jt = solver.rd_forward(*split(trial))
                except Exception as exc:
                    # a trial whose solve turns non-finite (RD_ERR_NONFINITE) is a
                    # rejected step, not a failure of the run
                    if getattr(exc, "status", None) != 6:
                        raise
                    Jt = math.inf
                # projected Armijo condition: sufficient decrease along the
                # actual (projected) displacement
                if Jt <= J + armijo_c * float(g @ (trial - theta)):
                    accepted = True
                    break
            step *= 0.5
        if not accepted:
            hist.append({"iter": k, "misfit": J, "grad_norm": gn, "step": 0.0, "hessvecs": n_hv,
                         "line_search": n_ls, "seconds": time.perf_counter() - t0})
            break
        theta = trial
        J = Jt
        g = solver.rd_adjoint()          # adjoint of the accepted trial's forward solve
        rec = {"iter": k, "misfit": J, "grad_norm": float(np.linalg.norm(g[scale != 0.0])), "step": step,
               "hessvecs": n_hv, "line_search": n_ls, "seconds": time.perf_counter() - t0}
        hist.append(rec)
        if callback:
            callback(rec, theta)
    return GNResult(theta=theta, misfit=J, history=hist)
