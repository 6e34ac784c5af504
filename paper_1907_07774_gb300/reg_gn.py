"""Inexact Gauss-Newton-Krylov solve of the registration sub-problem
(Sec. 3.2): each outer iteration takes the reduced gradient
(``rg_gradient``), solves ``H s = -g`` by preconditioned CG on the
Gauss-Newton Hessian (``rg_hessvec``, preconditioner ``rg_apply_precond``)
to a relative tolerance proportional to the gradient norm (forcing
``min(0.5, sqrt(|g| / |g_0|))`` after Eisenstat and Walker), and an Armijo
backtracking line search on the objective (``rg_forward``).

The PDE solves run in the CUDA library.  The Krylov vectors live on the
host as FP64 arrays (three fields each); their inner products carry the
quadrature weight h^3, so that ``h^3 <g, s>`` is the directional derivative
of J.
"""

from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class RegGNResult:
    v: list
    objective: float
    history: list = field(default_factory=list)


def _ip(h3, a, b):
    return h3 * sum(float(np.vdot(x, y)) for x, y in zip(a, b))


def _axpy(alpha, x, y):
    return [yy + alpha * xx for xx, yy in zip(x, y)]


def pcg(hv, precond, b, h3, rtol, maxit):
    """PCG on H x = b, x0 = 0; stops at |r| <= rtol |b|, after maxit
    products, or on non-positive curvature.  Returns (x, products)."""
    x = [np.zeros_like(bb) for bb in b]
    r = [bb.copy() for bb in b]
    z = precond(r)
    p = [zz.copy() for zz in z]
    rz = _ip(h3, r, z)
    bn = math.sqrt(_ip(h3, b, b))
    used = 0
    for _ in range(maxit):
        if math.sqrt(_ip(h3, r, r)) <= rtol * bn:
            break
        q = hv(p)
        used += 1
        pq = _ip(h3, p, q)
        if pq <= 0.0:
            if used == 1:
                x = [zz.copy() for zz in z]
            break
        a = rz / pq
        x = _axpy(a, p, x)
        r = _axpy(-a, q, r)
        z = precond(r)
        rz_new = _ip(h3, r, z)
        p = _axpy(rz_new / rz, p, z)
        rz = rz_new
    return x, used


def gauss_newton(solver, v0, h3, iters=5, cg_maxit=10, forcing=None, armijo_c=1e-4, max_backtracks=10,
                 gtol_rel=1e-6, callback=None):
    """Run up to ``iters`` Gauss-Newton iterations from the velocity ``v0``
    (three fields) with a registration context that has its images set."""
    v = [np.array(x, dtype=np.float64) for x in v0]
    J, g = solver.rg_gradient(v)
    g0 = math.sqrt(_ip(h3, g, g))
    hist = []
    for k in range(iters):
        t0 = time.perf_counter()
        gn = math.sqrt(_ip(h3, g, g))
        if gn <= gtol_rel * g0:
            break
        eta = min(0.5, math.sqrt(gn / g0)) if forcing is None else float(forcing)
        s, used = pcg(lambda p: solver.rg_hessvec(v, p), solver.rg_apply_precond, [-x for x in g], h3, eta, cg_maxit)
        slope = _ip(h3, g, s)
        if slope >= 0.0:
            s = solver.rg_apply_precond([-x for x in g])
            slope = _ip(h3, g, s)
        step, accepted = 1.0, False
        for _ in range(max_backtracks):
            trial = _axpy(step, s, v)
            Jt = solver.rg_forward(trial)
            if math.isfinite(Jt) and Jt <= J + armijo_c * step * slope:
                accepted = True
                break
            step *= 0.5
        if not accepted:
            hist.append({"iter": k, "objective": J, "grad_norm": gn, "step": 0.0, "hessvecs": used,
                         "seconds": time.perf_counter() - t0})
            break
        v = trial
        J, g = solver.rg_gradient(v)
        rec = {"iter": k, "objective": J, "grad_norm": math.sqrt(_ip(h3, g, g)), "step": step, "hessvecs": used,
               "seconds": time.perf_counter() - t0}
        hist.append(rec)
        if callback:
            callback(rec, v)
    return RegGNResult(v=v, objective=J, history=hist)
