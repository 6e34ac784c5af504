"""Picard iteration of the Moving-Atlas scheme (Sec. 2.2 and 2.3).

Iteration j, given the registration velocity v_j:

1. warp the atlas anatomy with v_j (``rg_forward``): the approximation m~ of
   the healthy patient anatomy;
2. tumor inversion in m~ (``rd_set_tissue``), objective D_c + D_m
   (Eq. ``objective_tu``, Moving-Atlas data set on the tumor context): a few
   Gauss-Newton iterations on (p, k_f, rho_f) (``gn.gauss_newton``);
3. the tumor c(1) and the coupling field q(x) of the new parameters
   (``rd_forward``, ``rd_adjoint``, ``rd_coupling_field``);
4. the modified registration problem (Eq. ``objective_reg``) from v_j with
   c(1) and q held fixed: Gauss-Newton-Krylov (``reg_gn.gauss_newton``).

beta_v continuation (Sec. 2.3): start at ``beta_init``, divide by ten after
each Picard iteration down to ``beta_final``, and run ``final_repeats``
iterations at ``beta_final`` (the paper always runs two there).  The paper's
determinant-of-the-deformation-gradient safeguard belongs to the
registration solver's internals and is not reproduced.

All PDE work runs in the CUDA library; this module moves the parameter
vector and host copies of the fields between the two solvers.
"""

from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import gn
from . import reg_gn


@dataclass
class PicardResult:
    theta: np.ndarray
    v: list
    history: list = field(default_factory=list)


def beta_schedule(beta_init, beta_final, final_repeats=2, factor=10.0):
    """beta_init, beta_init / factor, ... down to beta_final, then
    beta_final repeated so that it appears ``final_repeats`` times."""
    out = []
    b = float(beta_init)
    while b > beta_final * (1.0 + 1e-12):
        out.append(b)
        b /= factor
    out += [float(beta_final)] * max(1, int(final_repeats))
    return out


def picard(tumor, make_reg, m_atlas, m_patient, theta0, beta_init=1e-1, beta_final=1e-3, final_repeats=2,
           tumor_iters=3, tumor_cg=10, tumor_forcing=1e-3, reg_iters=3, reg_cg=5, callback=None):
    """Run the Picard iteration.

    ``tumor``: a tumor context (``rd.Context``) created with
    ``moving_atlas=True, coupling=True``, with basis, data and the patient
    anatomy (``rd_set_anatomy_data``) set.  ``make_reg(beta_v)``: returns a
    registration context (``rg.RegContext``) on the same grid.  Fields are
    host FP64 arrays."""
    n = tuple(np.asarray(m_atlas[0]).shape)
    h3 = (2.0 * math.pi) ** 3 / float(np.prod(n))
    theta = np.asarray(theta0, dtype=np.float64).copy()
    npar = tumor.np
    split = lambda th: (th[:npar], th[npar], th[npar + 1])
    v = [np.zeros(n) for _ in range(3)]
    c1 = np.zeros(n)
    q = [np.zeros(n) for _ in range(3)]
    hist = []
    for j, beta in enumerate(beta_schedule(beta_init, beta_final, final_repeats)):
        t0 = time.perf_counter()
        reg = make_reg(beta)
        # 1. warped atlas
        reg.rg_set_images(m_atlas, m_patient, c1, q)
        mw = [np.zeros(n) for _ in range(3)]
        reg.rg_forward(v, mw)
        # 2. tumor inversion in the warped atlas
        tumor.rd_set_tissue(*mw)
        tres = gn.gauss_newton(tumor, theta, iters=tumor_iters, cg_maxit=tumor_cg, forcing=tumor_forcing)
        theta = tres.theta
        # 3. c(1) and q of the new parameters
        c1 = np.zeros(n)
        J_T = tumor.rd_forward(*split(theta), c1)
        tumor.rd_adjoint()
        q = list(tumor.rd_coupling_field())
        # 4. modified registration problem from v
        reg.rg_set_images(m_atlas, m_patient, c1, q)
        J_R0 = reg.rg_forward(v)
        rres = reg_gn.gauss_newton(reg, v, h3, iters=reg_iters, cg_maxit=reg_cg)
        v = rres.v
        rec = {"iter": j, "beta_v": beta, "tumor_objective": J_T, "tumor_iters": len(tres.history),
               "reg_objective_start": J_R0, "reg_objective": rres.objective, "reg_iters": len(rres.history),
               "k_f": float(theta[npar]), "rho_f": float(theta[npar + 1]), "seconds": time.perf_counter() - t0}
        hist.append(rec)
        if callback:
            callback(rec, theta, v)
    return PicardResult(theta=theta, v=v, history=hist)
