"""``torch.autograd`` view of the misfit J(p, k_f, rho_f).

``RDSolve.apply(p, k_f, rho_f, ctx)`` returns J as a 0-d FP64 tensor.  Its
forward runs the state solve (``rd_forward``, which keeps the trajectory or
its checkpoints on the device) and its backward runs the discrete adjoint
(``rd_adjoint``) of that same solve, so ``J.backward()`` fills ``p.grad``,
``k_f.grad`` and ``rho_f.grad`` with the reduced gradient of Eq. tumor:inv /
tumor:inv_diff (and the rho_f analogue).  All arithmetic runs in the CUDA
library; this module only moves the n_p + 2 parameters across.
"""

from __future__ import annotations

import numpy as np
import torch


def _theta(p, k_f, rho_f):
    return (np.asarray(p.detach().cpu(), dtype=np.float64).reshape(-1), float(k_f), float(rho_f))


class RDSolve(torch.autograd.Function):
    """J = 1/2 h^3 |c(1) - d|^2 (+ 1/2 beta_p |p|^2) with a hand-written adjoint."""

    @staticmethod
    def forward(fctx, p, k_f, rho_f, solver):
        pv, kf, rf = _theta(p, k_f, rho_f)
        J = solver.rd_forward(pv, kf, rf)
        fctx.solver = solver
        fctx.theta = (pv.copy(), kf, rf)
        fctx.p_meta = (p.device, p.dtype, p.shape)
        return torch.tensor(J, dtype=torch.float64, device=p.device)

    @staticmethod
    def backward(fctx, grad_out):
        solver = fctx.solver
        pv, kf, rf = fctx.theta
        cur = solver.last_theta
        if cur is None or cur[1] != kf or cur[2] != rf or not np.array_equal(cur[0], pv):
            solver.rd_forward(pv, kf, rf)        # another solve ran in between
        g = solver.rd_adjoint()
        dev, dt, shape = fctx.p_meta
        go = float(grad_out)
        gp = torch.as_tensor(go * g[:-2], dtype=dt, device=dev).reshape(shape)
        gk = torch.tensor(go * g[-2], dtype=torch.float64, device=dev)
        gr = torch.tensor(go * g[-1], dtype=torch.float64, device=dev)
        return gp, gk, gr, None


def misfit(p, k_f, rho_f, solver):
    """Differentiable misfit; see :class:`RDSolve`."""
    return RDSolve.apply(p, k_f, rho_f, solver)
