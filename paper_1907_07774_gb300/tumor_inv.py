"""The tumor inversion solver of Sec. 2.3 and Sec. 3.1: an l1 phase (GIST with
a Hoyer-driven binary search for beta_p) followed by a weighted-l2 phase
(L-BFGS with the More-Thuente line search) on (p, k_f).

Everything here runs on the host over the n_p + 2 parameters; each objective
value is one state solve (``rd_forward``) and each gradient one adjoint
(``rd_adjoint`` after that solve, or ``rd_gradient``), all in the CUDA library.
The context's own ``beta_p`` term should be 0: the regularisers of this
module are added here.

Readings where the paper leaves room:

* l1 phase objective: ``F(p) = D(p) + beta ||p||_1`` with D the context's
  misfit (D_c, plus D_m with Moving-Atlas data) at fixed ``k_f``, ``rho_f``.
  The soft threshold ``sign(x) max(0, |x| - alpha beta)`` printed in Sec. 3.1
  is the proximal map of ``alpha beta ||.||_1``, so that is the regulariser
  (the 1/2 ||p||_1^2 of Sec. 2.3 and the alpha beta / 2 of the subproblem are
  not used).
* Step length: Barzilai-Borwein ``s.s / s.y`` as the first trial (GIST), then
  halving until ``F(p+) <= F(p) - sigma / (2 alpha) ||p+ - p||^2`` (the
  Armijo rule of a proximal step).
* Stopping: both tests of Sec. 3.1 must hold (objective change below
  ``tau_J (1 + F(p^0))`` and ``||dp||_inf < sqrt(tau_J) (1 + ||p+||_inf)``).
* beta search: bisection on ``[0, ||grad D(p^0)||_inf]``; a solution with
  Hoyer sparsity >= target lowers beta, a denser one raises it; the zero
  vector counts as too sparse.  The result is the smallest tried beta whose
  solution is non-zero and sparse enough.
* ``p >= 0`` (default ``nonneg=True``): with positive Gaussians, c(0) = Phi p
  is a concentration only for non-negative p, and a negative c(0) drives the
  exact logistic step towards its singular denominator.  The l1 prox is then
  the one-sided threshold ``max(0, x - alpha beta)``.
* A trial point whose solve fails with a non-finite value is treated as a
  failed trial: GIST halves alpha, L-BFGS restarts the line search from a
  ten times shorter step.
* l2 phase: the bound ``k_f >= 0`` caps the line-search step (``stpmax``);
  on the bound, k_f is held fixed while its gradient points outward, and
  convergence is measured on the projected gradient.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


class NonFiniteTrial(Exception):
    """A trial point whose state or adjoint solve produced a non-finite value."""


def _is_nonfinite_error(exc):
    # the library reports RD_ERR_NONFINITE (6) through RDError.status
    return getattr(exc, "status", None) == 6


def _forward(solver, p, k_f, rho_f):
    try:
        J = solver.rd_forward(p, k_f, rho_f)
    except Exception as exc:
        if _is_nonfinite_error(exc):
            return math.inf
        raise
    return J if np.isfinite(J) else math.inf


def _gradient(solver, p, k_f, rho_f):
    try:
        J, g = solver.rd_gradient(p, k_f, rho_f)
    except Exception as exc:
        if _is_nonfinite_error(exc):
            raise NonFiniteTrial() from exc
        raise
    g = np.asarray(g, dtype=np.float64)
    if not (np.isfinite(J) and np.all(np.isfinite(g))):
        raise NonFiniteTrial()
    return J, g


# ------------------------------------------------------------------ l1 phase
def soft_threshold(x, t, nonneg=False):
    """``sign(x) max(0, |x| - t)`` elementwise (the closed form of Sec. 3.1);
    with ``nonneg`` the prox of ``t |.|`` plus the constraint ``>= 0``,
    ``max(0, x - t)``."""
    if nonneg:
        return np.maximum(0.0, x - t)
    return np.sign(x) * np.maximum(0.0, np.abs(x) - t)


def hoyer(p):
    """Sparsity measure of Sec. 3.1: ``(n - ||p||_1 / ||p||_inf) / (n - 1)``,
    1 for a single non-zero entry, 0 for equal magnitudes everywhere; the
    zero vector (no magnitude to compare) gives 1."""
    p = np.asarray(p, dtype=np.float64)
    n = p.size
    if n < 2:
        return 1.0
    m = float(np.max(np.abs(p)))
    if m == 0.0:
        return 1.0
    return (n - float(np.sum(np.abs(p))) / m) / (n - 1)


def l2_weights(p_l1, tau_s, w_large, w_small):
    """Weights of the l2 phase (Sec. 2.3): ``w_large`` where
    ``|p_i| < tau_s ||p||_inf``, else ``w_small``."""
    p_l1 = np.asarray(p_l1, dtype=np.float64)
    cut = tau_s * float(np.max(np.abs(p_l1))) if p_l1.size else 0.0
    return np.where(np.abs(p_l1) < cut, w_large, w_small).astype(np.float64)


@dataclass
class GistResult:
    p: np.ndarray
    objective: float
    misfit: float
    iters: int
    evals: int
    converged: bool
    history: list = field(default_factory=list)


def gist(solver, p0, k_f, rho_f, beta, alpha0=1.0, sigma=1e-5, tau_j=1e-4, maxit=50,
         max_backtracks=60, alpha_min=1e-30, alpha_max=1e10, nonneg=True):
    """GIST (Sec. 3.1) on ``F(p) = D(p) + beta ||p||_1`` at fixed k_f, rho_f.

    Each iteration takes a gradient step of length alpha on D, applies the
    soft threshold ``alpha beta``, halves alpha until the proximal Armijo
    condition holds, and proposes the next alpha by Barzilai-Borwein."""
    npar = solver.np
    p = np.asarray(p0, dtype=np.float64).copy()
    if nonneg:
        p = np.maximum(p, 0.0)
    D, g = _gradient(solver, p, k_f, rho_f)
    g = g[:npar]
    F = D + beta * float(np.sum(np.abs(p)))
    F0 = F
    alpha = float(alpha0)
    evals = 1
    hist = []
    converged = False
    it = 0
    for it in range(1, maxit + 1):
        accepted = False
        for _ in range(max_backtracks):
            p_new = soft_threshold(p - alpha * g, alpha * beta, nonneg)
            D_new = _forward(solver, p_new, k_f, rho_f)
            evals += 1
            F_new = D_new + beta * float(np.sum(np.abs(p_new)))
            dp = p_new - p
            if np.isfinite(F_new) and F_new <= F - sigma / (2.0 * alpha) * float(dp @ dp):
                accepted = True
                break
            alpha *= 0.5
            if alpha < alpha_min:
                break
        if not accepted:
            break
        g_new = np.asarray(solver.rd_adjoint()[:npar], dtype=np.float64)
        s, y = dp, g_new - g
        small_change = abs(F_new - F) < tau_j * (1.0 + F0)
        small_step = float(np.max(np.abs(dp))) < math.sqrt(tau_j) * (1.0 + float(np.max(np.abs(p_new))))
        hist.append({"iter": it, "objective": F_new, "misfit": D_new, "alpha": alpha,
                     "nnz": int(np.count_nonzero(p_new))})
        p, g, F, D = p_new, g_new, F_new, D_new
        if small_change and small_step:
            converged = True
            break
        sy = float(s @ y)
        # Barzilai-Borwein; without positive curvature along s, try a longer step
        alpha = min(max(float(s @ s) / sy, alpha_min), alpha_max) if sy > 0.0 else min(2.0 * alpha, alpha_max)
        if not np.isfinite(alpha):
            alpha = alpha0
    return GistResult(p=p, objective=F, misfit=D, iters=it, evals=evals, converged=converged, history=hist)


@dataclass
class BetaSearchResult:
    p: np.ndarray
    beta: float
    sparsity: float
    tried: list


def beta_search(solver, p0, k_f, rho_f, target=0.95, steps=6, beta_max=None, **gist_kw):
    """beta_p continuation by binary search on the Hoyer sparsity (Sec. 3.1):
    start from ``beta_max = ||grad D(p0)||_inf`` and bisect, warm-starting
    each GIST solve from the last sparse-enough solution."""
    npar = solver.np
    p0 = np.asarray(p0, dtype=np.float64)
    if beta_max is None:
        _, g0 = _gradient(solver, p0, k_f, rho_f)
        beta_max = float(np.max(np.abs(g0[:npar])))
    lo, hi = 0.0, float(beta_max)
    beta = hi
    best = None
    start = p0
    tried = []
    for _ in range(steps):
        res = gist(solver, start, k_f, rho_f, beta, **gist_kw)
        hs = hoyer(res.p)
        nonzero = bool(np.any(res.p != 0.0))
        tried.append({"beta": beta, "sparsity": hs, "nnz": int(np.count_nonzero(res.p)),
                      "objective": res.objective, "iters": res.iters})
        if nonzero and hs >= target:
            best = (beta, res.p, hs)
            hi = beta
            start = res.p
        elif not nonzero:
            hi = beta
        else:
            lo = beta
        beta = 0.5 * (lo + hi)
    if best is None:
        return BetaSearchResult(p=res.p, beta=tried[-1]["beta"], sparsity=tried[-1]["sparsity"], tried=tried)
    return BetaSearchResult(p=best[1], beta=best[0], sparsity=best[2], tried=tried)


# ---------------------------------------------------------- line search
def _trial_step(stx, fx, dx, sty, fy, dy, stp, fp, dp, brackt, stmin, stmax):
    """One safeguarded update of the More-Thuente interval (More and Thuente,
    ACM TOMS 20(3), 1994, Sec. 4): chooses the next trial from cubic,
    quadratic and secant models of the two best points and the trial, and
    shrinks the interval [stx, sty] that brackets a step satisfying the
    strong Wolfe conditions.  Returns the new state."""
    sgnd = dp * (dx / abs(dx)) if dx != 0.0 else 0.0

    def cubic_min(a, fa, da, b, fb, db):
        # minimiser of the cubic interpolating f and f' at a and b
        theta = 3.0 * (fa - fb) / (b - a) + da + db
        s = max(abs(theta), abs(da), abs(db))
        gamma = s * math.sqrt(max(0.0, (theta / s) ** 2 - (da / s) * (db / s)))
        if b < a:
            gamma = -gamma
        pp = (gamma - da) + theta
        qq = ((gamma - da) + gamma) + db
        return a + (pp / qq) * (b - a)

    if fp > fx:
        # case 1: higher value, the minimiser lies between stx and stp
        stpc = cubic_min(stx, fx, dx, stp, fp, dp)
        stpq = stx + ((dx / ((fx - fp) / (stp - stx) + dx)) / 2.0) * (stp - stx)
        stpf = stpc if abs(stpc - stx) < abs(stpq - stx) else stpc + (stpq - stpc) / 2.0
        brackt = True
    elif sgnd < 0.0:
        # case 2: lower value, derivatives of opposite sign
        stpc = cubic_min(stp, fp, dp, stx, fx, dx)
        stpq = stp + (dp / (dp - dx)) * (stx - stp)
        stpf = stpc if abs(stpc - stp) > abs(stpq - stp) else stpq
        brackt = True
    elif abs(dp) < abs(dx):
        # case 3: lower value, same sign, derivative shrinking
        theta = 3.0 * (fx - fp) / (stp - stx) + dx + dp
        s = max(abs(theta), abs(dx), abs(dp))
        gamma = s * math.sqrt(max(0.0, (theta / s) ** 2 - (dx / s) * (dp / s)))
        if stp > stx:
            gamma = -gamma
        pp = (gamma - dp) + theta
        qq = (gamma + (dx - dp)) + gamma
        r = pp / qq
        if r < 0.0 and gamma != 0.0:
            stpc = stp + r * (stx - stp)
        elif stp > stx:
            stpc = stmax
        else:
            stpc = stmin
        stpq = stp + (dp / (dp - dx)) * (stx - stp)
        if brackt:
            stpf = stpc if abs(stpc - stp) < abs(stpq - stp) else stpq
            if stp > stx:
                stpf = min(stp + 0.66 * (sty - stp), stpf)
            else:
                stpf = max(stp + 0.66 * (sty - stp), stpf)
        else:
            stpf = stpc if abs(stpc - stp) > abs(stpq - stp) else stpq
            stpf = min(stmax, max(stmin, stpf))
    else:
        # case 4: lower value, same sign, derivative not shrinking
        if brackt:
            stpf = cubic_min(stp, fp, dp, sty, fy, dy)
        else:
            stpf = stmax if stp > stx else stmin
    # update the interval
    if fp > fx:
        sty, fy, dy = stp, fp, dp
    else:
        if sgnd < 0.0:
            sty, fy, dy = stx, fx, dx
        stx, fx, dx = stp, fp, dp
    return stx, fx, dx, sty, fy, dy, stpf, brackt


@dataclass
class LineSearchResult:
    stp: float
    f: float
    g: float
    evals: int
    status: str      # "wolfe", "stpmax", "stpmin", "xtol", "rounding", "maxfev"


def more_thuente(phi, f0, g0, stp=1.0, ftol=1e-4, gtol=0.9, xtol=0.1, stpmin=0.0, stpmax=1e10, maxfev=20):
    """Line search for a step satisfying the strong Wolfe conditions
    ``phi(a) <= phi(0) + ftol a phi'(0)`` and ``|phi'(a)| <= gtol |phi'(0)|``
    (More and Thuente 1994).  ``phi(a)`` returns ``(value, derivative)``;
    ``g0 = phi'(0)`` must be negative."""
    if not g0 < 0.0:
        raise ValueError("not a descent direction")
    stp = min(max(stp, stpmin), stpmax)
    gtest = ftol * g0
    width = stpmax - stpmin
    width1 = 2.0 * width
    brackt = False
    stage = 1
    stx = sty = 0.0
    fx = fy = f0
    gx = gy = g0
    stmin, stmax = 0.0, stp + 4.0 * stp
    evals = 0
    f, g = f0, g0
    while True:
        f, g = phi(stp)
        evals += 1
        ftest = f0 + stp * gtest
        if stage == 1 and f <= ftest and g >= 0.0:
            stage = 2
        # exits, most significant first: strong Wolfe, then the bounds, the
        # interval width and rounding
        if f <= ftest and abs(g) <= gtol * (-g0):
            return LineSearchResult(stp, f, g, evals, "wolfe")
        if stp == stpmin and (f > ftest or g >= gtest):
            return LineSearchResult(stp, f, g, evals, "stpmin")
        if stp == stpmax and f <= ftest and g <= gtest:
            return LineSearchResult(stp, f, g, evals, "stpmax")
        if brackt and stmax - stmin <= xtol * stmax:
            return LineSearchResult(stp, f, g, evals, "xtol")
        if brackt and (stp <= stmin or stp >= stmax):
            return LineSearchResult(stp, f, g, evals, "rounding")
        if evals >= maxfev:
            return LineSearchResult(stp, f, g, evals, "maxfev")
        if stage == 1 and f <= fx and f > ftest:
            # first stage: work on psi(a) = phi(a) - phi(0) - ftol a phi'(0)
            fm, fxm, fym = f - stp * gtest, fx - stx * gtest, fy - sty * gtest
            gm, gxm, gym = g - gtest, gx - gtest, gy - gtest
            stx, fxm, gxm, sty, fym, gym, stp, brackt = _trial_step(
                stx, fxm, gxm, sty, fym, gym, stp, fm, gm, brackt, stmin, stmax)
            fx, fy = fxm + stx * gtest, fym + sty * gtest
            gx, gy = gxm + gtest, gym + gtest
        else:
            stx, fx, gx, sty, fy, gy, stp, brackt = _trial_step(
                stx, fx, gx, sty, fy, gy, stp, f, g, brackt, stmin, stmax)
        if brackt:
            # force sufficient shrinkage of the interval
            if abs(sty - stx) >= 0.66 * width1:
                stp = stx + 0.5 * (sty - stx)
            width1 = width
            width = abs(sty - stx)
            stmin, stmax = min(stx, sty), max(stx, sty)
        else:
            stmin = stp + 1.1 * (stp - stx)
            stmax = stp + 4.0 * (stp - stx)
        stp = min(max(stp, stpmin), stpmax)
        if (brackt and (stp <= stmin or stp >= stmax)) or (brackt and stmax - stmin <= xtol * stmax):
            stp = stx


# ---------------------------------------------------------------- L-BFGS
def lbfgs_direction(g, S, Y):
    """``-H g`` by the two-loop recursion (Nocedal and Wright, Algorithm 7.4)
    over the stored pairs (oldest first), initial matrix ``gamma I`` with
    ``gamma = s.y / y.y`` of the newest pair."""
    q = np.array(g, dtype=np.float64)
    a = []
    for s, y in zip(reversed(S), reversed(Y)):
        r = 1.0 / float(y @ s)
        ai = r * float(s @ q)
        q -= ai * y
        a.append((r, ai))
    if S:
        q *= float(S[-1] @ Y[-1]) / float(Y[-1] @ Y[-1])
    for (s, y), (r, ai) in zip(zip(S, Y), reversed(a)):
        b = r * float(y @ q)
        q += (ai - b) * s
    return -q


@dataclass
class LbfgsResult:
    x: np.ndarray
    f: float
    g: np.ndarray
    iters: int
    evals: int
    converged: bool
    history: list = field(default_factory=list)


def lbfgs(fg, x0, m=10, maxit=100, gtol_rel=1e-5, g_ref=None, lower=None, ls_kw=None, callback=None):
    """L-BFGS with the More-Thuente line search on ``fg(x) -> (f, grad)``.
    Stops when the projected gradient satisfies ``|P grad| <= gtol_rel
    |g_ref|`` (g_ref: the gradient at x0 if not given).

    ``lower``: optional lower bounds (-inf where none).  Variables on their
    bound whose gradient or search direction points out of the feasible set
    are held fixed for the iteration (the two-loop recursion then runs on
    the free variables only), and the line-search step is capped so that the
    iterate stays feasible."""
    ls_kw = dict(ls_kw or {})
    x = np.asarray(x0, dtype=np.float64).copy()
    lo = None if lower is None else np.asarray(lower, dtype=np.float64)
    if lo is not None:
        x = np.maximum(x, lo)
    f, g = fg(x)
    g = np.asarray(g, dtype=np.float64)
    evals = 1
    gref = float(np.linalg.norm(g if g_ref is None else g_ref))
    S, Y, hist = [], [], []
    converged = False

    def active_set(x, g):
        if lo is None:
            return np.zeros(x.size, dtype=bool)
        return (x <= lo) & (g > 0.0)

    def direction(g, act):
        free = ~act
        if not act.any():
            return lbfgs_direction(g, S, Y)
        pairs = [(s_[free], y_[free]) for s_, y_ in zip(S, Y) if float(s_[free] @ y_[free]) > 0.0]
        d = np.zeros_like(g)
        d[free] = lbfgs_direction(g[free], [a for a, _ in pairs], [b for _, b in pairs])
        return d

    it = 0
    for it in range(1, maxit + 1):
        act = active_set(x, g)
        gp = np.where(act, 0.0, g)
        if float(np.linalg.norm(gp)) <= gtol_rel * gref:
            converged = True
            it -= 1
            break
        d = direction(g, act)
        if lo is not None:
            # hold variables on the bound that the direction would push out
            for _ in range(x.size):
                out = (x <= lo) & (d < 0.0) & ~act
                if not out.any():
                    break
                act = act | out
                d = direction(g, act)
        slope = float(g @ d)
        if not slope < 0.0:
            d = -np.where(act, 0.0, g)
            slope = float(g @ d)
            if not slope < 0.0:
                converged = True
                break
        stpmax = 1e10
        if lo is not None:
            neg = d < 0.0
            if np.any(neg):
                stpmax = max(float(np.min((lo[neg] - x[neg]) / d[neg])), 0.0)
        stp0 = 1.0 if S else min(1.0, 1.0 / max(float(np.linalg.norm(d)), 1e-300))
        cache = {}

        def phi(a):
            xa = x + a * d
            if lo is not None:
                xa = np.maximum(xa, lo)
            fa, ga = fg(xa)
            ga = np.asarray(ga, dtype=np.float64)
            cache[a] = (xa, fa, ga)
            return fa, float(ga @ d)

        ls = None
        stp_try = min(stp0, stpmax)
        for _ in range(12):
            try:
                ls = more_thuente(phi, f, slope, stp=stp_try, stpmin=0.0, stpmax=stpmax, **ls_kw)
                break
            except NonFiniteTrial:
                evals += 1
                stp_try *= 0.1
                stpmax = stp_try      # never step back into the failing region
        if ls is None:
            break
        evals += ls.evals
        x_new, f_new, g_new = cache[ls.stp]
        if not f_new < f:
            break
        s, y = x_new - x, g_new - g
        if float(s @ y) > 1e-12 * float(np.linalg.norm(s)) * float(np.linalg.norm(y)):
            S.append(s)
            Y.append(y)
            if len(S) > m:
                S.pop(0)
                Y.pop(0)
        x, f, g = x_new, f_new, g_new
        rec = {"iter": it, "f": f, "grad_norm": float(np.linalg.norm(np.where(active_set(x, g), 0.0, g))),
               "step": ls.stp, "ls": ls.status, "evals": ls.evals}
        hist.append(rec)
        if callback:
            callback(rec, x)
    return LbfgsResult(x=x, f=f, g=g, iters=it, evals=evals, converged=converged, history=hist)


# ---------------------------------------------------------------- l2 phase
@dataclass
class TumorInversionResult:
    p: np.ndarray
    k_f: float
    rho_f: float
    misfit: float
    beta_l1: float
    sparsity: float
    weights: np.ndarray
    l1: BetaSearchResult
    l2: LbfgsResult


def weighted_l2(solver, p0, k_f0, rho_f, beta, weights, invert_rho=False, k_f_scale=None,
                rho_scale=None, opttol=1e-3, maxit=50, m=10, g_ref=None, callback=None, nonneg=True):
    """Weighted-l2 phase: L-BFGS + More-Thuente on
    ``D(p, k_f) + beta / 2 sum_i w_i p_i^2`` (Sec. 2.3, Sec. 3.1), k_f >= 0,
    optionally also rho_f.  Variables are scaled (k_f by ``k_f_scale``,
    default ``max(k_f0, 1e-2)``; ``"auto"``: the scale that gives k_f's
    initial scaled gradient the root-mean-square size of the p components,
    so that the first quasi-Newton steps move both).  Stops when the gradient norm falls below
    ``opttol`` times the reference gradient, by default the gradient at
    p = 0 (Sec. 3.1)."""
    npar = solver.np
    w = np.asarray(weights, dtype=np.float64)
    if isinstance(k_f_scale, str) and k_f_scale == "auto":
        p0v = np.asarray(p0, dtype=np.float64)
        _, g0 = _gradient(solver, p0v, max(float(k_f0), 0.0), rho_f)
        rms = math.sqrt(float(np.mean((g0[:npar] + beta * w * p0v) ** 2)))
        gk = abs(float(g0[npar]))
        ks = rms / gk if (gk > 0.0 and rms > 0.0) else max(abs(float(k_f0)), 1e-2)
    else:
        ks = float(k_f_scale) if k_f_scale else max(abs(float(k_f0)), 1e-2)
    rs = float(rho_scale) if rho_scale else max(abs(float(rho_f)), 1.0)
    nv = npar + (2 if invert_rho else 1)
    scale = np.ones(nv)
    scale[npar] = ks
    if invert_rho:
        scale[npar + 1] = rs

    def unpack(x):
        th = x * scale
        return th[:npar], th[npar], (th[npar + 1] if invert_rho else rho_f)

    def fg(x):
        p, kf, rf = unpack(x)
        J, g = _gradient(solver, p, max(kf, 0.0), rf)
        J = J + 0.5 * beta * float(np.sum(w * p * p))
        gx = np.empty(nv)
        gx[:npar] = g[:npar] + beta * w * p
        gx[npar] = g[npar]
        if invert_rho:
            gx[npar + 1] = g[npar + 1]
        return J, gx * scale

    x0 = np.concatenate([np.asarray(p0, dtype=np.float64), [k_f0]] + ([[rho_f]] if invert_rho else [])) / scale
    if g_ref is None:
        xr = x0.copy()
        xr[:npar] = 0.0
        g_ref = fg(xr)[1]
    lower = np.full(nv, -np.inf)
    lower[npar] = 0.0
    if nonneg:
        lower[:npar] = 0.0
    return lbfgs(fg, x0, m=m, maxit=maxit, gtol_rel=opttol, g_ref=g_ref, lower=lower, callback=callback), scale


def tumor_inversion(solver, rho_f, k_f_l2=None, p0=None, target=0.95, beta_steps=6, gist_kw=None,
                    tau_s=0.1, w_large=1.0, w_small=0.0, beta_l2=1e-4, opttol=1e-3, l2_maxit=50,
                    invert_rho=False, nonneg=True, k_f_scale="auto"):
    """Both phases (Sec. 2.3): l1 with k_f = 0 and the Hoyer beta search,
    then weighted l2 on (p, k_f) from the l1 solution; ``k_f_l2`` is the
    starting diffusivity of the l2 phase (default 0)."""
    npar = solver.np
    p0 = np.zeros(npar) if p0 is None else np.asarray(p0, dtype=np.float64)
    l1 = beta_search(solver, p0, 0.0, rho_f, target=target, steps=beta_steps,
                     **dict({"nonneg": nonneg}, **(gist_kw or {})))
    w = l2_weights(l1.p, tau_s, w_large, w_small)
    kf0 = 0.0 if k_f_l2 is None else float(k_f_l2)
    l2, scale = weighted_l2(solver, l1.p, kf0, rho_f, beta_l2, w, invert_rho=invert_rho, opttol=opttol,
                            maxit=l2_maxit, nonneg=nonneg, k_f_scale=k_f_scale)
    th = l2.x * scale
    rf = th[npar + 1] if invert_rho else rho_f
    return TumorInversionResult(p=th[:npar], k_f=max(th[npar], 0.0), rho_f=rf, misfit=l2.f, beta_l1=l1.beta,
                                sparsity=l1.sparsity, weights=w, l1=l1, l2=l2)
