"""Seeded synthetic inputs for the tumor reaction-diffusion calibration path.

This module holds input recipes only: tissue probability maps, the Gaussian
lattice of the initial-condition parametrisation, parameter vectors and the
thresholded/flipped target labels. It contains none of the solver's
arithmetic (no operator, no time stepping, no Gaussian basis evaluation), so
that both the FP64 CPU oracle and the CUDA path can consume the same inputs.

Recipes (all FP64, NumPy ``default_rng(seed)``):

* tissue maps (Sec. 2 notation, Eq. ``coeff_tumor``): three random fields
  ``f_j(x) = sum_w a_w cos(w.x) + b_w sin(w.x)`` over integer wave vectors
  ``0 < |w|_2 <= 6`` taken in a half space, ``a_w, b_w ~ N(0, 1/M)`` with
  ``M`` the number of such modes (unit pointwise variance, so the maps are
  smooth and the same continuous field is sampled at every grid size); a softmax
  over the three fields per voxel; the result multiplied by the indicator of
  an ellipsoid centred at ``(pi, pi, pi)`` with half-axes
  ``(0.8 pi, 0.9 pi, 0.7 pi)`` along array axes ``(0, 1, 2)``.  Field 0 is
  white matter, field 1 gray matter, field 2 CSF.
* Gaussian lattice (Sec. 4.1, "Common Model and Numerical Parameters"):
  ``m^3`` centres ``pi + (j - (m - 1)/2) * delta`` per axis.
* target labels (Sec. 4.3, selection function ``H``): ``d = [c >= 0.5]``
  followed by flipping a seeded fraction of the voxels inside the ellipsoid.

Grid convention: point ``i`` on an axis of length ``n`` sits at
``x = 2 pi i / n``; arrays are C-ordered ``[i0, i1, i2]`` with ``i2`` fastest.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

TWO_PI = 2.0 * math.pi
HALF_AXES = (0.8 * math.pi, 0.9 * math.pi, 0.7 * math.pi)


def grid_coords(n):
    """Coordinates ``2 pi i / n`` for each axis length in ``n`` (3-tuple)."""
    return [np.arange(k, dtype=np.float64) * (TWO_PI / k) for k in n]


def half_space_modes(radius=6):
    """Integer wave vectors with ``0 < |w| <= radius`` in the half space
    ``w0 > 0``, or ``w0 == 0 and w1 > 0``, or ``w0 == w1 == 0 and w2 > 0``,
    in lexicographic order."""
    out = []
    r2 = radius * radius
    for a in range(-radius, radius + 1):
        for b in range(-radius, radius + 1):
            for c in range(-radius, radius + 1):
                if a * a + b * b + c * c == 0 or a * a + b * b + c * c > r2:
                    continue
                if a > 0 or (a == 0 and b > 0) or (a == 0 and b == 0 and c > 0):
                    out.append((a, b, c))
    return np.array(out, dtype=np.int64)


def random_smooth_field(n, rng, radius=6):
    """``sum_w a_w cos(w.x) + b_w sin(w.x)`` on the grid, ``a, b ~ N(0,1/M)``.

    Evaluated by placing ``a_w - i b_w`` at index ``w mod n`` of a spectrum
    and taking the real part of its unnormalised inverse DFT (an input
    recipe; any exact evaluation of the trigonometric sum would do)."""
    modes = half_space_modes(radius)
    ab = rng.standard_normal((len(modes), 2)) / math.sqrt(len(modes))
    spec = np.zeros(tuple(n), dtype=np.complex128)
    idx = tuple((modes[:, a] % n[a]) for a in range(3))
    np.add.at(spec, idx, ab[:, 0] - 1j * ab[:, 1])
    return np.real(np.fft.ifftn(spec)) * float(np.prod(n))


def ellipsoid_mask(n, half_axes=HALF_AXES):
    x = grid_coords(n)
    r = ((x[0][:, None, None] - math.pi) / half_axes[0]) ** 2 \
        + ((x[1][None, :, None] - math.pi) / half_axes[1]) ** 2 \
        + ((x[2][None, None, :] - math.pi) / half_axes[2]) ** 2
    return (r <= 1.0).astype(np.float64)


def tissue_maps(n, seed):
    """``(m_WM, m_GM, m_CSF)`` as FP64 arrays of shape ``n``."""
    n = tuple(int(k) for k in n)
    rng = np.random.default_rng(seed)
    f = np.stack([random_smooth_field(n, rng) for _ in range(3)])
    f -= f.max(axis=0, keepdims=True)
    e = np.exp(f)
    sm = e / e.sum(axis=0, keepdims=True)
    mask = ellipsoid_mask(n)
    return sm[0] * mask, sm[1] * mask, sm[2] * mask


def lattice_centers(m, delta, center=(math.pi, math.pi, math.pi)):
    """``m^3`` Gaussian centres on a cubic lattice of spacing ``delta``
    (row-major over (axis0, axis1, axis2) lattice indices)."""
    off = (np.arange(m, dtype=np.float64) - 0.5 * (m - 1)) * delta
    c = np.stack(np.meshgrid(off + center[0], off + center[1], off + center[2],
                             indexing="ij"), axis=-1)
    return c.reshape(-1, 3)


def two_site_truth(m, value=0.5):
    """Ground-truth ``p``: two adjacent lattice sites next to the centre set
    to ``value``, the rest zero ("two nearby Gaussians enabled")."""
    p = np.zeros(m ** 3)
    a = (m - 1) // 2
    p[(a * m + a) * m + a] = value
    p[(a * m + a) * m + a + 1] = value
    return p


def labels(c1, mask, seed, threshold=0.5, flip_fraction=0.01):
    """Threshold ``c1`` at ``threshold`` (``>=`` maps to 1) and flip a seeded
    ``flip_fraction`` of the voxels inside ``mask``."""
    # C order throughout: the flips index the row-major flattening, and
    # reshape(-1) of a C-ordered array is a view, so they land in d (an input
    # with permuted strides, e.g. a GPU FFT output, would otherwise give a
    # copy and the flips would be lost)
    d = np.ascontiguousarray(np.asarray(c1) >= threshold, dtype=np.float64)
    inside = np.flatnonzero(np.ascontiguousarray(mask).reshape(-1) > 0)
    k = int(round(flip_fraction * inside.size))
    if k:
        rng = np.random.default_rng(seed)
        sel = rng.choice(inside, size=k, replace=False)
        flat = d.reshape(-1)
        flat[sel] = 1.0 - flat[sel]
    return d


@dataclass
class Problem:
    """One synthetic calibration problem (inputs only)."""
    n: tuple
    nt: int
    m_wm: np.ndarray
    m_gm: np.ndarray
    m_csf: np.ndarray
    centers: np.ndarray
    sigma: float
    p: np.ndarray
    k_f: float
    rho_f: float
    k_w: tuple = (1.0, 0.1, 0.0)
    rho_w: tuple = (1.0, 0.2, 0.0)
    p_true: np.ndarray | None = None
    k_f_true: float | None = None
    rho_f_true: float | None = None
    seed: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def h3(self):
        return float(np.prod([TWO_PI / k for k in self.n]))


def forward_problem(n=64, nt=16, seed=0):
    """Plain forward solve recipe: 8 Gaussians, sigma = 2 pi/64, a 2x2x2
    lattice of spacing 4h near the centre, weights U(0.2, 0.6) clipped to
    [0, 1], k_f = 0.05, rho_f = 8, k = (1, 0.1, 0), rho = (1, 0.2, 0)."""
    n3 = (n, n, n) if np.isscalar(n) else tuple(n)
    h = TWO_PI / n3[0]
    m_wm, m_gm, m_csf = tissue_maps(n3, seed)
    rng = np.random.default_rng(seed + 1)
    p = np.clip(rng.uniform(0.2, 0.6, size=8), 0.0, 1.0)
    return Problem(n=n3, nt=nt, m_wm=m_wm, m_gm=m_gm, m_csf=m_csf,
                   centers=lattice_centers(2, 4.0 * h), sigma=TWO_PI / 64.0,
                   p=p, k_f=0.05, rho_f=8.0, seed=seed)


def calibration_problem(n=128, nt=16, m=4, seed=1000, k_f_true=0.05,
                        rho_f_true=10.0, k_f=0.02, rho_f=6.0,
                        flip_fraction=0.01, sigma=TWO_PI / 64.0):
    """Gradient / Gauss-Newton recipe: ``m^3`` Gaussians of width ``sigma``
    on a lattice of spacing 1.5 sigma centred at (pi, pi, pi); truth = two
    adjacent central sites at 0.5 with (k_f_true, rho_f_true); evaluation
    point ``p = 0.1 * truth + 0.05``, ``(k_f, rho_f)``.  The target labels
    need ``c_true(1)``, which the caller computes and passes to
    :func:`labels`."""
    n3 = (n, n, n) if np.isscalar(n) else tuple(n)
    m_wm, m_gm, m_csf = tissue_maps(n3, seed)
    p_true = two_site_truth(m)
    return Problem(n=n3, nt=nt, m_wm=m_wm, m_gm=m_gm, m_csf=m_csf,
                   centers=lattice_centers(m, 1.5 * sigma), sigma=sigma,
                   p=0.1 * p_true + 0.05, k_f=k_f, rho_f=rho_f,
                   p_true=p_true, k_f_true=k_f_true, rho_f_true=rho_f_true,
                   seed=seed, extra={"flip_fraction": flip_fraction})


def random_directions(count, dim, seed):
    """Seeded unit directions for finite-difference checks."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((count, dim))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


# ------------------------------------------------------------ registration
# Inputs of the registration sub-problem (atlas and patient anatomy, a fixed
# tumor c(1), a coupling field q, divergence-free velocities).  Every field
# is a trigonometric sum evaluated exactly at arbitrary points, so the
# patient anatomy can be the atlas seen through a smooth displacement.
@dataclass
class TrigSum:
    """``sum_w a_w cos(w.x) + b_w sin(w.x)`` with its analytic derivatives."""
    modes: np.ndarray       # (M, 3) integer wave vectors
    a: np.ndarray           # (M,)
    b: np.ndarray           # (M,)

    @staticmethod
    def random(rng, radius, amp=1.0):
        modes = half_space_modes(radius)
        ab = rng.standard_normal((len(modes), 2)) * (amp / math.sqrt(len(modes)))
        return TrigSum(modes, ab[:, 0].copy(), ab[:, 1].copy())

    def _phase(self, X):
        return sum(self.modes[:, a][:, None] * X[a].reshape(1, -1) for a in range(3))

    def __call__(self, X):
        shape = X[0].shape
        out = np.zeros(X[0].size)
        for lo in range(0, len(self.modes), 64):      # chunks keep memory small
            sl = slice(lo, lo + 64)
            ph = sum(self.modes[sl, a][:, None] * X[a].reshape(1, -1) for a in range(3))
            out += self.a[sl] @ np.cos(ph) + self.b[sl] @ np.sin(ph)
        return out.reshape(shape)

    def _grid_spectrum(self, n, coef):
        spec = np.zeros(tuple(n), dtype=np.complex128)
        idx = tuple((self.modes[:, a] % n[a]) for a in range(3))
        np.add.at(spec, idx, coef)
        return np.real(np.fft.ifftn(spec)) * float(np.prod(n))

    def grid(self, n):
        """The sum on the grid of ``n`` (same values as ``self(coords_mesh(n))``,
        evaluated through one inverse DFT; exact while every |w_a| < n_a / 2)."""
        return self._grid_spectrum(n, self.a - 1j * self.b)

    def grid_deriv(self, n, axis):
        """``d/dx_axis`` of the sum on the grid, exactly as :meth:`deriv`."""
        return self._grid_spectrum(n, self.modes[:, axis] * (self.b + 1j * self.a))

    def deriv(self, X, axis):
        shape = X[0].shape
        out = np.zeros(X[0].size)
        w = self.modes[:, axis].astype(np.float64)
        for lo in range(0, len(self.modes), 64):
            sl = slice(lo, lo + 64)
            ph = sum(self.modes[sl, a][:, None] * X[a].reshape(1, -1) for a in range(3))
            out += (w[sl] * self.b[sl]) @ np.cos(ph) - (w[sl] * self.a[sl]) @ np.sin(ph)
        return out.reshape(shape)


def coords_mesh(n):
    x = grid_coords(n)
    return np.meshgrid(x[0], x[1], x[2], indexing="ij")


def curl_field(pots, X):
    """``curl A`` of three trigonometric potentials at the points X:
    divergence-free by construction."""
    d = lambda c, a: pots[c].deriv(X, a)
    return [d(2, 1) - d(1, 2), d(0, 2) - d(2, 0), d(1, 0) - d(0, 1)]


def curl_field_grid(pots, n):
    """:func:`curl_field` on the grid of ``n``."""
    d = lambda c, a: pots[c].grid_deriv(n, a)
    return [d(2, 1) - d(1, 2), d(0, 2) - d(2, 0), d(1, 0) - d(0, 1)]


def smooth_anatomy(fields, X, half_axes=HALF_AXES, width=0.15, values=None):
    """Softmax of three smooth fields times a smooth ellipsoid indicator
    ``1 / (1 + exp((r - 1) / width))``, r the ellipsoid radius (``values``:
    the three fields already evaluated at X)."""
    f = np.stack(values if values is not None else [fl(X) for fl in fields])
    f -= f.max(axis=0, keepdims=True)
    e = np.exp(f)
    sm = e / e.sum(axis=0, keepdims=True)
    r = np.sqrt(sum(((X[a] - math.pi) / half_axes[a]) ** 2 for a in range(3)))
    mask = 1.0 / (1.0 + np.exp((r - 1.0) / width))
    return [sm[i] * mask for i in range(3)]


@dataclass
class RegistrationProblem:
    n: tuple
    nt: int
    m_atlas: list
    m_patient: list
    c1: np.ndarray
    q: list
    v: list            # a divergence-free test velocity
    directions: list   # divergence-free directions (lists of 3 fields)
    beta_v: float
    seed: int


def registration_problem(n=64, nt=8, seed=4000, radius=3, disp_amp=0.25, v_amp=0.3, q_amp=0.02,
                         beta_v=1e-2, ndir=2):
    """Atlas = smooth anatomy; patient = the atlas at ``x - u(x)`` with ``u``
    a smooth divergence-free displacement of amplitude ``disp_amp``; tumor
    c(1) = a Gaussian of width 0.5 at (pi, pi, pi) scaled to 0.9; q = small
    smooth fields; a test velocity and directions as curls of random
    potentials (wave vectors of norm <= radius)."""
    n3 = (n, n, n) if np.isscalar(n) else tuple(int(k) for k in n)
    rng = np.random.default_rng(seed)
    X = coords_mesh(n3)
    fields = [TrigSum.random(rng, radius, amp=2.0) for _ in range(3)]
    m_atlas = smooth_anatomy(fields, X, values=[fl.grid(n3) for fl in fields])
    upot = [TrigSum.random(rng, 2, amp=disp_amp / 2.0) for _ in range(3)]
    u = curl_field_grid(upot, n3)
    m_patient = smooth_anatomy(fields, [X[a] - u[a] for a in range(3)])
    r2 = sum((X[a] - math.pi) ** 2 for a in range(3))
    c1 = 0.9 * np.exp(-r2 / (2 * 0.5 ** 2))
    q = [TrigSum.random(rng, radius, amp=q_amp).grid(n3) for _ in range(3)]
    vpot = [TrigSum.random(rng, radius, amp=v_amp / radius) for _ in range(3)]
    v = curl_field_grid(vpot, n3)
    dirs = []
    for _ in range(ndir):
        pots = [TrigSum.random(rng, radius, amp=1.0 / radius) for _ in range(3)]
        dirs.append(curl_field_grid(pots, n3))
    return RegistrationProblem(n=n3, nt=nt, m_atlas=m_atlas, m_patient=m_patient, c1=c1, q=q, v=v,
                               directions=dirs, beta_v=beta_v, seed=seed)
