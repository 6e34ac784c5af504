"""Writes the stored FP64 oracle results of the full-size calibration cases
under tests/golden/ (regression fixtures of the oracle at the grids where the
CUDA path runs its production kernels; the paper prints no worked example
that could serve).

Calls only the oracle and the seeded input recipe.  Each case is one run of
the oracle's gradient (Sec. 3.1: state solve, adjoint solve, then Eq.
``tumor:inv`` and ``tumor:inv_diff``), optionally followed by one Gauss-Newton
Hessian-vector product for a seeded direction; the target labels are those of
the oracle's own ``c_true(1)`` (threshold 0.5, 1 % seeded flips inside the
ellipsoid).  Stored: the labels (packed bits), the misfit, the gradient, the
Hessian-vector product, the PCG iterations of every solve, checksums of
``c(1)`` and ``alpha(0)`` (sum, sum of squares and the inner product with a
seeded weight field) and the three planes of ``c(1)`` through the centre of
the grid.

Run from the repository root, one case per process (the 256^3 cases take
hours on one core):

    python tests/golden/make_golden_full.py grad128_nt16
    python tests/golden/make_golden_full.py grad256_nt2
    python tests/golden/make_golden_full.py grad256_nt32
    python tests/golden/make_golden_full.py work256_nt32_rtol1e-6

A change of a stored value is a change of the oracle's arithmetic and names,
in its commit message, the passage of the paper that justifies it."""

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import rd as orc  # noqa: E402
from paper_1907_07774_gb300 import synth  # noqa: E402

# calibration recipe: m^3 Gaussians of width 2 pi / 64, tissue seed 1000,
# label seed 1007, evaluation point p = 0.1 truth + 0.05, k_f = 0.02,
# rho_f = 6; data from k_f = 0.05, rho_f = 10
CASES = {
    # config 1 of the workload list: 128^3, nt = 16, 4^3 Gaussians
    "grad128_nt16": {"n": 128, "nt": 16, "m": 4, "rtol": 1e-12, "hessvec": True, "alpha_plane": True},
    # the benchmark grid with two time steps: every production kernel at L = 256
    "grad256_nt2": {"n": 256, "nt": 2, "m": 5, "rtol": 1e-12, "hessvec": True, "alpha_plane": False},
    # the benchmark workload itself (256^3, nt = 32, 5^3 Gaussians)
    "grad256_nt32": {"n": 256, "nt": 32, "m": 5, "rtol": 1e-12, "hessvec": False, "alpha_plane": False},
    # the benchmark workload at the benchmark's stopping tolerance: the
    # oracle's own PCG work for the same gradient (CPU baseline)
    "work256_nt32_rtol1e-6": {"n": 256, "nt": 32, "m": 5, "rtol": 1e-6, "hessvec": False, "alpha_plane": False},
}
SEED = 1000
WEIGHT_SEED = 2024
DIR_SEED = 77


def weight_field(n):
    """Seeded weights for the inner-product checksums (input recipe only)."""
    return np.random.default_rng(WEIGHT_SEED).standard_normal((n, n, n))


def checksums(u, w):
    return {"sum": float(u.sum()), "sumsq": float((u * u).sum()), "dot_w": float((u * w).sum())}


def paths(name):
    return os.path.join(HERE, f"oracle_full_{name}.json"), os.path.join(HERE, f"oracle_full_{name}.npz")


def problem(case):
    return synth.calibration_problem(n=case["n"], nt=case["nt"], m=case["m"], seed=SEED)


def direction(np_total):
    return synth.random_directions(1, np_total, DIR_SEED)[0]


def compute(name, fft_kind="numpy"):
    case = CASES[name]
    n = case["n"]
    prob = problem(case)
    M = orc.model_from_problem(prob, rtol=case["rtol"], maxit=5000, kind=fft_kind)
    t0 = time.perf_counter()
    c_true = M.forward(prob.p_true, prob.k_f_true, prob.rho_f_true)[0]   # its trajectory is not kept
    d = synth.labels(c_true, synth.ellipsoid_mask(prob.n), prob.seed + 7)
    del c_true
    M.iters = []
    t1 = time.perf_counter()
    p = np.asarray(prob.p, dtype=np.float64)
    c1, traj = M.forward(p, prob.k_f, prob.rho_f)
    fwd_iters = list(M.iters)
    J = M.misfit(c1, d, p)
    alpha0, g_kf, g_rho = M.adjoint(traj, M.final_adjoint(c1, d), prob.k_f, prob.rho_f)
    g = np.concatenate([-M.h3 * M.phi_t(alpha0), [g_kf, g_rho]])
    adj_iters = list(M.iters[len(fwd_iters):])
    t2 = time.perf_counter()
    w = weight_field(n)
    out = {"case": dict(case, name=name, seed=SEED, label_seed=prob.seed + 7, weight_seed=WEIGHT_SEED),
           "labels_sum": float(d.sum()), "misfit": float(J), "gradient": [float(x) for x in g],
           "c1": checksums(c1, w), "alpha0": checksums(alpha0, w),
           "pcg_iters_forward": fwd_iters, "pcg_iters_adjoint": adj_iters,
           "seconds_gradient": t2 - t1, "seconds_data": t1 - t0}
    arrays = {"labels_bits": np.packbits(d.astype(bool).ravel()),
              "c1_plane0": c1[n // 2, :, :].copy(), "c1_plane1": c1[:, n // 2, :].copy(),
              "c1_plane2": c1[:, :, n // 2].copy()}
    if case["alpha_plane"]:
        arrays["alpha0_plane0"] = alpha0[n // 2, :, :].copy()
    del w
    if case["hessvec"]:
        v = direction(len(p) + 2)
        M.iters = []
        t3 = time.perf_counter()
        hv = M.hessvec(p, prob.k_f, prob.rho_f, v, traj=traj)
        out["hessvec_direction_seed"] = DIR_SEED
        out["hessvec"] = [float(x) for x in hv]
        out["pcg_iters_hessvec"] = list(M.iters)
        out["seconds_hessvec"] = time.perf_counter() - t3
    return out, arrays


def load(name):
    """(stored scalars, stored arrays with the labels unpacked)."""
    js, nz = paths(name)
    with open(js) as f:
        want = json.load(f)
    z = np.load(nz)
    n = want["case"]["n"]
    arr = {k: z[k] for k in z.files if k != "labels_bits"}
    arr["labels"] = np.unpackbits(z["labels_bits"])[: n ** 3].reshape(n, n, n).astype(np.float64)
    return want, arr


if __name__ == "__main__":
    # optional second argument: threads for the library FFT (scipy), which
    # only shortens the run; the numpy and scipy transforms agree to rounding
    name = sys.argv[1]
    threads = int(sys.argv[2]) if len(sys.argv) > 2 else 0
    if threads > 0:
        from oracle import fft as _fft
        _fft.SCIPY_WORKERS = threads
    out, arrays = compute(name, "scipy" if threads > 0 else "numpy")
    out["case"]["fft"] = f"scipy, {threads} threads" if threads > 0 else "numpy"
    js, nz = paths(name)
    np.savez_compressed(nz, **arrays)
    with open(js, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print("wrote", js, nz)
