"""The tumor inversion solver (l1 GIST + Hoyer beta search, weighted-l2
L-BFGS) driven by the CUDA context on a small two-site calibration problem."""

import math

import numpy as np
import pytest

pytest.importorskip("torch")

from oracle import rd as orc
from paper_1907_07774_gb300 import rd as R
from paper_1907_07774_gb300 import synth
from paper_1907_07774_gb300 import tumor_inv as T

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1907_07774_gb300 import build
    build.build()


def test_tumor_inversion_on_gpu_gives_a_sparse_start_and_lowers_the_misfit():
    prob = synth.calibration_problem(n=32, nt=8, m=4, sigma=2 * math.pi / 16)
    M = orc.model_from_problem(prob, rtol=1e-12, kind="numpy")
    c_true, _ = M.forward(prob.p_true, prob.k_f_true, prob.rho_f_true)
    d = synth.labels(c_true, synth.ellipsoid_mask(prob.n), 7)
    ctx = R.context_for(prob, prec="mixed", pcg_rtol=1e-6, pcg_maxit=500)
    ctx.rd_set_data(d)
    out = T.tumor_inversion(ctx, rho_f=prob.rho_f_true, k_f_l2=0.02, beta_steps=5,
                            gist_kw={"maxit": 40, "tau_j": 1e-6}, tau_s=0.1, w_large=1.0,
                            w_small=0.0, beta_l2=1e-4, opttol=1e-3, l2_maxit=20)
    l1 = out.l1
    assert np.any(l1.p) and l1.sparsity >= 0.95
    # the search bisected: both a too-dense and a sparse-enough beta were tried
    assert any(t["sparsity"] < 0.95 and t["nnz"] > 0 for t in l1.tried)
    # the l2 phase lowers the misfit well below its start and keeps k_f >= 0
    J0 = ctx.rd_forward(l1.p, 0.02, prob.rho_f_true)
    assert out.misfit < 0.8 * J0
    assert out.k_f >= 0.0
    fs = [h["f"] for h in out.l2.history]
    assert fs and all(b < a for a, b in zip(fs, fs[1:])), [(h["f"], h["ls"]) for h in out.l2.history]
