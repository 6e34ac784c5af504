"""The Picard iteration of the Moving-Atlas scheme on the GPU: tumor
inversion in the warped atlas, then the modified registration problem with
the tumor's c(1) and coupling field q, under beta_v continuation."""

import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1907_07774_gb300 import picard as P
from paper_1907_07774_gb300 import rd as R
from paper_1907_07774_gb300 import rg as RG
from paper_1907_07774_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1907_07774_gb300 import build
    build.build()


def test_picard_iteration_registers_the_atlas_and_fits_the_tumor():
    n, nt = (32, 32, 32), 8
    prob = synth.registration_problem(n=n, nt=4, seed=4800, disp_amp=0.25, q_amp=0.0)
    atlas, healthy = prob.m_atlas, prob.m_patient
    sigma = 2 * math.pi / 16
    centers = synth.lattice_centers(3, 1.5 * sigma)
    p_true = synth.two_site_truth(3)
    # the tumor grows in the patient's anatomy
    gen = R.Context(n, nt, len(p_true), prec="fp64")
    gen.rd_set_tissue(*healthy)
    gen.rd_set_basis(centers, sigma)
    c_true = np.zeros(n)
    gen.rd_forward(p_true, 0.05, 10.0, c_true)
    d = synth.labels(c_true, synth.ellipsoid_mask(n), 7)
    m_P = [m * (1.0 - c_true) for m in healthy]
    tumor = R.Context(n, nt, len(p_true), prec="mixed", pcg_rtol=1e-6, moving_atlas=True, coupling=True)
    tumor.rd_set_tissue(*atlas)
    tumor.rd_set_basis(centers, sigma)
    tumor.rd_set_data(d)
    tumor.rd_set_anatomy_data(*m_P)
    theta0 = np.concatenate([0.1 * p_true + 0.05, [0.02, 6.0]])
    J_T0 = tumor.rd_forward(theta0[:-2], theta0[-2], theta0[-1])
    make_reg = lambda beta: RG.RegContext(n, 4, prec="mixed", beta_v=beta)
    res = P.picard(tumor, make_reg, atlas, m_P, theta0, beta_init=1e-1, beta_final=1e-2, final_repeats=2,
                   tumor_iters=2, reg_iters=2)
    assert [h["beta_v"] for h in res.history] == pytest.approx([1e-1, 1e-2, 1e-2])
    for h in res.history:
        assert h["reg_objective"] < h["reg_objective_start"]
    assert res.history[-1]["tumor_objective"] < J_T0
    # the warped atlas moved towards the patient's healthy anatomy
    reg = make_reg(1e-2)
    reg.rg_set_images(atlas, m_P, np.zeros(n), None)
    mw = [np.zeros(n) for _ in range(3)]
    reg.rg_forward(res.v, mw)
    before = math.sqrt(sum(float(np.sum((a - b) ** 2)) for a, b in zip(atlas, healthy)))
    after = math.sqrt(sum(float(np.sum((a - b) ** 2)) for a, b in zip(mw, healthy)))
    assert after < 0.8 * before, (before, after)
