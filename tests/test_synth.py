"""Input recipes: determinism, mask volume, flip count (CPU only)."""

import math

import numpy as np

from paper_1907_07774_gb300 import synth


def test_tissue_maps_are_seeded_partition_of_unity_inside_mask():
    a = synth.tissue_maps((16, 16, 16), 3)
    b = synth.tissue_maps((16, 16, 16), 3)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    mask = synth.ellipsoid_mask((16, 16, 16))
    tot = a[0] + a[1] + a[2]
    assert np.allclose(tot[mask > 0], 1.0) and np.all(tot[mask == 0] == 0)


def test_mask_volume_close_to_ellipsoid_fraction():
    mask = synth.ellipsoid_mask((64, 64, 64))
    want = 4.0 / 3.0 * math.pi * 0.8 * 0.9 * 0.7 * math.pi ** 3 / (2 * math.pi) ** 3
    assert abs(mask.mean() - want) < 0.01


def test_labels_flip_exact_count_inside_mask():
    n = (16, 16, 16)
    mask = synth.ellipsoid_mask(n)
    c = np.zeros(n)
    d = synth.labels(c, mask, 1, flip_fraction=0.05)
    assert d.sum() == round(0.05 * mask.sum())
    assert np.all(d[mask == 0] == 0)


def test_labels_do_not_depend_on_the_memory_order_of_the_input():
    # the flips index the row-major flattening; a field with permuted strides
    # (as a GPU FFT can return) must give the same labels, flips included
    n = (16, 12, 8)
    mask = synth.ellipsoid_mask(n)
    rng = np.random.default_rng(2)
    c = rng.random(n)
    ref = synth.labels(c, mask, 5, flip_fraction=0.05)
    for view in (np.asfortranarray(c), np.ascontiguousarray(c.transpose(2, 0, 1)).transpose(1, 2, 0)):
        assert not view.flags["C_CONTIGUOUS"]
        d = synth.labels(view, mask, 5, flip_fraction=0.05)
        assert np.array_equal(d, ref)
    assert np.sum(ref != (c >= 0.5)) == round(0.05 * mask.sum())


def test_lattice_centred_and_spaced():
    c = synth.lattice_centers(3, 0.5)
    assert c.shape == (27, 3)
    assert np.allclose(c.mean(axis=0), math.pi)
    assert np.allclose(np.unique(c[:, 2]) - math.pi, [-0.5, 0.0, 0.5])


def test_trig_sum_on_the_grid_matches_direct_evaluation_and_curls_are_divergence_free():
    import numpy as np
    from paper_1907_07774_gb300 import synth
    rng = np.random.default_rng(0)
    n = (8, 16, 12)
    X = synth.coords_mesh(n)
    T = synth.TrigSum.random(rng, 3)
    assert np.abs(T.grid(n) - T(X)).max() < 1e-12
    for a in range(3):
        assert np.abs(T.grid_deriv(n, a) - T.deriv(X, a)).max() < 1e-12
    pots = [synth.TrigSum.random(rng, 3) for _ in range(3)]
    v = synth.curl_field_grid(pots, n)
    w = synth.curl_field(pots, X)
    assert max(np.abs(a - b).max() for a, b in zip(v, w)) < 1e-12
    # divergence of the curl through exact derivatives of its modes
    k = [np.fft.fftfreq(m, 1.0 / m) for m in n]
    V = [np.fft.fftn(x) for x in v]
    D = sum(1j * k[a].reshape([-1 if b == a else 1 for b in range(3)]) * V[a] for a in range(3))
    assert np.abs(np.fft.ifftn(D)).max() < 1e-10
