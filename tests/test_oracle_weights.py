"""Pins of the oracle's partially-overlapping-views support (Suppl. Note
"Partially overlapping datasets"): weight normalisation and the weighted
sequential update psi <- psi (1 + w_v (c_v - 1))."""
import numpy as np
import pytest

import oracle
import synth


def _case(seed=21, dims=(12, 10, 8), n_views=3, noise_free=False):
    w = synth.small_case(seed, dims=dims, n_views=n_views, n_iter=3, asymmetric=True)
    if noise_free:
        truth = w.truth.astype(np.float64) + 0.5
        psfs = [p.astype(np.float64) / p.astype(np.float64).sum() for p in w.psfs]
        return [oracle.conv(truth, p) for p in psfs], psfs, truth
    return w.views, w.psfs, w.truth


def test_normalisation_invariants():
    rng = np.random.default_rng(3)
    ws = [rng.uniform(0, 1, (8, 9, 10)) * (rng.uniform(size=(8, 9, 10)) > 0.3) for _ in range(4)]
    for norm, value in (("sum1", 0), ("min_overlap", 0), ("avg_overlap", 0), ("user", 2.5)):
        out, T = oracle.normalize_weights(ws, norm, value)
        S = sum(ws)
        So = sum(out)
        assert (So <= T * (1 + 1e-12) + 1e-15).all()
        for w, o in zip(ws, out):
            assert (o <= w + 1e-15).all() and (o >= 0).all() and (o <= 1).all()
            keep = S <= T
            assert np.array_equal(o[keep], w[keep])  # never changed where the sum is within T
        ratio = np.where(ws[0] > 0, out[0] / np.where(ws[0] > 0, ws[0], 1), np.nan)
        ratio1 = np.where(ws[1] > 0, out[1] / np.where(ws[1] > 0, ws[1], 1), np.nan)
        both = (ws[0] > 0) & (ws[1] > 0)
        assert np.allclose(ratio[both], ratio1[both], rtol=1e-12)  # one factor per voxel


def test_overlap_counts_on_a_constructed_layout():
    """Voxels covered by exactly 1, 2 or 3 views in known numbers (and some by none)."""
    shape = (1, 1, 10)
    w1, w2, w3 = (np.zeros(shape) for _ in range(3))
    w1[..., 0:6] = 1.0   # voxels 0-5
    w2[..., 3:8] = 0.5   # voxels 3-7
    w3[..., 5:9] = 0.25  # voxels 5-8 ; voxel 9 uncovered
    # counts: 0-2 -> 1, 3-4 -> 2, 5 -> 3, 6-7 -> 2, 8 -> 1, 9 -> 0
    _, tmin = oracle.normalize_weights([w1, w2, w3], "min_overlap")
    _, tavg = oracle.normalize_weights([w1, w2, w3], "avg_overlap")
    assert tmin == 1.0
    assert tavg == pytest.approx((1 + 1 + 1 + 2 + 2 + 3 + 2 + 2 + 1) / 9.0, rel=1e-15)
    out, _ = oracle.normalize_weights([w1, w2, w3], "sum1")
    assert out[0][0, 0, 5] == pytest.approx(1.0 / 1.75) and out[2][0, 0, 5] == pytest.approx(0.25 / 1.75)
    assert out[0][0, 0, 0] == 1.0 and out[1][0, 0, 7] == 0.5


@pytest.mark.parametrize("variant", ["plain", "efficient"])
def test_unit_weights_are_the_unweighted_method(variant):
    views, psfs, _ = _case()
    ones = [np.ones_like(np.asarray(v, np.float64)) for v in views]
    a, _ = oracle.deconvolve_weighted(views, psfs, 3, ones, variant)
    b, _ = oracle.deconvolve(views, psfs, 3, variant)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


def test_a_view_with_zero_weight_drops_out():
    views, psfs, _ = _case()
    ws = [np.ones_like(np.asarray(v, np.float64)) for v in views]
    ws[1][:] = 0.0
    a, eps = oracle.deconvolve_weighted(views, psfs, 3, ws, "efficient")
    b, _ = oracle.deconvolve(views, psfs, 3, "efficient", schedule=[0, 2], eps=eps)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


def test_fractional_weight_applies_that_fraction_of_the_change():
    """One update with weight w is the w-interpolation between psi and the full RL update."""
    views, psfs, truth = _case(noise_free=True)
    start = np.full_like(truth, truth.mean())
    rng = np.random.default_rng(5)
    wv = rng.uniform(0, 1, truth.shape)
    zero = np.zeros_like(truth)
    full, eps = oracle.deconvolve(views, psfs, 1, "efficient", schedule=[0], psi_init=start)
    part, _ = oracle.deconvolve_weighted(views, psfs, 1, [wv, zero, zero], "efficient", eps=eps, psi_init=start)
    want = start + wv * (full - start)
    assert np.abs(part - want).max() <= 1e-12 * np.abs(want).max()


def test_noise_free_truth_is_a_fixed_point_for_any_weights():
    views, psfs, truth = _case(noise_free=True)
    rng = np.random.default_rng(6)
    ws, _ = oracle.normalize_weights([rng.uniform(0, 1, truth.shape) for _ in views], "min_overlap")
    a, _ = oracle.deconvolve_weighted(views, psfs, 3, ws, "efficient", psi_init=truth)
    assert np.abs(a - truth).max() <= 1e-10 * truth.max()


# ---------------------------------------------------------------------------
# Tikhonov regularisation (Green's one-step-late form, factor c / (1 + lambda psi))
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("variant", ["plain", "efficient"])
def test_zero_lambda_is_the_unregularised_method(variant):
    views, psfs, _ = _case()
    a, _ = oracle.deconvolve_weighted(views, psfs, 3, None, variant, lam=0.0)
    b, _ = oracle.deconvolve(views, psfs, 3, variant)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


@pytest.mark.parametrize("lam", [0.0006, 0.006, 0.06])
def test_constant_data_converge_to_the_closed_form(lam):
    """Spatially constant views phi with normalised PSFs: every blur of a constant is the constant,
    so the update is psi <- phi / (1 + lam psi), whose fixed point solves lam psi^2 + psi - phi = 0."""
    phi = 40.0
    views = [np.full((6, 5, 4), phi) for _ in range(2)]
    psfs = [np.ones((3, 3, 3)), np.ones((1, 3, 5))]
    psi, _ = oracle.deconvolve_weighted(views, psfs, 200, None, "efficient", lam=lam)
    want = (-1.0 + np.sqrt(1.0 + 4.0 * lam * phi)) / (2.0 * lam)
    assert np.abs(psi - want).max() <= 1e-10 * want


def test_regularisation_with_weights_applies_the_fraction_of_the_regularised_change():
    views, psfs, truth = _case(noise_free=True)
    start = np.full_like(truth, truth.mean())
    rng = np.random.default_rng(8)
    wv = rng.uniform(0, 1, truth.shape)
    zero = np.zeros_like(truth)
    one = np.ones_like(truth)
    lam = 0.006
    full, eps = oracle.deconvolve_weighted(views, psfs, 1, [one, zero, zero], "efficient", psi_init=start, lam=lam)
    part, _ = oracle.deconvolve_weighted(views, psfs, 1, [wv, zero, zero], "efficient", eps=eps, psi_init=start,
                                         lam=lam)
    want = start + wv * (full - start)
    assert np.abs(part - want).max() <= 1e-12 * np.abs(want).max()
