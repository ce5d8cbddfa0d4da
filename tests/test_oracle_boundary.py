"""Pins of the oracle's zero-boundary convolution and deconvolution (the volume
continued by zeros instead of periodically)."""
import numpy as np
import pytest
from scipy import ndimage

import oracle
import synth


@pytest.mark.parametrize("shape,kshape", [((7, 6, 9), (3, 5, 3)), ((5, 8, 4), (5, 3, 7)), ((4, 4, 4), (7, 7, 7))])
def test_zero_boundary_convolution_matches_scipy(shape, kshape):
    rng = np.random.default_rng(1)
    vol = rng.normal(size=shape)
    k = rng.normal(size=kshape)
    want = ndimage.convolve(vol, k, mode="constant", cval=0.0)
    got = oracle.conv_zero(vol, k)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


def _noise_free(seed=31, dims=(14, 12, 10), background=2.0):
    w = synth.small_case(seed, dims=dims, n_views=3, n_iter=3, asymmetric=True)
    truth = w.truth.astype(np.float64) + background
    psfs = [p.astype(np.float64) / p.astype(np.float64).sum() for p in w.psfs]
    return [oracle.conv_zero(truth, p) for p in psfs], psfs, truth


def test_plain_update_conserves_the_sensitivity_weighted_intensity():
    """ML-EM identity: with s = 1 * P^* (zero boundary) the plain update gives
    sum(s psi') = sum(psi (r * P^*)) = sum(r (psi * P)) = sum(phi): the zero-boundary back-projection
    is the transpose of the zero-boundary blur (no floor active)."""
    views, psfs, _ = _noise_free()
    psi = None
    for v in (0, 1, 2, 0):
        s = oracle.conv_zero(np.ones_like(views[v]), oracle.mirror(psfs[v]))
        psi, _ = oracle.deconvolve_zero([views[v]], [psfs[v]], 1, "plain", psi_init=psi, eps=1e-12)
        assert abs((s * psi).sum() - views[v].sum()) <= 1e-10 * views[v].sum()


def test_interior_sensitivity_is_one():
    """Away from the faces (farther than the kernel half-width) the sensitivity is the kernel's sum, 1."""
    _, psfs, truth = _noise_free()
    k = oracle.compound(psfs, 0, "efficient")
    s = oracle.conv_zero(np.ones_like(truth), k)
    hz, hy, hx = [(n - 1) // 2 for n in k.shape]
    inner = s[hz:s.shape[0] - hz, hy:s.shape[1] - hy, hx:s.shape[2] - hx]
    assert inner.size > 0 and np.abs(inner - 1.0).max() <= 1e-12
    assert s.min() < 0.9


@pytest.mark.parametrize("variant", ["plain", "efficient"])
def test_noise_free_truth_is_a_fixed_point(variant):
    views, psfs, truth = _noise_free()
    psi, _ = oracle.deconvolve_zero(views, psfs, 3, variant, psi_init=truth)
    assert np.abs(psi - truth).max() <= 1e-10 * truth.max()


def test_the_boundary_matters():
    """With a bright object touching the faces, periodic and zero boundaries differ."""
    views, psfs, _ = _noise_free()
    a, _ = oracle.deconvolve_zero(views, psfs, 2, "efficient")
    b, _ = oracle.deconvolve(views, psfs, 2, "efficient")
    assert np.abs(a - b).max() > 1e-3 * np.abs(b).max()
