"""Pins of the oracle's combined (simultaneous) update, Eq. 50 / Eq. 220:
psi <- psi . prod_v c_v, or with the |V|-th root (the geometric mean of the
view factors, as in the convergence proof)."""
import numpy as np
import pytest

import oracle
import synth


def _case(n_views=3, seed=11, dims=(12, 10, 8), noise_free=False, background=0.5):
    w = synth.small_case(seed, dims=dims, n_views=n_views, n_iter=3, asymmetric=True)
    if noise_free:
        truth = w.truth.astype(np.float64) + background
        psfs = [p.astype(np.float64) / p.astype(np.float64).sum() for p in w.psfs]
        views = [oracle.conv(truth, p) for p in psfs]
        return views, psfs, truth
    return w.views, w.psfs, w.truth.astype(np.float64)


@pytest.mark.parametrize("variant", ["plain", "efficient"])
@pytest.mark.parametrize("root", [True, False])
def test_one_view_is_richardson_lucy(variant, root):
    views, psfs, _ = _case(n_views=1)
    a, _ = oracle.deconvolve_combined(views, psfs, 4, variant, root=root)
    b, _ = oracle.deconvolve(views, psfs, 4, "plain")
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


@pytest.mark.parametrize("variant", ["plain", "efficient", "opt1", "opt2"])
@pytest.mark.parametrize("root", [True, False])
def test_noise_free_truth_is_a_fixed_point(variant, root):
    views, psfs, truth = _case(noise_free=True)
    a, _ = oracle.deconvolve_combined(views, psfs, 3, variant, root=root, psi_init=truth)
    assert np.abs(a - truth).max() <= 1e-10 * truth.max()


def test_identical_views_reduce_to_one_view():
    """N copies of one view and PSF: the product is the single factor to the N-th power, and its
    N-th root is the single-view update (pins the product over views and the exponent 1/N)."""
    views, psfs, _ = _case(n_views=1)
    a, _ = oracle.deconvolve_combined(views * 3, psfs * 3, 3, "plain", root=True)
    b, _ = oracle.deconvolve(views, psfs, 3, "plain")
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


def test_root_is_the_geometric_mean_of_the_factors():
    """One step from the same start: psi_root = psi0 (psi_noroot / psi0)^(1/N) where no floor acts."""
    views, psfs, truth = _case(noise_free=True)
    start = np.full_like(truth, truth.mean())
    a, eps = oracle.deconvolve_combined(views, psfs, 1, "efficient", root=True, psi_init=start)
    b, _ = oracle.deconvolve_combined(views, psfs, 1, "efficient", root=False, psi_init=start, eps=eps)
    want = start * (b / start) ** (1.0 / len(views))
    assert np.abs(a - want).max() <= 1e-12 * np.abs(want).max()


def test_likelihood_increases_with_the_root():
    """Convergence proof (Section "Proof of convergence"): for noise-free data the likelihood
    L(psi^r; psi*) = -sum psi* log(psi* / psi^r) does not decrease under the combined update with the
    |V|-th root and plain kernels."""
    views, psfs, truth = _case(n_views=3, noise_free=True)
    psi = np.full_like(truth, np.mean([v.mean() for v in views]))
    lik = []
    for _ in range(12):
        lik.append(-np.sum(truth * np.log(truth / psi)))
        psi, _ = oracle.deconvolve_combined(views, psfs, 1, "plain", root=True, psi_init=psi, eps=1e-12)
    lik.append(-np.sum(truth * np.log(truth / psi)))
    d = np.diff(lik)
    assert (d >= -1e-9 * np.abs(lik[0])).all(), d
    assert lik[-1] > lik[0]
