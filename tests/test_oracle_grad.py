"""Pins of the oracle's reverse-mode gradient of the unrolled iteration against
FP64 central finite differences of the oracle's own forward run (the loss is
mean((psi_K - truth)^2) after n iterations from the flat start)."""
import numpy as np
import pytest

import oracle
import synth


def _problem(seed, dims=(10, 9, 8), boxes=((3, 5, 3), (5, 3, 3), (3, 3, 5))):
    w = synth.small_case(seed, dims=dims, n_views=len(boxes), boxes=list(boxes), asymmetric=True)
    psfs = [p.astype(np.float64) for p in w.psfs]
    truth = w.truth.astype(np.float64) + 1.0
    # noise-free, strictly positive views keep every floor inactive
    views = [synth.workloads.blur_circular(truth, p / p.sum()) + 0.5 for p in psfs]
    return views, psfs, truth


def _loss(views, psfs, truth, n_iter, variant):
    psi, _ = oracle.deconvolve(views, psfs, n_iter, variant)
    return float(np.mean((psi - truth) ** 2))


@pytest.mark.parametrize("variant", ["plain", "efficient", "opt1", "opt2"])
def test_unrolled_gradient_matches_finite_differences(variant):
    views, psfs, truth = _problem(71)
    n_iter = 2
    loss, gv, gp, psik = oracle.unrolled_grad(views, psfs, n_iter, truth, variant)
    assert abs(loss - _loss(views, psfs, truth, n_iter, variant)) < 1e-12 * loss
    rng = np.random.default_rng(3)
    # view voxels
    for v in range(len(views)):
        for idx in rng.choice(views[v].size, 3, replace=False):
            h = 1e-4 * views[v].ravel()[idx]
            vp = [x.copy() for x in views]
            vm = [x.copy() for x in views]
            vp[v].ravel()[idx] += h
            vm[v].ravel()[idx] -= h
            fd = (_loss(vp, psfs, truth, n_iter, variant) - _loss(vm, psfs, truth, n_iter, variant)) / (2 * h)
            assert abs(gv[v].ravel()[idx] - fd) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(gv[v]).max()), (v, idx)
    # raw PSF taps
    for v in range(len(psfs)):
        for idx in rng.choice(psfs[v].size, 3, replace=False):
            h = 1e-4 * psfs[v].ravel()[idx]
            pp = [x.copy() for x in psfs]
            pm = [x.copy() for x in psfs]
            pp[v].ravel()[idx] += h
            pm[v].ravel()[idx] -= h
            fd = (_loss(views, pp, truth, n_iter, variant) - _loss(views, pm, truth, n_iter, variant)) / (2 * h)
            assert abs(gp[v].ravel()[idx] - fd) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(gp[v]).max()), (v, idx)


def test_directional_derivative_over_all_views():
    """<grad_phi L, u> against a central difference along a random direction u."""
    views, psfs, truth = _problem(72, dims=(12, 10, 9))
    _, gv, _, _ = oracle.unrolled_grad(views, psfs, 3, truth, "efficient")
    rng = np.random.default_rng(9)
    u = [rng.standard_normal(v.shape) for v in views]
    h = 1e-5
    lp = _loss([v + h * d for v, d in zip(views, u)], psfs, truth, 3, "efficient")
    lm = _loss([v - h * d for v, d in zip(views, u)], psfs, truth, 3, "efficient")
    fd = (lp - lm) / (2 * h)
    an = sum(float(np.sum(g * d)) for g, d in zip(gv, u))
    assert abs(an - fd) < 1e-6 * abs(fd)
