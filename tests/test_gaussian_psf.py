"""The library's Gaussian PSF model and its parameter gradient (host code, no
GPU): the model equals the point-sampled anisotropic Gaussian of the seeded
workloads, and the vector-Jacobian product equals FP64 central differences of
that independent numpy model."""
import numpy as np
import pytest

import __graft_entry__
from paper_1308_0730_gb300 import mvd
from synth.workloads import gaussian_psf, rotated_box


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    return mvd.load()


CASES = [((1.2, 4.0), (7, 7, 13), 0.0, "z"), ((1.2, 4.0), (7, 7, 13), 90.0, "z"),
         ((0.96, 4.8), (7, 7, 13), 270.0, "z"), ((1.5, 5.0), (9, 9, 15), 51.4, "z"),
         ((1.0, 2.5), (13, 7, 7), 0.0, "x"), ((1.0, 2.5), (7, 13, 7), 0.0, "y")]


@pytest.mark.parametrize("sig,box,angle,axis", CASES)
def test_model_matches_sampled_gaussian(lib, sig, box, angle, axis):
    rbox = rotated_box(box, angle)
    want = gaussian_psf(sig[0], sig[1], box, axis, angle)
    got = mvd.mvd_gaussian_psf(sig[0], sig[1], rbox, angle, axis)
    assert got.shape == want.shape
    assert np.abs(got - want).max() <= 2e-7 * want.max()


@pytest.mark.parametrize("sig,box,angle,axis", CASES)
def test_vjp_matches_central_differences(lib, sig, box, angle, axis):
    rbox = rotated_box(box, angle)
    rng = np.random.default_rng(7)
    g = rng.standard_normal(gaussian_psf(sig[0], sig[1], box, axis, angle).shape).astype(np.float32)
    got = mvd.mvd_gaussian_psf_vjp(sig[0], sig[1], rbox, g, angle, axis)
    h = 1e-6
    fd = []
    for k in range(2):
        sp, sm = list(sig), list(sig)
        sp[k] += h
        sm[k] -= h
        dP = (gaussian_psf(sp[0], sp[1], box, axis, angle) - gaussian_psf(sm[0], sm[1], box, axis, angle)) / (2 * h)
        fd.append(float(np.sum(g.astype(np.float64) * dP)))
    fd = np.array(fd)
    assert np.abs(got - fd).max() <= 1e-6 * max(1.0, np.abs(fd).max()), (got, fd)


def test_rejects_bad_arguments(lib):
    with pytest.raises(mvd.MvdError):
        mvd.mvd_gaussian_psf(0.0, 1.0, (3, 3, 3))
    with pytest.raises(mvd.MvdError):
        mvd.mvd_gaussian_psf(1.0, 1.0, (4, 3, 3))
    with pytest.raises(mvd.MvdError):
        mvd.mvd_gaussian_psf_vjp(1.0, -1.0, (3, 3, 3), np.zeros((3, 3, 3), np.float32))
