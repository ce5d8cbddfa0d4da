"""Pins of the oracle's FFT leg (`oracle.deconvolve_fft`, `oracle.conv_fft`).

The FFT leg evaluates every periodic convolution of the sequential update
through FP64 FFTs (the Convolution Theorem). It exists so that whole-volume
parity tests at full size finish in seconds. Each test here compares it with
something other than itself: the direct-sum oracle (itself pinned in
test_oracle_pins.py), the stored direct-oracle values of the 20-iteration
256x256x128 run, or an invariant of the method (noise-free fixed point,
conservation with plain kernels).
"""
import numpy as np
import pytest

import oracle
import synth
from tests._util import rel_err


def test_conv_fft_matches_direct_sums_with_wrap():
    """A kernel box as large as the grid (taps wrap around) on a non-cubic grid."""
    rng = np.random.default_rng(11)
    f = rng.uniform(0.0, 5.0, size=(7, 10, 9))
    k = rng.uniform(0.0, 1.0, size=(7, 9, 9))
    k[0, 0, 0] += 2.0
    got = oracle.conv_fft(f, k)
    want = oracle.conv(f, k)
    assert np.max(np.abs(got - want)) < 1e-12 * np.abs(want).max()


def test_blobs32_fft_leg_equals_direct_oracle():
    """The 32^3 blob workload, 10 iterations (efficient): FFT leg = direct oracle."""
    w = synth.config1()
    want, eps = oracle.deconvolve(w.views, w.psfs, w.n_iter)
    got, eps2 = oracle.deconvolve_fft(w.views, w.psfs, w.n_iter)
    assert abs(eps2 - eps) <= 1e-14 * eps
    assert rel_err(got, want) < 1e-10


@pytest.mark.parametrize("variant", ["plain", "efficient", "opt1", "opt2"])
def test_fft_leg_every_variant_and_schedule(variant):
    """Asymmetric PSFs (a flipped kernel would show), odd non-cubic grid, a custom schedule
    with a repeat."""
    w = synth.small_case(71, dims=(15, 12, 10), n_views=3, boxes=[(5, 3, 7), (3, 5, 5), (7, 3, 3)], n_iter=2,
                         asymmetric=True)
    sched = [2, 0, 0, 1]
    want, _ = oracle.deconvolve(w.views, w.psfs, 2, variant, schedule=sched)
    got, _ = oracle.deconvolve_fft(w.views, w.psfs, 2, variant, schedule=sched)
    assert rel_err(got, want) < 1e-10


def test_fft_leg_with_seven_rotated_large_boxes():
    """The 1024x1024x512 specimen's seven rotated PSFs (boxes up to 53x19x53) on a small grid,
    one iteration: FFT leg = direct oracle. Plain kernels: the compound kernels come from the
    same C function on both sides (pinned elsewhere), and those of these boxes take a minute."""
    w = synth.config3(dims=(64, 24, 64), n_objects=12)
    want, _ = oracle.deconvolve(w.views, w.psfs, 1, "plain")
    got, _ = oracle.deconvolve_fft(w.views, w.psfs, 1, "plain")
    assert rel_err(got, want) < 1e-10


def test_fft_leg_noise_free_fixed_point():
    """Noise-free views (truth blurred with each PSF) leave the truth unchanged (Eq. 15's fixed point)."""
    w = synth.small_case(72, dims=(16, 14, 12), n_views=3, asymmetric=True)
    truth = w.truth.astype(np.float64) + 1.0
    pn = [p.astype(np.float64) / p.astype(np.float64).sum() for p in w.psfs]
    views = [oracle.conv(truth, p) for p in pn]
    got, _ = oracle.deconvolve_fft(views, pn, 3, "efficient", psi_init=truth)
    assert np.max(np.abs(got - truth) / truth) < 1e-12


def test_fft_leg_plain_update_conserves_intensity():
    """Plain kernels: after a view update sum(psi) = sum(phi_v) (Suppl. Note, conservation)."""
    w = synth.small_case(73, dims=(20, 16, 12), n_views=2, asymmetric=True)
    got, _ = oracle.deconvolve_fft(w.views, w.psfs, 1, "plain", schedule=[1])
    tot = float(w.views[1].astype(np.float64).sum())
    assert abs(got.sum() - tot) < 1e-12 * tot


def test_fft_leg_matches_stored_direct_oracle_at_full_size():
    """The 256x256x128 four-view workload after 20 iterations: the FFT leg against the direct
    oracle's stored values at 4096 seeded voxels (tests/golden/oracle_samples_mid.txt, 581 s of
    direct sums)."""
    from tests.golden.make_oracle_samples import input_digest, read

    digest, eps, max_abs, idx, want = read("mid")
    w = synth.config2()
    assert input_digest(w) == digest
    got, eps2 = oracle.deconvolve_fft(w.views, w.psfs, w.n_iter)
    assert abs(eps2 - eps) <= 1e-15 * eps
    tau = 1e-3 * max_abs
    g = got.ravel()[idx]
    assert float(np.max(np.abs(g - want) / np.maximum(np.abs(want), tau))) < 1e-10
    assert abs(float(np.abs(got).max()) - max_abs) < 1e-10 * max_abs
