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


# ---------------------------------------------------------------------------
# mirror boundary (half-sample symmetric reflection at every face)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("shape,kshape", [((7, 6, 9), (3, 5, 3)), ((5, 8, 4), (5, 3, 7)), ((4, 4, 4), (7, 7, 7))])
def test_mirror_convolution_matches_scipy(shape, kshape):
    """scipy's 'reflect' mode is the half-sample symmetric continuation (d c b a | a b c d | d c b a)."""
    rng = np.random.default_rng(2)
    vol = rng.normal(size=shape)
    k = rng.normal(size=kshape)
    want = ndimage.convolve(vol, k, mode="reflect")
    got = oracle.conv_mirror(vol, k)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("shape,kshape", [((7, 6, 9), (3, 5, 3)), ((4, 4, 4), (7, 7, 7))])
def test_mirror_backprojection_is_the_transpose_of_the_mirrored_blur(shape, kshape):
    """<conv_mirror(x, k(-e)), y> = <x, backproject_mirror(y, k)> for any x, y and an asymmetric k."""
    rng = np.random.default_rng(3)
    x, y = rng.normal(size=shape), rng.normal(size=shape)
    k = rng.uniform(0.0, 1.0, size=kshape)
    lhs = float((oracle.conv_mirror(x, oracle.mirror(k)) * y).sum())
    rhs = float((x * oracle.backproject_mirror(y, k)).sum())
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


def test_mirror_backprojection_away_from_the_faces_is_the_convolution():
    rng = np.random.default_rng(4)
    k = rng.uniform(0.0, 1.0, size=(3, 5, 3))
    r = np.zeros((12, 14, 10))
    r[3:9, 4:10, 2:8] = rng.uniform(size=(6, 6, 6))
    assert np.abs(oracle.backproject_mirror(r, k) - oracle.conv(r, k)).max() <= 1e-12


def _separable_symmetric(kshape):
    ax = [np.exp(-0.5 * ((np.arange(n) - (n - 1) / 2) / 1.3) ** 2) for n in kshape]
    k = ax[0][:, None, None] * ax[1][None, :, None] * ax[2][None, None, :]
    return k / k.sum()


def test_mirror_sensitivity():
    """A kernel symmetric under each face's reflection sends back across the face exactly what
    crosses it: the sensitivity is 1 everywhere. An asymmetric kernel's is not."""
    ones = np.ones((9, 8, 7))
    s = oracle.backproject_mirror(ones, _separable_symmetric((5, 3, 7)))
    assert np.abs(s - 1.0).max() <= 1e-13
    k = np.random.default_rng(5).uniform(0.0, 1.0, size=(5, 3, 7))
    s = oracle.backproject_mirror(ones, k / k.sum())
    assert np.abs(s - 1.0).max() > 1e-3


def _mirror_noise_free(seed=32, dims=(14, 12, 10), background=2.0):
    w = synth.small_case(seed, dims=dims, n_views=3, n_iter=3, asymmetric=True)
    truth = w.truth.astype(np.float64) + background
    psfs = [p.astype(np.float64) / p.astype(np.float64).sum() for p in w.psfs]
    return [oracle.conv_mirror(truth, p) for p in psfs], psfs, truth


def test_mirror_plain_update_conserves_the_sensitivity_weighted_intensity():
    """ML-EM identity for the mirror model: sum(s psi') = sum(phi) with s the back-projection of ones."""
    views, psfs, _ = _mirror_noise_free()
    psi = None
    for v in (0, 1, 2, 0):
        s = oracle.backproject_mirror(np.ones_like(views[v]), oracle.mirror(psfs[v]))
        psi, _ = oracle.deconvolve_mirror([views[v]], [psfs[v]], 1, "plain", psi_init=psi, eps=1e-12)
        assert abs((s * psi).sum() - views[v].sum()) <= 1e-10 * views[v].sum()


@pytest.mark.parametrize("variant", ["plain", "efficient"])
def test_mirror_noise_free_truth_is_a_fixed_point(variant):
    views, psfs, truth = _mirror_noise_free()
    psi, _ = oracle.deconvolve_mirror(views, psfs, 3, variant, psi_init=truth)
    assert np.abs(psi - truth).max() <= 1e-10 * truth.max()


def test_mirror_symmetric_single_view_is_richardson_lucy_with_reflected_convolutions():
    """One view, a kernel symmetric per axis, plain variant: s = 1 and the back-projection with
    P^* = P is the mirror convolution itself (P symmetric), so one step is
    psi * conv_mirror(phi / conv_mirror(psi, P), P)."""
    rng = np.random.default_rng(6)
    P = _separable_symmetric((5, 3, 7))
    phi = rng.uniform(1.0, 3.0, size=(9, 8, 7))
    psi0 = rng.uniform(1.0, 2.0, size=phi.shape)
    want = psi0 * oracle.conv_mirror(phi / oracle.conv_mirror(psi0, P), P)
    got, _ = oracle.deconvolve_mirror([phi], [P], 1, "plain", psi_init=psi0, eps=1e-12)
    assert np.abs(got - want).max() <= 1e-12 * want.max()


def test_the_three_boundaries_differ():
    views, psfs, _ = _mirror_noise_free()
    a, _ = oracle.deconvolve_mirror(views, psfs, 2, "efficient")
    b, _ = oracle.deconvolve_zero(views, psfs, 2, "efficient")
    c, _ = oracle.deconvolve(views, psfs, 2, "efficient")
    assert np.abs(a - b).max() > 1e-3 * np.abs(b).max()
    assert np.abs(a - c).max() > 1e-3 * np.abs(c).max()


# ---------------------------------------------------------------------------
# view weights and Tikhonov regularisation with the zero and mirror boundaries
# ---------------------------------------------------------------------------

BOUNDED = {"zero": (oracle.deconvolve_zero, oracle.conv_zero), "mirror": (oracle.deconvolve_mirror, oracle.conv_mirror)}


def _weights(shape, n, seed):
    rng = np.random.default_rng(seed)
    return [rng.uniform(0.2, 1.0, size=shape) for _ in range(n)]


@pytest.mark.parametrize("boundary", ["zero", "mirror"])
def test_unit_weights_and_no_regularisation_reduce_to_the_plain_update(boundary):
    deconv, blur = BOUNDED[boundary]
    views, psfs, _ = _noise_free() if boundary == "zero" else _mirror_noise_free()
    a, _ = deconv(views, psfs, 2, "efficient")
    b, _ = deconv(views, psfs, 2, "efficient", weights=[np.ones_like(v) for v in views], lam=0.0)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


@pytest.mark.parametrize("boundary", ["zero", "mirror"])
def test_a_zero_weight_view_drops_out(boundary):
    """Plain kernels (P_v^comp = P_v^*, no dependence on the other views): weight 0 for view 1
    equals running views 0 and 2 alone from the same start and floor."""
    deconv, _ = BOUNDED[boundary]
    views, psfs, truth = _noise_free() if boundary == "zero" else _mirror_noise_free()
    start = np.full_like(truth, truth.mean())
    w = [np.ones_like(v) for v in views]
    w[1] = np.zeros_like(views[1])
    a, _ = deconv(views, psfs, 2, "plain", eps=1e-9, psi_init=start, weights=w)
    b, _ = deconv([views[0], views[2]], [psfs[0], psfs[2]], 2, "plain", eps=1e-9, psi_init=start)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


@pytest.mark.parametrize("boundary", ["zero", "mirror"])
def test_weighted_noise_free_truth_is_a_fixed_point(boundary):
    deconv, _ = BOUNDED[boundary]
    views, psfs, truth = _noise_free() if boundary == "zero" else _mirror_noise_free()
    psi, _ = deconv(views, psfs, 2, "efficient", psi_init=truth, weights=_weights(truth.shape, 3, 7))
    assert np.abs(psi - truth).max() <= 1e-10 * truth.max()


@pytest.mark.parametrize("boundary", ["zero", "mirror"])
def test_one_weighted_regularised_update_matches_the_periodic_one_away_from_the_faces(boundary):
    """From a flat start the first update at voxels farther than twice the kernel reach from
    every face sees no boundary: it equals the periodic weighted, regularised update there."""
    deconv, _ = BOUNDED[boundary]
    rng = np.random.default_rng(8)
    shape = (20, 22, 24)
    views = [rng.uniform(1.0, 3.0, size=shape)]
    psfs = [_separable_symmetric((5, 3, 7))]
    w = _weights(shape, 1, 9)
    start = np.full(shape, 2.0)
    a, _ = deconv(views, psfs, 1, "efficient", eps=1e-9, psi_init=start, weights=w, lam=0.05)
    b, _ = oracle.deconvolve_weighted(views, psfs, 1, w, "efficient", eps=1e-9, psi_init=start, lam=0.05)
    hz, hy, hx = 2 * 2, 2 * 1, 2 * 3  # twice the half-widths of the 5 x 3 x 7 ([z][y][x]) box
    inner = (slice(hz, shape[0] - hz), slice(hy, shape[1] - hy), slice(hx, shape[2] - hx))
    assert np.abs(a[inner] - b[inner]).max() <= 1e-12 * np.abs(b[inner]).max()
    assert np.abs(a - b).max() > 1e-6  # the faces do differ


# ---------------------------------------------------------------------------
# the combined (simultaneous) update with the zero and mirror boundaries
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("boundary", ["zero", "mirror"])
@pytest.mark.parametrize("root", [True, False])
def test_combined_with_one_view_is_the_sequential_update(boundary, root):
    deconv, _ = BOUNDED[boundary]
    views, psfs, _ = _noise_free() if boundary == "zero" else _mirror_noise_free()
    a, _ = oracle.deconvolve_combined(views[:1], psfs[:1], 3, "efficient", root=root, boundary=boundary)
    b, _ = deconv(views[:1], psfs[:1], 3, "efficient")
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


@pytest.mark.parametrize("boundary", ["zero", "mirror"])
def test_combined_noise_free_truth_is_a_fixed_point(boundary):
    views, psfs, truth = _noise_free() if boundary == "zero" else _mirror_noise_free()
    for root in (True, False):
        psi, _ = oracle.deconvolve_combined(views, psfs, 2, "efficient", root=root, psi_init=truth,
                                            boundary=boundary)
        assert np.abs(psi - truth).max() <= 1e-10 * truth.max()


@pytest.mark.parametrize("boundary", ["zero", "mirror"])
def test_combined_root_of_identical_views_is_one_view(boundary):
    """Plain kernels: N copies of one view give N identical factors, whose geometric mean is
    the single view's factor."""
    views, psfs, _ = _noise_free() if boundary == "zero" else _mirror_noise_free()
    a, _ = oracle.deconvolve_combined([views[0]] * 3, [psfs[0]] * 3, 2, "plain", root=True, boundary=boundary)
    b, _ = oracle.deconvolve_combined(views[:1], psfs[:1], 2, "plain", root=True, boundary=boundary)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


@pytest.mark.parametrize("boundary", ["zero", "mirror"])
def test_one_combined_update_matches_the_periodic_one_away_from_the_faces(boundary):
    rng = np.random.default_rng(10)
    shape = (20, 22, 24)
    views = [rng.uniform(1.0, 3.0, size=shape) for _ in range(2)]
    psfs = [_separable_symmetric((5, 3, 7)), _separable_symmetric((3, 5, 5))]
    start = np.full(shape, 2.0)
    a, _ = oracle.deconvolve_combined(views, psfs, 1, "efficient", eps=1e-9, psi_init=start, boundary=boundary)
    b, _ = oracle.deconvolve_combined(views, psfs, 1, "efficient", eps=1e-9, psi_init=start)
    # compound kernels live on each PSF's box: reach (2, 2, 3) in (z, y, x); twice that
    inner = (slice(4, shape[0] - 4), slice(4, shape[1] - 4), slice(6, shape[2] - 6))
    assert np.abs(a[inner] - b[inner]).max() <= 1e-12 * np.abs(b[inner]).max()
    assert np.abs(a - b).max() > 1e-6
