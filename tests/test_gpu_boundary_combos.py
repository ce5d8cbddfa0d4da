"""Zero and mirror boundaries combined with the other update forms on the GPU:
view weights (Suppl. Note "Partially overlapping datasets"), Tikhonov
regularisation (Green's one-step-late form) and the combined update of Eq. 50 /
Eq. 220 (factors c_v / s_v, with and without the |V|-th root), each against the
FP64 oracle's bounded form (`deconvolve_zero` / `deconvolve_mirror` with weights
and lambda, `deconvolve_combined(boundary=...)`), on both engines."""
import numpy as np
import pytest

import oracle
import synth
from synth.workloads import blend_weights
from tests._util import PARITY_TOL, err_report, rel_err

pytestmark = pytest.mark.gpu

BOUNDARIES = ["zero", "mirror"]
BLUR = {"zero": oracle.conv_zero, "mirror": oracle.conv_mirror}
DECONVOLVE = {"zero": oracle.deconvolve_zero, "mirror": oracle.deconvolve_mirror}


@pytest.fixture(scope="module")
def mvd():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1308_0730_gb300 import mvd as m

    m.load()
    return m


def _case(boundary, seed=81, dims=(30, 24, 20)):
    """Asymmetric PSFs (a missing mirror would show), mixed-radix padded grids; views blurred
    with the boundary's own model, Poisson noise, + 0.5."""
    w = synth.small_case(seed, dims=dims, n_views=3, boxes=[(7, 5, 9), (9, 7, 5), (5, 9, 7)], n_iter=4,
                         asymmetric=True)
    rng = np.random.default_rng(seed)
    truth = w.truth.astype(np.float64)
    views = []
    for p in w.psfs:
        p = p.astype(np.float64)
        b = BLUR[boundary](truth, p / p.sum())
        views.append(rng.poisson(np.maximum(b, 0.0)).astype(np.float32) + np.float32(0.5))
    return w, views


def _layout(dims):
    X, Y, Z = dims
    boxes = [((0, 0, 0), (int(0.7 * X), Y, Z)), ((int(0.3 * X), 0, 0), (X, Y, Z)),
             ((0, 0, int(0.2 * Z)), (X, int(0.8 * Y), Z))]
    return [blend_weights(dims, lo, hi, (4, 4, 4)) for lo, hi in boxes]


@pytest.mark.parametrize("boundary", BOUNDARIES)
@pytest.mark.parametrize("path", ["direct", "fft"])
@pytest.mark.parametrize("form", ["weights", "lambda", "weights+lambda"])
def test_sequential_forms_with_boundary_match_oracle(mvd, boundary, path, form):
    w, views = _case(boundary)
    raw = _layout(w.dims) if "weights" in form else None
    lam = 0.01 if "lambda" in form else 0.0
    ws = oracle.normalize_weights(raw, "min_overlap")[0] if raw is not None else None
    want, eps = DECONVOLVE[boundary](views, w.psfs, w.n_iter, "efficient", weights=ws, lam=lam)
    with mvd.Deconvolver(views, w.psfs, "efficient", path=path, boundary=boundary) as d:
        if raw is not None:
            d.set_weights(raw, "min_overlap")
            for v in range(w.n_views):  # the weights come back in the user's layout
                assert np.abs(d.weights(v) - ws[v]).max() <= 1e-6
        d.set_regularization(lam)
        d.iterate(w.n_iter)
        got = d.result().astype(np.float64)
        assert abs(d.eps - eps) <= 1e-6 * eps
    assert rel_err(got, want) < PARITY_TOL, err_report(got, want)


@pytest.mark.parametrize("boundary", BOUNDARIES)
@pytest.mark.parametrize("path", ["direct", "fft"])
@pytest.mark.parametrize("root,n_iter", [(True, 4), (False, 2)])
def test_combined_update_with_boundary_matches_oracle(mvd, boundary, path, root, n_iter):
    w, views = _case(boundary, seed=82)
    want, _ = oracle.deconvolve_combined(views, w.psfs, n_iter, "efficient", root=root, boundary=boundary)
    with mvd.Deconvolver(views, w.psfs, "efficient", path=path, boundary=boundary) as d:
        d.iterate_combined(n_iter, root)
        got = d.result().astype(np.float64)
    assert rel_err(got, want) < PARITY_TOL, err_report(got, want)


@pytest.mark.parametrize("boundary", BOUNDARIES)
@pytest.mark.parametrize("precision", ["fast", "mixed"])
def test_boundary_forms_in_the_fp32_pipelines(mvd, boundary, precision):
    """Weights with lambda, and the combined update, through the FP32 back-projection: a few
    iterations stay within the bar."""
    w, views = _case(boundary, seed=83)
    raw = _layout(w.dims)
    ws = oracle.normalize_weights(raw, "sum1")[0]
    want, _ = DECONVOLVE[boundary](views, w.psfs, 2, "efficient", weights=ws, lam=0.01)
    want_c, _ = oracle.deconvolve_combined(views, w.psfs, 2, "efficient", root=True, boundary=boundary)
    with mvd.Deconvolver(views, w.psfs, "efficient", path="fft", boundary=boundary, precision=precision) as d:
        d.set_weights(raw, "sum1")
        d.set_regularization(0.01)
        d.iterate(2)
        got = d.result().astype(np.float64)
        d.set_weights(None)
        d.set_regularization(0.0)
        d.set_estimate(None)
        d.iterate_combined(2, True)
        got_c = d.result().astype(np.float64)
    assert rel_err(got, want) < PARITY_TOL, err_report(got, want)
    assert rel_err(got_c, want_c) < PARITY_TOL, err_report(got_c, want_c)


@pytest.mark.parametrize("boundary", BOUNDARIES)
def test_combined_rejects_weights_and_lambda(mvd, boundary):
    w, views = _case(boundary, seed=84, dims=(16, 12, 10))
    with mvd.Deconvolver(views, w.psfs, path="fft", boundary=boundary) as d:
        d.set_regularization(0.01)
        with pytest.raises(mvd.MvdError) as e:
            d.iterate_combined(1)
        assert e.value.status == mvd.MVD_ERR_UNSUPPORTED
        d.set_regularization(0.0)
        d.set_weights(_layout(w.dims)[:w.n_views])
        with pytest.raises(mvd.MvdError) as e:
            d.iterate_combined(1)
        assert e.value.status == mvd.MVD_ERR_UNSUPPORTED
