"""Partially overlapping views on the GPU: weight normalisation and the weighted
sequential update, against the FP64 oracle."""
import numpy as np
import pytest

import oracle
import synth
from synth.workloads import blend_weights
from tests._util import PARITY_TOL, err_report, rel_err

pytestmark = pytest.mark.gpu


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


def _layout(w):
    """Three views covering overlapping slabs of the volume (x, y, z boxes) with cosine edges."""
    X, Y, Z = w.dims
    boxes = [((0, 0, 0), (int(0.7 * X), Y, Z)), ((int(0.3 * X), 0, 0), (X, Y, Z)),
             ((0, 0, int(0.2 * Z)), (X, int(0.8 * Y), Z))]
    return [blend_weights(w.dims, lo, hi, (4, 4, 4)) for lo, hi in boxes][: w.n_views]


@pytest.mark.parametrize("norm,value", [("sum1", 0.0), ("min_overlap", 0.0), ("avg_overlap", 0.0), ("user", 1.5)])
def test_normalised_weights_match_oracle(mvd, norm, value):
    w = synth.config1()
    raw = _layout(w)
    want, T = oracle.normalize_weights(raw, norm, value)
    with mvd.Deconvolver(w.views, w.psfs) as d:
        got_T = d.set_weights(raw, norm, value)
        assert got_T == pytest.approx(T, rel=1e-6)
        for v in range(w.n_views):
            assert np.abs(d.weights(v) - want[v]).max() <= 1e-6


@pytest.mark.parametrize("path", ["direct", "fft"])
@pytest.mark.parametrize("norm", ["sum1", "min_overlap"])
def test_weighted_deconvolution_matches_oracle(mvd, path, norm):
    w = synth.config1()
    raw = _layout(w)
    ws, _ = oracle.normalize_weights(raw, norm)
    want, eps = oracle.deconvolve_weighted(w.views, w.psfs, w.n_iter, ws, "efficient")
    with mvd.Deconvolver(w.views, w.psfs, "efficient", path=path) as d:
        d.set_weights(raw, norm)
        d.iterate(w.n_iter)
        got = d.result().astype(np.float64)
    assert rel_err(got, want) < PARITY_TOL, err_report(got, want)


def test_weighted_mixed_radix_dims(mvd):
    w = synth.small_case(51, dims=(30, 24, 20), n_views=3, n_iter=4, asymmetric=True)
    raw = _layout(w)
    ws, _ = oracle.normalize_weights(raw, "avg_overlap")
    want, _ = oracle.deconvolve_weighted(w.views, w.psfs, w.n_iter, ws, "efficient")
    with mvd.Deconvolver(w.views, w.psfs, "efficient", path="fft") as d:
        d.set_weights(raw, "avg_overlap")
        d.iterate(w.n_iter)
        got = d.result().astype(np.float64)
    assert rel_err(got, want) < PARITY_TOL, err_report(got, want)


def test_removing_weights_restores_the_unweighted_update(mvd):
    import torch

    w = synth.config1()
    s = torch.cuda.Stream()
    with mvd.Deconvolver(w.views, w.psfs, path="fft", stream=s) as a, \
            mvd.Deconvolver(w.views, w.psfs, path="fft", stream=s) as b:
        a.set_weights(_layout(w), "sum1")
        a.iterate(1)  # captures a graph with the weights
        a.set_weights(None)
        a.set_estimate(None)
        a.iterate(3)
        b.iterate(3)
        assert np.array_equal(a.result(), b.result())


def test_weights_reject_bad_input_and_unsupported_forms(mvd):
    w = synth.config1()
    raw = _layout(w)
    with mvd.Deconvolver(w.views, w.psfs, path="fft") as d:
        bad = [r.copy() for r in raw]
        bad[0][0, 0, 0] = 1.5
        with pytest.raises(mvd.MvdError) as e:
            d.set_weights(bad)
        assert e.value.status == mvd.MVD_ERR_ARG
        d.set_weights(raw, "min_overlap")
        with pytest.raises(mvd.MvdError) as e:
            d.iterate_combined(1)
        assert e.value.status == mvd.MVD_ERR_UNSUPPORTED
        with pytest.raises(mvd.MvdError) as e:
            mvd.mvd_set_weights(d.ctx, raw, "user", 0.0)
        assert e.value.status == mvd.MVD_ERR_ARG


# ---------------------------------------------------------------------------
# Tikhonov regularisation (one-step-late form)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("path", ["direct", "fft"])
@pytest.mark.parametrize("lam", [0.0006, 0.006, 0.06])
def test_regularised_deconvolution_matches_oracle(mvd, path, lam):
    w = synth.config1()
    want, _ = oracle.deconvolve_weighted(w.views, w.psfs, w.n_iter, None, "efficient", lam=lam)
    with mvd.Deconvolver(w.views, w.psfs, "efficient", path=path) as d:
        d.set_regularization(lam)
        d.iterate(w.n_iter)
        got = d.result().astype(np.float64)
    assert rel_err(got, want) < PARITY_TOL, err_report(got, want)


@pytest.mark.parametrize("path", ["direct", "fft"])
def test_regularised_and_weighted_matches_oracle(mvd, path):
    w = synth.small_case(52, dims=(30, 24, 20), n_views=3, n_iter=4, asymmetric=True)
    raw = _layout(w)
    ws, _ = oracle.normalize_weights(raw, "min_overlap")
    want, _ = oracle.deconvolve_weighted(w.views, w.psfs, w.n_iter, ws, "efficient", lam=0.006)
    with mvd.Deconvolver(w.views, w.psfs, "efficient", path=path) as d:
        d.set_weights(raw, "min_overlap")
        d.set_regularization(0.006)
        d.iterate(w.n_iter)
        got = d.result().astype(np.float64)
    assert rel_err(got, want) < PARITY_TOL, err_report(got, want)


def test_regularisation_rejects_bad_values_and_unsupported_forms(mvd):
    w = synth.config1()
    with mvd.Deconvolver(w.views, w.psfs, path="fft") as d:
        for bad in (-1.0, float("nan"), float("inf")):
            with pytest.raises(mvd.MvdError) as e:
                d.set_regularization(bad)
            assert e.value.status == mvd.MVD_ERR_ARG
        d.set_regularization(0.006)
        with pytest.raises(mvd.MvdError) as e:
            d.iterate_combined(1)
        assert e.value.status == mvd.MVD_ERR_UNSUPPORTED
        d.set_regularization(0.0)
        d.iterate_combined(1)
