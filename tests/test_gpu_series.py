"""Time series with fixed PSFs: new views loaded into an existing context
(mvd_set_views) against fresh contexts and the FP64 oracle."""
import numpy as np
import pytest

import oracle
import synth
from tests._util import PARITY_TOL, err_report, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1308_0730_gb300 import mvd as m

    m.load()
    return torch, m


def _series(n=3):
    """Time points of one acquisition: the same PSFs, a drifting object, fresh noise."""
    from synth.workloads import time_series

    base = synth.small_case(71, dims=(40, 32, 24), n_views=3, n_iter=4, asymmetric=True)
    return base, time_series(base, n, 500)


@pytest.mark.parametrize("path", ["direct", "fft"])
@pytest.mark.parametrize("boundary", ["periodic", "zero"])
def test_loaded_views_match_fresh_contexts(env, path, boundary):
    torch, mvd = env
    base, series = _series()
    s = torch.cuda.Stream()
    with mvd.Deconvolver(series[0], base.psfs, path=path, stream=s, boundary=boundary) as d:
        for views in series:
            d.set_views(views)
            d.iterate(base.n_iter)
            got = d.result()
            with mvd.Deconvolver(views, base.psfs, path=path, stream=s, boundary=boundary) as f:
                assert d.eps == f.eps and d.psi0 == f.psi0
                f.iterate(base.n_iter)
                assert np.array_equal(got, f.result())


def test_warm_start_from_the_previous_time_point(env):
    torch, mvd = env
    base, series = _series(2)
    with mvd.Deconvolver(series[0], base.psfs, path="fft", stream=torch.cuda.Stream()) as d:
        d.iterate(base.n_iter)
        prev = d.result()
        d.set_views(series[1])
        eps = d.eps
        d.set_estimate(prev)
        d.iterate(2)
        got = d.result()
    want, _ = oracle.deconvolve(series[1], base.psfs, 2, "efficient", eps=eps, psi_init=prev)
    assert rel_err(got, want) < PARITY_TOL, err_report(got, want)


def test_fixed_eps_and_device_views(env):
    torch, mvd = env
    base, series = _series(2)
    with mvd.Deconvolver(series[0], base.psfs, path="fft", eps=0.01, stream=torch.cuda.Stream()) as d:
        d.set_views([torch.from_numpy(v).cuda() for v in series[1]])
        assert d.eps == pytest.approx(0.01)
        d.iterate(base.n_iter)
        got = d.result()
    want, _ = oracle.deconvolve(series[1], base.psfs, base.n_iter, "efficient", eps=0.01)
    assert rel_err(got, want) < PARITY_TOL, err_report(got, want)


def test_rejected_views_block_iteration_until_a_good_load(env):
    torch, mvd = env
    base, series = _series(2)
    with mvd.Deconvolver(series[0], base.psfs, path="fft", stream=torch.cuda.Stream()) as d:
        bad = [v.copy() for v in series[1]]
        bad[1][3, 4, 5] = -1.0
        with pytest.raises(mvd.MvdError) as e:
            d.set_views(bad)
        assert e.value.status == mvd.MVD_ERR_ARG
        with pytest.raises(mvd.MvdError) as e:
            d.iterate(1)
        assert e.value.status == mvd.MVD_ERR_STATE
        with pytest.raises(mvd.MvdError) as e:
            d.set_views([np.zeros_like(v) for v in series[1]])
        assert e.value.status == mvd.MVD_ERR_ARG
        d.set_views(series[1])
        d.iterate(base.n_iter)
        got = d.result()
    want, _ = oracle.deconvolve(series[1], base.psfs, base.n_iter, "efficient")
    assert rel_err(got, want) < PARITY_TOL, err_report(got, want)
