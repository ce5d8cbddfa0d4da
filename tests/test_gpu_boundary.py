"""Zero and mirror boundaries on the GPU (the volume continued by zeros or by
its reflection): the padded-grid engines with the sensitivity-normalised
update, against the FP64 oracle's zero- and mirror-boundary deconvolutions."""
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


BLUR = {"zero": oracle.conv_zero, "mirror": oracle.conv_mirror}
DECONVOLVE = {"zero": oracle.deconvolve_zero, "mirror": oracle.deconvolve_mirror}
BOUNDARIES = ["zero", "mirror"]


def _boundary_views(w, seed, boundary="zero"):
    """Views of the workload's object blurred with the given boundary, with Poisson noise."""
    rng = np.random.default_rng(seed)
    truth = w.truth.astype(np.float64)
    views = []
    for p in w.psfs:
        p = p.astype(np.float64)
        b = BLUR[boundary](truth, p / p.sum())
        views.append(rng.poisson(np.maximum(b, 0.0)).astype(np.float32) + np.float32(0.5))
    return views


def _run(mvd, views, psfs, n_iter, variant, path, boundary, precision="precise"):
    with mvd.Deconvolver(views, psfs, variant, path=path, precision=precision, boundary=boundary) as d:
        d.iterate(n_iter)
        return d.result().astype(np.float64)


@pytest.mark.parametrize("boundary", BOUNDARIES)
@pytest.mark.parametrize("path", ["direct", "fft"])
@pytest.mark.parametrize("variant", ["plain", "efficient"])
def test_boundary_matches_oracle(env, boundary, path, variant):
    _, mvd = env
    w = synth.config1()  # 32^3, padded to 40^3 (zero) or 45 x 45 x 45 (mirror): mixed-radix FFT lengths
    views = _boundary_views(w, 7, boundary)
    want, _ = DECONVOLVE[boundary](views, w.psfs, w.n_iter, variant)
    got = _run(mvd, views, w.psfs, w.n_iter, variant, path, boundary)
    assert got.shape == want.shape
    assert rel_err(got, want) < PARITY_TOL, err_report(got, want)


@pytest.mark.parametrize("boundary,dims", [("zero", (60, 28, 24)), ("zero", (37, 29, 23)),
                                           ("mirror", (58, 28, 24)), ("mirror", (37, 29, 23))])
def test_boundary_odd_and_power_of_two_padding(env, boundary, dims):
    """Zero: (60, 28, 24) pads to 64 x 30 x 27 and (37, 29, 23) to 40 x 32 x 27. Mirror (twice
    the halo): (58, 28, 24) pads to 64 x 32 x 30 and (37, 29, 23) to 45 x 36 x 30. The
    power-of-two x lengths take the register-resident double-float x transforms."""
    _, mvd = env
    w = synth.small_case(61, dims=dims, n_views=3, n_iter=4, asymmetric=True)
    views = _boundary_views(w, 8, boundary)
    want, _ = DECONVOLVE[boundary](views, w.psfs, w.n_iter, "efficient")
    for path in ("fft", "direct"):
        got = _run(mvd, views, w.psfs, w.n_iter, "efficient", path, boundary)
        assert rel_err(got, want) < PARITY_TOL, f"{path}: {err_report(got, want)}"


@pytest.mark.parametrize("boundary", BOUNDARIES)
def test_boundary_fast_fp32_mode(env, boundary):
    """MVD_FAST: the FP32 engine (and its FP32 sensitivity) for two iterations."""
    _, mvd = env
    w = synth.small_case(67, dims=(40, 30, 24), n_views=3, n_iter=2, asymmetric=True)
    views = _boundary_views(w, 12, boundary)
    want, _ = DECONVOLVE[boundary](views, w.psfs, 2, "efficient")
    got = _run(mvd, views, w.psfs, 2, "efficient", "fft", boundary, precision="fast")
    assert rel_err(got, want) < PARITY_TOL, err_report(got, want)


@pytest.mark.parametrize("boundary", BOUNDARIES)
def test_noise_free_truth_is_a_fixed_point(env, boundary):
    """Views blurred with the boundary, estimate set to the object: the update keeps it."""
    _, mvd = env
    w = synth.small_case(62, dims=(24, 20, 16), n_views=3, n_iter=2, asymmetric=True)
    truth = w.truth.astype(np.float64) + 2.0
    psfs = [p.astype(np.float64) / p.astype(np.float64).sum() for p in w.psfs]
    views = [BLUR[boundary](truth, p).astype(np.float32) for p in psfs]
    for path in ("fft", "direct"):
        with mvd.Deconvolver(views, w.psfs, "efficient", path=path, boundary=boundary) as d:
            d.set_estimate(truth.astype(np.float32))
            d.iterate(2)
            got = d.result().astype(np.float64)
        assert rel_err(got, truth) < PARITY_TOL, f"{path}: {err_report(got, truth)}"


@pytest.mark.parametrize("boundary", BOUNDARIES)
def test_estimate_layout_and_device_views(env, boundary):
    """set_estimate / result / result_device keep the user's X*Y*Z layout; device views match host views."""
    torch, mvd = env
    w = synth.small_case(63, dims=(20, 18, 14), n_views=2, n_iter=3)
    views = _boundary_views(w, 9, boundary)
    rng = np.random.default_rng(5)
    psi = rng.uniform(0.5, 2.0, size=w.truth.shape).astype(np.float32)
    with mvd.Deconvolver(views, w.psfs, path="fft", boundary=boundary) as d:
        d.set_estimate(psi)
        assert np.array_equal(d.result(), psi)
        ptr = mvd.mvd_result_device(d.ctx)
        mvd.mvd_synchronize(d.ctx)

        class _Dev:
            __cuda_array_interface__ = {"shape": psi.shape, "typestr": "<f4", "data": (ptr, False), "version": 3}

        assert np.array_equal(torch.as_tensor(_Dev(), device="cuda").cpu().numpy(), psi)
        d.set_estimate(torch.from_numpy(psi).cuda())
        assert np.array_equal(d.result(), psi)
        bad = psi.copy()
        bad[3, 4, 5] = 0.0
        with pytest.raises(mvd.MvdError):
            d.set_estimate(bad)  # rejected: the estimate falls back to the flat start
        assert np.allclose(d.result(), mvd.mvd_get_psi0(d.ctx))
        d.set_estimate(psi)
        d.iterate(w.n_iter)
        host = d.result()
    dev_views = [torch.from_numpy(v).cuda() for v in views]
    with mvd.Deconvolver(dev_views, w.psfs, path="fft", boundary=boundary) as d:
        d.set_estimate(psi)
        d.iterate(w.n_iter)
        assert np.array_equal(d.result(), host)


def test_branch_batch_takes_zero_and_mirror_boundary_contexts(env):
    torch, mvd = env
    ws = [synth.small_case(64, dims=(24, 20, 16), n_views=2, n_iter=3),
          synth.small_case(65, dims=(30, 16, 12), n_views=3, n_iter=3)]
    ws.append(synth.small_case(68, dims=(20, 24, 14), n_views=2, n_iter=3))
    bounds = ["zero", "periodic", "mirror"]
    vs = [_boundary_views(w, 10 + i, "mirror" if bd == "mirror" else "zero") for i, (w, bd) in
          enumerate(zip(ws, bounds))]
    s = torch.cuda.Stream()
    plain = []
    for w, v, bd in zip(ws, vs, bounds):
        with mvd.Deconvolver(v, w.psfs, path="fft", stream=s, boundary=bd) as d:
            d.iterate(3)
            plain.append(d.result())
    ds = [mvd.Deconvolver(v, w.psfs, path="fft", stream=s, boundary=bd) for w, v, bd in zip(ws, vs, bounds)]
    try:
        with pytest.raises(mvd.MvdError) as e:
            mvd.mvd_batch_create(ds, 3, "persistent")
        assert e.value.status == mvd.MVD_ERR_UNSUPPORTED
        b = mvd.mvd_batch_create(ds, 3, "branches")
        try:
            mvd.mvd_batch_run(b)
            mvd.mvd_batch_wait(b)
            got = [d.result() for d in ds]
        finally:
            mvd.mvd_batch_destroy(b)
    finally:
        for d in ds:
            d.close()
    for g, p in zip(got, plain):
        assert np.array_equal(g, p)


@pytest.mark.parametrize("boundary", BOUNDARIES)
def test_boundary_rejects_the_unrolled_form(env, boundary):
    """The unrolled (differentiable) form needs the periodic boundary; the context stays
    usable after the refusal. (Weights, lambda and the combined update with these
    boundaries: tests/test_gpu_boundary_combos.py.)"""
    _, mvd = env
    w = synth.small_case(66, dims=(16, 12, 10), n_views=2, n_iter=1)
    with mvd.Deconvolver(w.views, w.psfs, path="fft", boundary=boundary) as d:
        with pytest.raises(mvd.MvdError) as e:
            mvd.mvd_unrolled_forward(d.ctx, 1)
        assert e.value.status == mvd.MVD_ERR_UNSUPPORTED
        d.iterate(1)
