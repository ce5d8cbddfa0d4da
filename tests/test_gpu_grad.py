"""GPU adjoint of the unrolled iteration (through the C ABI and the autograd
front end) against the FP64 oracle's reverse-mode gradient and FP64 central
finite differences of the oracle run."""
import hashlib
import os

import numpy as np
import pytest

import oracle
import synth
from synth.workloads import config5_sigmas, gaussian_psf

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-3  # relative to the largest gradient component


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1308_0730_gb300 import autograd, mvd

    mvd.load()
    return torch, mvd, autograd


def _rel(got, want):
    got, want = np.asarray(got, np.float64), np.asarray(want, np.float64)
    return float(np.abs(got - want).max() / max(np.abs(want).max(), 1e-300))


def _gpu_run(env, w, psfs, n_iter, variant="efficient", path="auto"):
    torch, _, ag = env
    views = torch.from_numpy(np.stack([np.asarray(v, np.float32) for v in w.views])).cuda().requires_grad_(True)
    ps = [torch.from_numpy(np.asarray(p, np.float32)).requires_grad_(True) for p in psfs]
    psi = ag.unrolled_deconvolve(views, ps, n_iter, variant, path)
    truth = torch.from_numpy(np.asarray(w.truth, np.float32)).cuda()
    loss = torch.mean((psi.double() - truth.double()) ** 2)
    loss.backward()
    return float(loss.detach()), psi.detach().cpu().numpy(), views.grad.cpu().numpy(), [p.grad.numpy() for p in ps]


@pytest.fixture(scope="module")
def small():
    return synth.small_case(21, dims=(20, 16, 12), n_views=3, asymmetric=True, n_iter=3)


@pytest.mark.parametrize("path", ["direct", "fft"])
def test_unrolled_forward_equals_iterate(env, small, path):
    _, mvd, _ = env
    _, psi, _, _ = _gpu_run(env, small, small.psfs, small.n_iter, path=path)
    with mvd.Deconvolver(small.views, small.psfs, path=path) as d:
        d.iterate(small.n_iter)
        want = d.result()
    assert np.array_equal(psi, want)


@pytest.mark.parametrize("path", ["direct", "fft"])
@pytest.mark.parametrize("variant", ["efficient", "opt1", "opt2", "plain"])
def test_adjoint_matches_oracle_gradient(env, small, variant, path):
    loss, psi, gv, gp = _gpu_run(env, small, small.psfs, small.n_iter, variant, path)
    oloss, ogv, ogp, opsi = oracle.unrolled_grad(small.views, small.psfs, small.n_iter, small.truth, variant)
    assert abs(loss - oloss) <= 1e-4 * oloss
    err_v = _rel(np.stack(gv), np.stack(ogv))
    assert err_v < GRAD_TOL, f"view gradients: {err_v:.3e}"
    for v in range(small.n_views):
        err_p = _rel(gp[v], ogp[v])
        assert err_p < GRAD_TOL, f"PSF {v} gradient: {err_p:.3e}"


def test_zero_iterations_spread_the_flat_start(env, small):
    loss, psi, gv, gp = _gpu_run(env, small, small.psfs, 0)
    psi0 = oracle.mean_views(small.views)
    assert np.allclose(psi, psi0, rtol=1e-6)
    g = 2.0 * (psi0 - np.asarray(small.truth, np.float64)) / small.truth.size
    want = g.sum() / (small.n_views * small.truth.size)
    assert np.allclose(np.stack(gv), want, rtol=1e-4, atol=1e-12)
    for p in gp:
        assert np.abs(p).max() == 0.0


def test_backward_needs_a_forward_run(env, small):
    torch, mvd, _ = env
    with mvd.Deconvolver(small.views, small.psfs) as d:
        g = torch.zeros(small.truth.shape, dtype=torch.float32, device="cuda")
        gv = [torch.empty_like(g) for _ in range(small.n_views)]
        with pytest.raises(mvd.MvdError) as e:
            mvd.mvd_unrolled_backward(d.ctx, g, gv, [p.shape for p in small.psfs])
        assert e.value.status == mvd.MVD_ERR_STATE


def _sigma_chain(env, w, sigmas, n_iter, path="auto"):
    """Full calibration chain on the GPU: sigma -> Gaussian PSFs -> K iterations -> MSE; returns dL/dsigma."""
    torch, _, ag = env
    box, angles = w.meta["box"], w.meta["angles"]
    from synth.workloads import rotated_box

    sig = [torch.tensor(s, dtype=torch.float64, requires_grad=True) for s in sigmas]
    psfs = [ag.gaussian_psf(s, rotated_box(box, a), a, "z") for s, a in zip(sig, angles)]
    views = torch.from_numpy(np.stack(w.views)).cuda()
    psi = ag.unrolled_deconvolve(views, psfs, n_iter, path=path)
    truth = torch.from_numpy(w.truth).cuda()
    loss = torch.mean((psi.double() - truth.double()) ** 2)
    loss.backward()
    return float(loss.detach()), np.array([s.grad.numpy() for s in sig])


@pytest.mark.parametrize("path", ["direct", "fft"])
def test_sigma_gradient_matches_finite_differences_24cubed(env, path):
    """The 24^3 copy of the calibration workload: FP64 central differences (step 1e-4) of the oracle run."""
    w = synth.config5_crop()
    sig0 = config5_sigmas(w.n_views)
    box, angles = w.meta["box"], w.meta["angles"]
    truth64 = w.truth.astype(np.float64)

    def oracle_loss(sig):
        psfs = [gaussian_psf(s[0], s[1], box, "z", a) for s, a in zip(sig, angles)]
        psi, _ = oracle.deconvolve(w.views, psfs, w.n_iter)
        return float(np.mean((psi - truth64) ** 2))

    h = 1e-4
    fd = np.zeros((w.n_views, 2))
    for v in range(w.n_views):
        for k in range(2):
            sp = [list(s) for s in sig0]
            sm = [list(s) for s in sig0]
            sp[v][k] += h
            sm[v][k] -= h
            fd[v, k] = (oracle_loss(sp) - oracle_loss(sm)) / (2 * h)
    loss, g = _sigma_chain(env, w, sig0, w.n_iter, path)
    assert abs(loss - oracle_loss(sig0)) <= 1e-4 * loss
    err = _rel(g, fd)
    assert err < GRAD_TOL, f"sigma gradient vs finite differences: {err:.3e}\n{g}\n{fd}"


GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "oracle_grad_unrolled_128x128x96.txt")


@pytest.mark.skipif(not os.path.exists(GOLDEN), reason="stored oracle gradients not written")
def test_full_size_gradients_match_stored_oracle(env):
    """128x128x96, 4 views, boxes 15x15x41 rotated, 8 iterations: sigma gradients against the stored FP64
    finite differences and reverse-mode values, view and PSF gradients at the stored samples."""
    from tests.golden import make_oracle_grad as mg

    torch, mvd, ag = env
    ref = mg.read()
    w = synth.config5()
    sig0 = config5_sigmas(w.n_views)
    assert mg.input_digest(w, mg.model_psfs(w, sig0)) == ref["digest"], "inputs differ from the stored run"
    loss, g = _sigma_chain(env, w, sig0, w.n_iter, "fft")
    assert abs(loss - ref["loss"]) <= 1e-4 * ref["loss"]
    assert _rel(g, ref["dsigma_fd"]) < GRAD_TOL, (g, ref["dsigma_fd"])
    assert _rel(g, ref["dsigma_adjoint"]) < GRAD_TOL, (g, ref["dsigma_adjoint"])
    psfs = [mvd.mvd_gaussian_psf(s[0], s[1], synth.workloads.rotated_box(w.meta["box"], a), a, "z")
            for s, a in zip(sig0, w.meta["angles"])]
    _, _, gv, gp = _gpu_run(env, w, psfs, w.n_iter, path="fft")
    for v in range(w.n_views):
        idx, val = ref["dview"][v]
        e = np.abs(gv[v].ravel()[idx] - val).max() / ref["max_abs_dview"][v]
        assert e < GRAD_TOL, f"view {v} gradient: {e:.3e}"
        idx, val = ref["dpsf"][v]
        e = np.abs(gp[v].ravel()[idx] - val).max() / ref["max_abs_dpsf"][v]
        assert e < GRAD_TOL, f"PSF {v} gradient: {e:.3e}"
