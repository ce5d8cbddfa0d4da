"""The 1024x1024x512 seven-view specimen (PSF boxes 19x19x51, rotated) at full size on
the GPU, with its inputs generated on the device (`synth.config3_device`, the
same recipe as the CPU generator; the CPU generator takes minutes and tens of GB
at this size).

- Parity over every voxel: the first iteration from the flat start (the seven
  view updates, PSF boxes 19x19x51 to 53x19x29) against the oracle's FFT leg
  (FP64, pinned against the direct sums in tests/test_oracle_fft.py), all 537 M
  voxels, tau from the whole volume.
- At any size: conservation with plain kernels after a view update, positivity
  and finiteness after the specimen's 10 iterations.

The iteration counts that the oracle cannot reach at this size (10 iterations
are 70 full-size updates) are covered on grids with the same transform lengths
and PSFs in tests/test_gpu_full_parity.py.
"""
import os

import numpy as np
import pytest

import oracle
import synth
from tests._util import PARITY_TOL, err_report, rel_err

pytestmark = pytest.mark.gpu

SCHEDULE = [0, 1, 2, 3, 4, 5, 6]  # one iteration


def _host_bytes():
    try:
        return os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES")
    except (ValueError, OSError, AttributeError):
        return 0


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    free, _ = torch.cuda.mem_get_info()
    if free < 120 * 2**30:
        pytest.skip("needs 120 GiB of free device memory")
    if _host_bytes() < 96 * 2**30:
        pytest.skip("needs 96 GiB of host memory for the FP64 oracle at this size")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1308_0730_gb300 import mvd

    mvd.load()
    return torch, mvd


def test_specimen_full_size(env):
    torch, mvd = env
    w = synth.config3_device(device="cuda:0")
    s = torch.cuda.Stream()
    with mvd.Deconvolver(w.views, w.psfs, "efficient", path="fft", stream=s) as d:
        hviews = w.host_views()
        w.views = None
        torch.cuda.empty_cache()
        eps = d.eps
        d.iterate(1, SCHEDULE)
        got = d.result()
        # the specimen's ten iterations: positive and finite
        d.set_estimate(None)
        d.iterate(w.n_iter)
        psi10 = d.result()
        assert psi10.min() >= eps * (1 - 1e-7)
        assert np.isfinite(psi10).all()
        del psi10
        # plain kernels: sum(psi) = sum(phi_v) after an update (the background keeps b above eps)
        mvd.mvd_precompute_kernels(d.ctx, "plain")
        d.set_estimate(None)
        d.iterate(1, [3])
        tot = float(hviews[3].astype(np.float64).sum())
        got_tot = float(d.result().astype(np.float64).sum())
        assert abs(got_tot - tot) < 1e-5 * tot, (got_tot, tot)
    want, oeps = oracle.deconvolve_fft(hviews, w.psfs, 1, schedule=SCHEDULE)
    assert abs(oeps - eps) <= 1e-6 * eps
    print(f"specimen, first iteration at full size: {err_report(got, want)}")
    assert rel_err(got, want) < PARITY_TOL, err_report(got, want)
