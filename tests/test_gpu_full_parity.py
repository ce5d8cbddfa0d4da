"""Whole-volume GPU parity at full iteration counts: every voxel of the CUDA path's
estimate against the oracle's FFT leg (`oracle.deconvolve_fft`, FP64, pinned
against the direct-sum oracle in tests/test_oracle_fft.py), on identical seeded
inputs, with the parity floor tau = 1e-3 * max|oracle| taken over the whole
volume.

- The 256x256x128 four-view workload after its 20 iterations (8.4 M voxels).
- Grids that carry the 1024x1024x512 specimen's transform lengths (1024 along x,
  1024 along y, 512 along z) with its seven rotated 19x19x51 PSFs (boxes up to
  53x19x53) and its object density, photon level and background, after its 10
  iterations. Each uses the same register-resident passes as the full specimen
  on its long axis.
"""
import numpy as np
import pytest

import oracle
import synth
from tests._util import PARITY_TOL, err_report, rel_err

pytestmark = pytest.mark.gpu

SPECIMEN_VOXELS = 1024 * 1024 * 512
SPECIMEN_OBJECTS = 150_000


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


def _gpu_run(mvd, w, n_iter):
    with mvd.Deconvolver(w.views, w.psfs, "efficient", path="fft") as d:
        d.iterate(n_iter)
        return d.result().astype(np.float64), d.eps


def test_mid_every_voxel_after_20_iterations(mvd):
    w = synth.config2()
    want, eps = oracle.deconvolve_fft(w.views, w.psfs, w.n_iter)
    got, geps = _gpu_run(mvd, w, w.n_iter)
    assert abs(geps - eps) <= 1e-6 * eps
    print(f"{w.name}, {w.n_iter} iterations, every voxel: {err_report(got, want)}")
    assert rel_err(got, want) < PARITY_TOL, err_report(got, want)


@pytest.fixture(scope="module")
def specimen_kernels():
    """Compound kernels (Eq. 222) of the specimen's seven PSFs, computed once by the oracle."""
    w = synth.config3(dims=(64, 24, 64), n_objects=1)
    pn = [p.astype(np.float64) / p.astype(np.float64).sum() for p in w.psfs]
    return [oracle.compound(pn, v, "efficient") for v in range(len(pn))]


@pytest.mark.parametrize("dims", [(1024, 32, 64), (64, 1024, 64), (64, 32, 512)],
                         ids=["x1024", "y1024", "z512"])
def test_specimen_lengths_every_voxel_after_10_iterations(mvd, specimen_kernels, dims):
    n_obj = max(1, round(SPECIMEN_OBJECTS * dims[0] * dims[1] * dims[2] / SPECIMEN_VOXELS))
    w = synth.config3(dims=dims, n_objects=n_obj)
    assert w.n_iter == 10
    want, eps = oracle.deconvolve_fft(w.views, w.psfs, w.n_iter, kernels=specimen_kernels)
    got, geps = _gpu_run(mvd, w, w.n_iter)
    assert abs(geps - eps) <= 1e-6 * eps
    print(f"{w.name}, {w.n_iter} iterations, every voxel: {err_report(got, want)}")
    assert rel_err(got, want) < PARITY_TOL, err_report(got, want)
