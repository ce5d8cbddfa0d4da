"""Combined (simultaneous) update of Eq. 50 / Eq. 220 on the GPU, with and
without the |V|-th root, against the FP64 oracle."""
import numpy as np
import pytest

import oracle
import synth
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


CASES = {
    "blobs32": lambda: synth.config1(),
    "smooth-30x24x20": lambda: synth.small_case(41, dims=(30, 24, 20), n_views=3, n_iter=3, asymmetric=True),
    "odd-21x17x13": lambda: synth.small_case(42, dims=(21, 17, 13), n_views=2, n_iter=3, asymmetric=True),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("path", ["direct", "fft"])
@pytest.mark.parametrize("root", [True, False])
def test_combined_matches_oracle(mvd, case, path, root):
    w = CASES[case]()
    if path == "fft" and case.startswith("odd"):
        pytest.skip("the FFT engine needs {2,3,5}-smooth dims")
    n_iter = 5 if root else 2  # the plain product grows quickly; two steps keep it in range
    want, eps = oracle.deconvolve_combined(w.views, w.psfs, n_iter, "efficient", root=root)
    with mvd.Deconvolver(w.views, w.psfs, "efficient", path=path) as d:
        assert abs(d.eps - eps) <= 1e-6 * eps
        d.iterate_combined(n_iter, root)
        got = d.result().astype(np.float64)
    assert rel_err(got, want) < PARITY_TOL, err_report(got, want)


@pytest.mark.parametrize("path", ["direct", "fft"])
@pytest.mark.parametrize("root", [True, False])
def test_noise_free_truth_is_a_fixed_point(mvd, path, root):
    w = synth.config1()
    truth = w.truth.astype(np.float64) + 1.0
    psfs = [p.astype(np.float64) / p.astype(np.float64).sum() for p in w.psfs]
    views = [oracle.conv(truth, p).astype(np.float32) for p in psfs]
    with mvd.Deconvolver(views, w.psfs, "efficient", path=path) as d:
        d.set_estimate(truth.astype(np.float32))
        d.iterate_combined(3, root)
        got = d.result().astype(np.float64)
    assert rel_err(got, truth) < PARITY_TOL, err_report(got, truth)


def test_graph_replay_equals_plain_launches(mvd, monkeypatch):
    import torch

    w = synth.config1()
    s = torch.cuda.Stream()
    outs = []
    for no_graph in ("0", "1"):
        monkeypatch.setenv("MVD_NO_GRAPH", no_graph)
        with mvd.Deconvolver(w.views, w.psfs, "efficient", path="fft", stream=s) as d:
            d.iterate_combined(3)
            d.iterate(1)  # the sequential and combined forms mix on one context
            d.iterate_combined(1)
            outs.append(d.result())
    assert np.array_equal(outs[0], outs[1])


def test_combined_rejects_bad_calls(mvd):
    w = synth.config1()
    with mvd.Deconvolver(w.views, w.psfs) as d:
        with pytest.raises(mvd.MvdError) as e:
            d.iterate_combined(-1)
        assert e.value.status == mvd.MVD_ERR_ARG
    lib = mvd.load()
    assert lib.mvd_iterate_combined(None, 1, 1) == mvd.MVD_ERR_ARG
