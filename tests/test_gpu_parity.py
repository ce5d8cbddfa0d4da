"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle,
element by element on identical seeded inputs."""
import os

import numpy as np
import pytest

import oracle
import synth
from tests._util import PARITY_TOL, err_report, rel_err

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


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


def _run_gpu(mvd, w, variant="efficient", path="auto", n_iter=None, schedule=None, eps=0.0):
    with mvd.Deconvolver(w.views, w.psfs, variant, eps=eps, path=path) as d:
        d.iterate(w.n_iter if n_iter is None else n_iter, schedule)
        return d.result().astype(np.float64), d.path, d.eps


# ---------------------------------------------------------------------------
# the tiny blob workload (32^3, 3 views, 10 iterations), both engines
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def cfg1():
    w = synth.config1()
    want, eps = oracle.deconvolve(w.views, w.psfs, w.n_iter, "efficient")
    return w, want, eps


@pytest.mark.parametrize("path", ["auto", "direct", "fft"])
def test_blobs32_parity(mvd, cfg1, path):
    w, want, eps = cfg1
    got, used, geps = _run_gpu(mvd, w, path=path)
    if path != "auto":
        assert used == path
    assert abs(geps - eps) <= 1e-6 * eps
    err = rel_err(got, want)
    assert err < PARITY_TOL, err_report(got, want)


def test_blobs32_parity_every_iteration(mvd, cfg1):
    """Error reported after every iteration, not only at the end."""
    w, _, _ = cfg1
    psi_o = None
    with mvd.Deconvolver(w.views, w.psfs, "efficient", path="fft") as d:
        for it in range(w.n_iter):
            d.iterate(1)
            got = d.result().astype(np.float64)
            psi_o, _ = oracle.deconvolve(w.views, w.psfs, 1, "efficient", psi_init=psi_o)
            assert rel_err(got, psi_o) < PARITY_TOL, f"iteration {it + 1}: {err_report(got, psi_o)}"


# ---------------------------------------------------------------------------
# small random problems: ragged tiles, mixed radices, asymmetric PSFs,
# every variant, custom schedules
# ---------------------------------------------------------------------------

CASES = [
    # dims (X,Y,Z), boxes, asymmetric
    ((16, 12, 10), [(5, 3, 7), (3, 5, 5)], True),
    ((24, 20, 18), [(7, 3, 5), (3, 7, 3), (5, 5, 9)], True),
    ((30, 25, 27), [(5, 5, 5), (9, 3, 3)], False),
    ((45, 36, 15), [(3, 3, 3), (5, 7, 9)], True),
    ((64, 48, 40), [(7, 7, 13), (13, 7, 7)], True),
    ((9, 10, 12), [(9, 3, 5), (3, 9, 11)], True),
]


@pytest.mark.parametrize("path", ["direct", "fft"])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_small_cases(mvd, case, path):
    dims, boxes, asym = CASES[case]
    w = synth.small_case(100 + case, dims=dims, n_views=len(boxes), boxes=boxes, n_iter=3, asymmetric=asym)
    want, _ = oracle.deconvolve(w.views, w.psfs, 3, "efficient")
    got, used, _ = _run_gpu(mvd, w, path=path, n_iter=3)
    assert used == path
    assert rel_err(got, want) < PARITY_TOL, err_report(got, want)


@pytest.mark.parametrize("variant", ["plain", "efficient", "opt1", "opt2"])
@pytest.mark.parametrize("path", ["direct", "fft"])
def test_variants(mvd, variant, path):
    w = synth.small_case(7, dims=(20, 18, 24), n_views=3, boxes=[(5, 5, 9), (9, 5, 5), (5, 9, 5)], n_iter=4,
                         asymmetric=True)
    want, _ = oracle.deconvolve(w.views, w.psfs, 4, variant)
    got, _, _ = _run_gpu(mvd, w, variant=variant, path=path, n_iter=4)
    assert rel_err(got, want) < PARITY_TOL, err_report(got, want)


@pytest.mark.parametrize("schedule", [[2, 0, 1], [1, 1, 0], [2]])
def test_custom_schedule(mvd, schedule):
    w = synth.small_case(8, dims=(16, 16, 16), n_views=3, boxes=[(5, 3, 3), (3, 5, 3), (3, 3, 5)], n_iter=2,
                         asymmetric=True)
    want, _ = oracle.deconvolve(w.views, w.psfs, 2, "efficient", schedule=schedule)
    for path in ("direct", "fft"):
        got, _, _ = _run_gpu(mvd, w, path=path, n_iter=2, schedule=schedule)
        assert rel_err(got, want) < PARITY_TOL, f"{path}: {err_report(got, want)}"


def test_compound_kernels_match_oracle(mvd):
    w = synth.small_case(9, dims=(40, 40, 48), n_views=4,
                         boxes=[(7, 7, 15), (15, 7, 7), (7, 7, 15), (15, 7, 7)], asymmetric=True)
    for variant in ("plain", "efficient", "opt1", "opt2"):
        with mvd.Deconvolver(w.views, w.psfs, variant, path="direct") as d:
            for v in range(w.n_views):
                got = d.compound_kernel(v).astype(np.float64)
                want = oracle.compound([p.astype(np.float64) / p.astype(np.float64).sum() for p in w.psfs], v,
                                       variant)
                assert np.max(np.abs(got - want)) < 2e-6 * np.max(want), (variant, v)


def test_hand_worked_example_on_gpu(mvd):
    """The 4x1x1 two-view example worked out by hand (golden file), PLAIN variant."""
    vals = {}
    for line in open(os.path.join(GOLDEN, "hand_update_4x1x1.txt")):
        if line.strip() and not line.startswith("#"):
            name, *nums = line.split()
            vals[name] = np.array([float(x) for x in nums])
    P0 = np.array([0.2, 0.8, 0.0], np.float32).reshape(1, 1, 3)
    P1 = np.array([0.25, 0.5, 0.25], np.float32).reshape(1, 1, 3)
    phi0 = np.array([2.0, 0.0, 1.0, 1.0], np.float32).reshape(1, 1, 4)
    phi1 = np.ones((1, 1, 4), np.float32)
    for path in ("direct", "fft"):
        with mvd.Deconvolver([phi0, phi1], [P0, P1], "plain", eps=1e-9, path=path) as d:
            d.set_estimate(np.ones((1, 1, 4), np.float32))
            d.iterate(1, [0])
            assert np.allclose(d.result().ravel(), vals["plain_view0"], rtol=1e-6), path
            d.set_estimate(np.ones((1, 1, 4), np.float32))
            d.iterate(1)
            assert np.allclose(d.result().ravel(), vals["plain_iter1"], rtol=1e-6), path
        with mvd.Deconvolver([phi0, phi1], [P0, P1], "efficient", path=path) as d:
            assert np.allclose(d.compound_kernel(0).ravel(), vals["efficient_comp0"], atol=1e-7)
            assert np.allclose(d.compound_kernel(1).ravel(), vals["efficient_comp1"], atol=1e-7)


# ---------------------------------------------------------------------------
# properties at the 256x256x128 size (any size)
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def cfg2():
    return synth.config2()


def test_mid_volume_single_update_sampled_parity(mvd, cfg2):
    """One view update at full size from the flat start, compared on sampled voxels
    that the oracle evaluates one by one from the definitions."""
    w = cfg2
    rng = np.random.default_rng(0)
    idx = rng.choice(w.voxels, 48, replace=False)
    psfs64 = [p.astype(np.float64) / p.astype(np.float64).sum() for p in w.psfs]
    with mvd.Deconvolver(w.views, w.psfs, "efficient", path="fft") as d:
        psi0 = np.full(w.truth.shape, d.psi0, np.float64)
        eps = d.eps
        d.iterate(1, [1])
        got = d.result().ravel()[idx].astype(np.float64)
    K = oracle.compound(psfs64, 1, "efficient")
    want = oracle.update_at(psi0, w.views[1], psfs64[1], K, eps, idx)
    assert rel_err(got, want) < PARITY_TOL, err_report(got, want)


def test_mid_volume_conservation_and_positivity(mvd, cfg2):
    """PLAIN kernels: after each view update sum(psi) = sum(phi_v) (normalised PSF, exact
    adjoint) while no clamp is active, up to FP32 rounding. Noise-free views of the truth plus
    a background keep every ratio and factor well above eps. Then, on the Poisson views (many
    zeros, clamps active), psi stays >= eps everywhere."""
    w = cfg2
    psfs64 = [p.astype(np.float64) / p.astype(np.float64).sum() for p in w.psfs]
    views = [synth.workloads.blur_circular(w.truth.astype(np.float64) + 2.0, p).astype(np.float32)
             for p in psfs64]
    with mvd.Deconvolver(views, w.psfs, "plain", path="fft") as d:
        for v in (0, 1, 2, 3, 0):
            d.iterate(1, [v])
            psi = d.result().astype(np.float64)
            tot = float(views[v].astype(np.float64).sum())
            assert abs(psi.sum() - tot) < 1e-5 * tot, (v, psi.sum(), tot)
    with mvd.Deconvolver(w.views, w.psfs, "efficient", path="fft") as d:
        d.iterate(2)
        assert d.result().min() >= d.eps * (1 - 1e-7)


def test_mid_volume_fixed_point(mvd):
    """Noise-free views phi_v = psi* * P_v: psi* is a fixed point of every update."""
    w = synth.config2()
    truth = w.truth.astype(np.float64) + 1.0
    psfs64 = [p.astype(np.float64) / p.astype(np.float64).sum() for p in w.psfs]
    views = [synth.workloads.blur_circular(truth, p).astype(np.float32) for p in psfs64]
    with mvd.Deconvolver(views, w.psfs, "efficient", path="fft") as d:
        d.set_estimate(truth.astype(np.float32))
        d.iterate(2)
        psi = d.result().astype(np.float64)
    assert rel_err(psi, truth) < 1e-4, err_report(psi, truth)


# ---------------------------------------------------------------------------
# misuse through the ABI
# ---------------------------------------------------------------------------

def test_state_and_argument_errors(mvd):
    w = synth.small_case(3, dims=(12, 12, 12), n_views=2)
    ctx = mvd.mvd_create(w.views, w.psfs)
    try:
        with pytest.raises(mvd.MvdError) as ei:
            mvd.mvd_iterate(ctx, 1)
        assert ei.value.status == mvd.MVD_ERR_STATE
        mvd.mvd_precompute_kernels(ctx, "efficient")
        with pytest.raises(mvd.MvdError) as ei:
            mvd.mvd_iterate(ctx, 1, [0, 5])
        assert ei.value.status == mvd.MVD_ERR_ARG
        with pytest.raises(mvd.MvdError) as ei:
            mvd.mvd_set_estimate(ctx, -np.ones(w.truth.shape, np.float32))
        assert ei.value.status == mvd.MVD_ERR_ARG
        with pytest.raises(mvd.MvdError) as ei:
            mvd.mvd_result(ctx, np.empty(10, np.float32))
        assert ei.value.status == mvd.MVD_ERR_SHAPE
        mvd.mvd_iterate(ctx, 1)
        mvd.mvd_synchronize(ctx)
    finally:
        mvd.mvd_destroy(ctx)
    bad = [v.copy() for v in w.views]
    bad[1][0, 0, 0] = -1.0
    with pytest.raises(mvd.MvdError) as ei:
        mvd.mvd_create(bad, w.psfs)
    assert ei.value.status == mvd.MVD_ERR_ARG


def test_device_views_and_stream(mvd):
    import torch

    w = synth.small_case(4, dims=(20, 16, 12), n_views=2)
    want, _ = oracle.deconvolve(w.views, w.psfs, 3, "efficient")
    s = torch.cuda.Stream()
    dv = [torch.from_numpy(v).cuda() for v in w.views]
    torch.cuda.synchronize()
    with mvd.Deconvolver(dv, w.psfs, "efficient", stream=s, path="fft") as d:
        d.iterate(3)
        got = d.result().astype(np.float64)
    assert rel_err(got, want) < PARITY_TOL, err_report(got, want)


# ---------------------------------------------------------------------------
# every power-of-two length of the register-resident passes, on each axis,
# with the generic passes forced as a second engine
# ---------------------------------------------------------------------------

POW2_CASES = [(16, 16, 16), (32, 64, 128), (256, 16, 32), (64, 512, 16), (16, 32, 1024), (2048, 16, 16),
              (16, 2048, 16), (16, 16, 2048), (48, 128, 96)]


@pytest.mark.parametrize("engine", ["fast", "generic"])
@pytest.mark.parametrize("dims", POW2_CASES)
def test_fft_lengths(mvd, monkeypatch, dims, engine):
    if engine == "generic":
        monkeypatch.setenv("MVD_FFT_GENERIC", "1")
    w = synth.small_case(200 + sum(dims), dims=dims, n_views=2, boxes=[(3, 5, 3), (5, 3, 7)], n_iter=2,
                         asymmetric=True)
    want, _ = oracle.deconvolve(w.views, w.psfs, 2, "efficient")
    got, used, _ = _run_gpu(mvd, w, path="fft", n_iter=2)
    assert used == "fft"
    assert rel_err(got, want) < PARITY_TOL, err_report(got, want)


# Mixed lengths whose plans take every radix of the generic passes: 2, 3, 4,
# 5, 8 and the composite 6 and 9 (both precisions) and 10 (FP32 only), on
# every axis, in both precisions.
MIXED_CASES = [(6, 9, 10), (12, 18, 20), (27, 30, 36), (45, 50, 54), (60, 81, 20), (100, 40, 15), (270, 8, 6),
               (8, 150, 12), (10, 12, 180)]


@pytest.mark.parametrize("precision", ["precise", "fast"])
@pytest.mark.parametrize("dims", MIXED_CASES)
def test_mixed_radix_lengths(mvd, dims, precision):
    w = synth.small_case(300 + sum(dims), dims=dims, n_views=2, boxes=[(3, 5, 3), (5, 3, 5)], n_iter=2,
                         asymmetric=True)
    want, _ = oracle.deconvolve(w.views, w.psfs, 2, "efficient")
    with mvd.Deconvolver(w.views, w.psfs, "efficient", path="fft", precision=precision) as d:
        d.iterate(2)
        got = d.result()
    assert rel_err(got, want) < PARITY_TOL, err_report(got, want)


def test_graph_replay_matches_plain_launches(mvd, monkeypatch):
    """On a non-default stream one iteration is captured as a CUDA graph and replayed; the
    result must equal the one-by-one launches bit for bit, and match the oracle."""
    import torch

    w = synth.small_case(41, dims=(64, 48, 32), n_views=3, boxes=[(7, 5, 9), (5, 9, 7), (9, 7, 5)], n_iter=3,
                         asymmetric=True)
    want, _ = oracle.deconvolve(w.views, w.psfs, 3, "efficient", schedule=[2, 0, 1])
    out = {}
    for mode in ("graph", "plain"):
        if mode == "plain":
            monkeypatch.setenv("MVD_NO_GRAPH", "1")
        s = torch.cuda.Stream()
        for path in ("fft", "direct"):
            with mvd.Deconvolver(w.views, w.psfs, "efficient", stream=s, path=path) as d:
                d.iterate(2, [2, 0, 1])
                d.iterate(1, [2, 0, 1])
                out[mode, path] = d.result()
    for path in ("fft", "direct"):
        assert np.array_equal(out["graph", path], out["plain", path]), path
        assert rel_err(out["graph", path], want) < PARITY_TOL, err_report(out["graph", path], want)


def test_mid_volume_full_run_against_stored_oracle(mvd, cfg2):
    """256x256x128, 4 views, 20 iterations, compared with the FP64 oracle's final estimate at
    4096 seeded voxels (tests/golden/oracle_samples_mid.txt, written by
    tests/golden/make_oracle_samples.py from the oracle alone)."""
    from tests.golden.make_oracle_samples import input_digest, read

    digest, eps, max_abs, idx, want = read("mid")
    w = cfg2
    assert input_digest(w) == digest, "the input generator produced different inputs on this machine"
    got, used, geps = _run_gpu(mvd, w, path="fft")
    assert abs(geps - eps) <= 1e-6 * eps
    g = got.ravel()[idx]
    tau = 1e-3 * max_abs
    err = float(np.max(np.abs(g - want) / np.maximum(np.abs(want), tau)))
    assert err < PARITY_TOL, f"max rel err {err:.3e} at sampled voxels"


def test_fast_fp32_mode(mvd):
    """MVD_FAST (everything in FP32): few iterations stay at 1e-4; the documented cost of FP32
    is slow growth of dim-voxel error with the iteration count."""
    w = synth.small_case(61, dims=(48, 40, 36), n_views=3, boxes=[(7, 5, 9), (9, 7, 5), (5, 9, 7)], n_iter=2,
                         asymmetric=True)
    want, _ = oracle.deconvolve(w.views, w.psfs, 2, "efficient")
    with mvd.Deconvolver(w.views, w.psfs, "efficient", path="fft", precision="fast") as d:
        d.iterate(2)
        got = d.result()
    assert rel_err(got, want) < PARITY_TOL, err_report(got, want)


def test_mixed_precision_mode(mvd):
    """MVD_MIXED (double-float forward blur, FP32 back-projection): not held to 1e-4 (its FP32
    rounding of a large r - 1 spreads over the volume; up to 4e-4 measured after 15
    iterations); held here to 1e-3, and it must differ from the precise path."""
    w = synth.small_case(61, dims=(48, 40, 36), n_views=3, boxes=[(7, 5, 9), (9, 7, 5), (5, 9, 7)], n_iter=4,
                         asymmetric=True)
    want, _ = oracle.deconvolve(w.views, w.psfs, 4, "efficient")
    out = {}
    for prec in ("mixed", "precise"):
        with mvd.Deconvolver(w.views, w.psfs, "efficient", path="fft", precision=prec) as d:
            d.iterate(4)
            out[prec] = d.result()
    assert rel_err(out["mixed"], want) < 1e-3, err_report(out["mixed"], want)
    assert rel_err(out["precise"], want) < PARITY_TOL, err_report(out["precise"], want)
    assert not np.array_equal(out["mixed"], out["precise"])


# ---------------------------------------------------------------------------
# concurrency and extreme shapes
# ---------------------------------------------------------------------------

def test_two_contexts_on_two_streams_run_concurrently(mvd):
    """Two problems enqueued on two streams at once give the same results as alone (no shared
    mutable state between contexts)."""
    import torch

    wa = synth.small_case(61, dims=(40, 32, 24), n_views=3, n_iter=4, asymmetric=True)
    wb = synth.config1()
    alone = []
    for w in (wa, wb):
        with mvd.Deconvolver(w.views, w.psfs, "efficient", path="fft") as d:
            d.iterate(w.n_iter)
            alone.append(d.result())
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    with mvd.Deconvolver(wa.views, wa.psfs, "efficient", path="fft", stream=sa) as da, \
            mvd.Deconvolver(wb.views, wb.psfs, "efficient", path="fft", stream=sb) as db:
        for i in range(max(wa.n_iter, wb.n_iter)):  # interleaved, one iteration at a time
            if i < wa.n_iter:
                da.iterate(1)
            if i < wb.n_iter:
                db.iterate(1)
        ra, rb = da.result(), db.result()
    assert rel_err(ra, alone[0]) < 1e-6 and rel_err(rb, alone[1]) < 1e-6


@pytest.mark.parametrize("path", ["direct", "fft"])
def test_psf_box_as_large_as_the_volume(mvd, path):
    """PSF boxes spanning the whole (odd) grid: every offset wraps around the periodic volume."""
    w = synth.small_case(62, dims=(15, 9, 25), n_views=2, boxes=[(15, 9, 25), (15, 9, 25)], n_iter=3)
    want, _ = oracle.deconvolve(w.views, w.psfs, w.n_iter, "efficient")
    got, _, _ = _run_gpu(mvd, w, path=path)
    assert rel_err(got, want) < PARITY_TOL, err_report(got, want)
