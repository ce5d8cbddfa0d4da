"""Batched form: many volumes of uneven size and view count in one launch (the
persistent kernel and the graph of per-volume branches), against per-volume
runs and the FP64 oracle."""
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
    from paper_1308_0730_gb300 import mvd

    mvd.load()
    return torch, mvd


SPECS = [  # dims, boxes (one per view)
    ((48, 40, 36), [(5, 7, 9), (9, 7, 5), (7, 5, 5)]),
    ((30, 64, 27), [(7, 5, 9), (5, 9, 7)]),
    ((24, 20, 45), [(5, 5, 11), (11, 5, 5), (5, 11, 5), (7, 7, 7)]),
    ((75, 18, 32), [(9, 5, 5), (5, 5, 9)]),
    ((16, 16, 16), [(3, 5, 7), (7, 5, 3), (5, 3, 5)]),
]


def _workloads(seed=500, n_iter=3):
    return [synth.small_case(seed + i, dims=d, n_views=len(b), boxes=b, n_iter=n_iter, asymmetric=True)
            for i, (d, b) in enumerate(SPECS)]


MODES = ["persistent", "branches"]


@pytest.mark.parametrize("mode", MODES)
def test_batch_matches_per_volume_runs_and_oracle(env, mode):
    torch, mvd = env
    ws = _workloads()
    s = torch.cuda.Stream()
    # the branch graph also takes direct-engine contexts
    paths = ["fft"] * len(ws) if mode == "persistent" else ["fft", "direct", "fft", "direct", "fft"]
    plain = []
    for w, path in zip(ws, paths):
        with mvd.Deconvolver(w.views, w.psfs, "efficient", path=path, stream=s) as d:
            d.iterate(w.n_iter)
            plain.append(d.result())
    ds = [mvd.Deconvolver(w.views, w.psfs, "efficient", path=path, stream=s) for w, path in zip(ws, paths)]
    try:
        b = mvd.mvd_batch_create(ds, ws[0].n_iter, mode)
        try:
            assert mvd.mvd_batch_mode(b) == mode
            assert mvd.mvd_batch_tasks(b) > 0
            mvd.mvd_batch_run(b)
            mvd.mvd_batch_wait(b)
            got = [d.result() for d in ds]
            # a second run continues from the current estimates
            mvd.mvd_batch_run(b)
            mvd.mvd_batch_wait(b)
            got2 = [d.result() for d in ds]
        finally:
            mvd.mvd_batch_destroy(b)
    finally:
        for d in ds:
            d.close()
    for w, g, p in zip(ws, got, plain):
        if mode == "branches":  # the same kernels as the per-volume run
            assert np.array_equal(g, p), w.name
        assert rel_err(g, p) < PARITY_TOL, f"{w.name}: {err_report(g, p)}"
    for i in (0, 3, 4):
        w = ws[i]
        want, _ = oracle.deconvolve(w.views, w.psfs, w.n_iter, "efficient")
        assert rel_err(got[i], want) < PARITY_TOL, f"{w.name}: {err_report(got[i], want)}"
        want2, _ = oracle.deconvolve(w.views, w.psfs, 2 * w.n_iter, "efficient")
        assert rel_err(got2[i], want2) < PARITY_TOL, f"{w.name} (second run): {err_report(got2[i], want2)}"


def test_batch_rejects_bad_contexts(env):
    torch, mvd = env
    ws = _workloads()[:2]
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    with mvd.Deconvolver(ws[0].views, ws[0].psfs, path="fft", stream=s1) as a, \
            mvd.Deconvolver(ws[1].views, ws[1].psfs, path="fft", stream=s2) as b, \
            mvd.Deconvolver(ws[1].views, ws[1].psfs, path="direct", stream=s1) as c:
        with pytest.raises(mvd.MvdError) as ei:
            mvd.mvd_batch_create([a, b], 1)
        assert ei.value.status == mvd.MVD_ERR_ARG
        with pytest.raises(mvd.MvdError) as ei:
            mvd.mvd_batch_create([a, c], 1, "persistent")
        assert ei.value.status == mvd.MVD_ERR_UNSUPPORTED
        with pytest.raises(mvd.MvdError) as ei:
            mvd.mvd_batch_create([a, a], 1)
        assert ei.value.status == mvd.MVD_ERR_ARG
        bc = mvd.mvd_batch_create([a, c], 1, "branches")
        mvd.mvd_batch_destroy(bc)


def test_batch_wait_times_out_and_context_stays_usable(env, monkeypatch):
    """A dependency that nothing satisfies (test hook) makes one block's bounded wait run
    out: the batch reports MVD_ERR_TIMEOUT, and the contexts keep working afterwards."""
    torch, mvd = env
    ws = _workloads()[:3]
    s = torch.cuda.Stream()
    monkeypatch.setenv("MVD_BATCH_STALL_ENTRY", "4")
    monkeypatch.setenv("MVD_BATCH_POLL_LIMIT", "20000")
    ds = [mvd.Deconvolver(w.views, w.psfs, "efficient", path="fft", stream=s) for w in ws]
    try:
        b = mvd.mvd_batch_create(ds, 1, "persistent")
        try:
            mvd.mvd_batch_run(b)
            with pytest.raises(mvd.MvdError) as ei:
                mvd.mvd_batch_wait(b)
            assert ei.value.status == mvd.MVD_ERR_TIMEOUT
        finally:
            mvd.mvd_batch_destroy(b)
        w = ws[0]
        ds[0].set_estimate(None)
        ds[0].iterate(2)
        got = ds[0].result()
        want, _ = oracle.deconvolve(w.views, w.psfs, 2, "efficient")
        assert rel_err(got, want) < PARITY_TOL
    finally:
        for d in ds:
            d.close()


@pytest.fixture(scope="module")
def cfg4_subset():
    ws = synth.config4(only=[0, 36, 19])
    return ws, [oracle.deconvolve(w.views, w.psfs, w.n_iter, "efficient")[0] for w in ws]


@pytest.mark.parametrize("mode", MODES)
def test_batched_volumes_of_the_48_volume_workload_match_oracle(env, cfg4_subset, mode):
    """Three of the 48 batched volumes (all-generic 48x60x60 with 5 views; 100x128x54 with 5
    views and 128x72x81 with 2 views, which have power-of-two axes), 15 iterations, against the
    FP64 oracle at 1e-4: per volume and inside one batch."""
    torch, mvd = env
    ws, wants = cfg4_subset
    s = torch.cuda.Stream()
    ds = [mvd.Deconvolver(w.views, w.psfs, "efficient", path="fft", stream=s) for w in ws]
    try:
        plain = []
        for d, w in zip(ds, ws):
            d.iterate(w.n_iter)
            plain.append(d.result())
            d.set_estimate(None)
        b = mvd.mvd_batch_create(ds, ws[0].n_iter, mode)
        try:
            mvd.mvd_batch_run(b)
            mvd.mvd_batch_wait(b)
        finally:
            mvd.mvd_batch_destroy(b)
        batched = [d.result() for d in ds]
    finally:
        for d in ds:
            d.close()
    for w, p, q, want in zip(ws, plain, batched, wants):
        assert rel_err(p, want) < PARITY_TOL, f"{w.name} per volume: {err_report(p, want)}"
        assert rel_err(q, want) < PARITY_TOL, f"{w.name} batched: {err_report(q, want)}"


@pytest.fixture(scope="module")
def cfg4_all():
    """All 48 volumes of the batched workload (every one has its own radix plan triple; 32
    distinct axis lengths from 48 to 320) and the oracle's FFT leg for each, 15 iterations."""
    import os

    ws = synth.config4(workers=os.cpu_count() or 1)
    return ws, [oracle.deconvolve_fft(w.views, w.psfs, w.n_iter)[0] for w in ws]


@pytest.mark.parametrize("mode", MODES)
def test_all_48_batched_volumes_every_voxel(env, cfg4_all, mode):
    """The whole 48-volume workload in one batch (15 iterations each), every voxel of every
    volume against the oracle's FFT leg (pinned to the direct sums in tests/test_oracle_fft.py),
    tau from each volume's maximum."""
    torch, mvd = env
    ws, wants = cfg4_all
    s = torch.cuda.Stream()
    ds = [mvd.Deconvolver(w.views, w.psfs, "efficient", path="fft", stream=s) for w in ws]
    try:
        b = mvd.mvd_batch_create(ds, ws[0].n_iter, mode)
        try:
            mvd.mvd_batch_run(b)
            mvd.mvd_batch_wait(b)
        finally:
            mvd.mvd_batch_destroy(b)
        got = [d.result() for d in ds]
    finally:
        for d in ds:
            d.close()
    errs = [(rel_err(g, want), w.name) for w, g, want in zip(ws, got, wants)]
    print(f"48-volume batch ({mode}): " + ", ".join(f"{n} {e:.2e}" for e, n in sorted(errs, reverse=True)[:6]))
    bad = [f"{w.name}: {err_report(g, want)}" for w, g, want in zip(ws, got, wants) if rel_err(g, want) >= PARITY_TOL]
    assert not bad, "; ".join(bad)
