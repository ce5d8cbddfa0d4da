"""Autotuner: the timed engine/tile choice, its persistence, and that a tuned
context still matches the FP64 oracle."""
import os

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


@pytest.mark.parametrize("cfg", ["blobs32", "small_odd"])
def test_tuned_context_matches_oracle_and_persists(mvd, tmp_path, cfg):
    w = synth.config1() if cfg == "blobs32" else synth.small_case(5, dims=(30, 20, 18), n_views=3, n_iter=4)
    want, _ = oracle.deconvolve(w.views, w.psfs, w.n_iter)
    cache = str(tmp_path / "tune.txt")
    with mvd.Deconvolver(w.views, w.psfs) as d:
        psi_before = d.result().copy()
        r = d.autotune(cache)
        assert not r["from_cache"] and r["ms_per_update"] > 0
        assert d.path == r["path"]
        if r["path"] == "direct":
            assert r["direct_tile_y"] in (8, 4, 2, 1)
        # timing left the estimate where it was
        assert np.array_equal(d.result(), psi_before)
        d.iterate(w.n_iter)
        got = d.result().astype(np.float64)
    err = rel_err(got, want)
    assert err < PARITY_TOL, err_report(got, want)
    lines = [ln for ln in open(cache) if ln.strip()]
    assert len(lines) == 1 and "|" in lines[0]
    with mvd.Deconvolver(w.views, w.psfs) as d:
        r2 = d.autotune(cache)
        assert r2["from_cache"] and r2["path"] == r["path"] and r2["direct_tile_y"] == r["direct_tile_y"]
    assert len([ln for ln in open(cache) if ln.strip()]) == 1


def test_auto_path_applies_cached_choice(mvd, tmp_path, monkeypatch):
    w = synth.small_case(6, dims=(32, 16, 16), n_views=2, n_iter=3)
    cache = tmp_path / "tune.txt"
    with mvd.Deconvolver(w.views, w.psfs) as d:
        d.autotune(str(cache))
    # rewrite the entry to force the other engine: AUTO must follow the cache
    key, choice = open(cache).read().strip().split("|")
    path, ty, fast, ms = choice.split()
    other = 1 if int(path) == 2 else 2
    cache.write_text(f"garbage line without a separator\n{key}| {other} 2 0 {ms}\n")
    monkeypatch.setenv("MVD_TUNE_CACHE", str(cache))
    with mvd.Deconvolver(w.views, w.psfs) as d:
        assert d.path == ("direct" if other == 1 else "fft")
        d.iterate(w.n_iter)
        got = d.result().astype(np.float64)
    want, _ = oracle.deconvolve(w.views, w.psfs, w.n_iter)
    assert rel_err(got, want) < PARITY_TOL


def test_every_direct_tile_height_gives_the_same_result(mvd, tmp_path):
    """Tile height changes only which thread computes a voxel, not the arithmetic."""
    w = synth.small_case(8, dims=(40, 24, 16), n_views=2, n_iter=2)
    outs = []
    for ty in (8, 4, 2, 1):
        cache = tmp_path / f"t{ty}.txt"
        with mvd.Deconvolver(w.views, w.psfs, path="direct") as d:
            d.autotune(str(cache))
        key = open(cache).read().split("|")[0]
        cache.write_text(f"{key}| 1 {ty} 1 1.0\n")
        with mvd.Deconvolver(w.views, w.psfs, path="direct") as d:
            r = d.autotune(str(cache))
            assert r["from_cache"] and r["direct_tile_y"] == ty
            d.iterate(w.n_iter)
            outs.append(d.result())
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
