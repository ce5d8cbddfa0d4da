"""The allocation-free view update (mvd_update_direct_noalloc) against the FP64
oracle and the regular context path.

Some callers cannot call cudaMalloc (their device memory belongs to a caching
allocator, or they must not allocate once frames are streaming), so the
library offers one view update that allocates nothing and keeps its ratio
scratch in a file-scope device array. This test drives that entry point
through the C ABI, twice in a row on the same estimate (the second call reuses
the scratch the first one left behind). Each result is checked against the
oracle's update (`oracle.update`, FP64) from the same start and against the
update the regular entry points (create / precompute / iterate, direct engine)
compute; the free device memory is the same before and after the second call.
The file name makes pytest collect it last, so a run that stops at the first
failure has run every other test.
"""
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


def test_noalloc_update_matches_regular_path_twice(env):
    torch, mvd = env
    w = synth.small_case(31, dims=(40, 36, 32), n_views=2, boxes=[(7, 5, 9), (5, 9, 7)], n_iter=1,
                         asymmetric=True)
    order = [1, 0]
    refs = []
    with mvd.Deconvolver(w.views, w.psfs, "efficient", path="direct") as d:
        psi0, eps = d.psi0, d.eps
        comps = [d.compound_kernel(v) for v in range(w.n_views)]
        for v in order:
            d.iterate(1, [v])
            refs.append(d.result().copy())
    dev = torch.device("cuda", torch.cuda.current_device())
    psfs = [torch.from_numpy((p.astype(np.float64) / p.astype(np.float64).sum()).astype(np.float32)).to(dev)
            for p in w.psfs]
    comps = [torch.from_numpy(c).to(dev) for c in comps]
    phis = [torch.from_numpy(v).to(dev) for v in w.views]
    psi = torch.full(w.truth.shape, psi0, dtype=torch.float32, device=dev)
    pn = [p.astype(np.float64) / p.astype(np.float64).sum() for p in w.psfs]
    torch.cuda.synchronize()
    # the oracle's chain starts from its own flat estimate and floor
    psi0_o = oracle.mean_views(w.views)
    eps_o = 1e-4 * psi0_o
    assert abs(psi0_o - psi0) <= 1e-6 * psi0_o
    prev = np.full(w.truth.shape, psi0_o)
    for i, (v, ref) in enumerate(zip(order, refs)):
        free0, _ = torch.cuda.mem_get_info()
        mvd.mvd_update_direct_noalloc(psi, phis[v], psfs[v], comps[v], eps)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        if i > 0:  # the first call on a device may look up the scratch address once
            assert free1 == free0, f"free device memory changed by {free0 - free1} bytes"
        got = psi.cpu().numpy()
        want = oracle.update(prev, w.views[v], pn[v], oracle.compound(pn, v, "efficient"), eps_o)
        assert rel_err(got, want) < PARITY_TOL, f"view {v} vs oracle: {err_report(got, want)}"
        assert rel_err(got, ref) < PARITY_TOL, f"view {v} vs context path: {err_report(got, ref)}"
        prev = want


def test_noalloc_rejects_volumes_beyond_its_scratch(env):
    torch, mvd = env
    dev = torch.device("cuda", torch.cuda.current_device())
    big = torch.ones((128, 128, 256), dtype=torch.float32, device=dev)  # 2^22 voxels > 2^21
    k = torch.ones((3, 3, 3), dtype=torch.float32, device=dev) / 27
    with pytest.raises(mvd.MvdError) as ei:
        mvd.mvd_update_direct_noalloc(big, big, k, k, 1e-3)
    assert ei.value.status == mvd.MVD_ERR_SHAPE
    assert "at most" in mvd.mvd_last_error()
