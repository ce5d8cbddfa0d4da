"""The seeded input generators (no method arithmetic): determinism and the shapes and
statistics their recipes state."""
import numpy as np

import synth
from synth.workloads import blend_weights, time_series


def test_small_case_is_deterministic():
    a = synth.small_case(5, dims=(16, 12, 10), n_views=2)
    b = synth.small_case(5, dims=(16, 12, 10), n_views=2)
    assert all(np.array_equal(x, y) for x, y in zip(a.views, b.views))
    assert all(np.array_equal(x, y) for x, y in zip(a.psfs, b.psfs))
    assert a.views[0].shape == (10, 12, 16) and a.views[0].dtype == np.float32
    assert all(abs(float(p.sum()) - 1.0) < 1e-6 for p in a.psfs)


def test_time_series_drifts_the_object_with_the_same_psfs():
    w = synth.small_case(6, dims=(20, 16, 12), n_views=2, n_iter=2)
    s1 = time_series(w, 3, 100)
    s2 = time_series(w, 3, 100)
    assert len(s1) == 3 and all(len(t) == 2 for t in s1)
    assert all(np.array_equal(x, y) for a, b in zip(s1, s2) for x, y in zip(a, b))
    assert all(v.shape == w.views[0].shape and v.dtype == np.float32 for t in s1 for v in t)
    # later time points differ (drift and fresh noise), with the same mean photon level
    assert not np.array_equal(s1[0][0], s1[1][0])
    m0, m1 = float(s1[0][0].mean()), float(s1[1][0].mean())
    assert abs(m0 - m1) <= 0.05 * m0


def test_blend_weights_layout_and_range():
    wt = blend_weights((20, 16, 12), (0, 0, 0), (14, 16, 12), (4, 4, 4))
    assert wt.shape == (12, 16, 20)
    assert float(wt.min()) >= 0.0 and float(wt.max()) <= 1.0
    assert np.all(wt[:, :, 15:] == 0.0)  # outside the box along x
