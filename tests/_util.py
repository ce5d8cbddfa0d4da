"""Shared helpers of the test suite (no method arithmetic)."""
import numpy as np

# Parity metric: max_i |g_i - o_i| / max(|o_i|, tau), tau = 1e-3 max|o|.
# The floor keeps voxels near the clamp value (eps = 1e-4 psi0) from turning
# FP32 absolute rounding into huge relative numbers; the bar is 1e-4.
PARITY_TOL = 1e-4
FLOOR = 1e-3


def rel_err(got, want, floor=FLOOR) -> float:
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    tau = floor * np.max(np.abs(want))
    return float(np.max(np.abs(got - want) / np.maximum(np.abs(want), tau)))


def err_report(got, want) -> str:
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    d = np.abs(got - want)
    return (f"floored max rel {rel_err(got, want):.3e}, unfloored max rel "
            f"{np.max(d / np.maximum(np.abs(want), 1e-300)):.3e}, max abs {d.max():.3e}, "
            f"rms rel {np.sqrt(np.mean((d / np.maximum(np.abs(want), 1e-300)) ** 2)):.3e}")
