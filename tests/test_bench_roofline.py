"""The benchmark's roofline record (no GPU): the dominant kernel is the one with the largest
share of the step's event time; `achieved` is its algorithmic bytes per launch over its mean
launch time, `frac` that over the measured peak; `traffic`, `dram_frac` and `alu_frac` come
from the committed ncu summary (profiles/traffic.json) for the headline grid; the update's
effective fraction counts 12 bytes per voxel-view."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

DIMS = (1024, 1024, 512)
PEAK = 6746.6


def _prof():
    # kernel -> (launches, total ms) of a step of 70 view updates
    return {"dd_x_forward": (70, 70 * 1.942), "dd_y": (280, 280 * 1.675), "dd_z_mul": (140, 140 * 3.496),
            "dd_x_ratio": (70, 70 * 3.326), "x_update": (70, 70 * 2.416)}


def test_algorithmic_bytes_of_the_passes():
    X, Y, Z = DIMS
    kb = bench._kernel_bytes(X, Y, Z)
    spec = 8 * (X // 2 + 1) * Y * Z
    M = X * Y * Z
    assert kb["dd_z_mul"] == 6 * spec                  # S2 and a kernel spectrum in, S2 out (16 B each)
    assert kb["dd_y"] == pytest.approx(3.75 * spec)    # three double-float launches, one FP32 in
    assert kb["dd_x_ratio"] == 3 * spec + 4 * M
    assert kb["x_update"] == 2 * spec + 8 * M
    assert kb["dd_x_forward"] == 4 * M + 2 * spec


def test_roofline_record_of_the_dominant_kernel():
    X, Y, Z = DIMS
    prof = _prof()
    kernels = bench._kernel_table(prof, bench._kernel_bytes(X, Y, Z), PEAK)
    alu = bench._alu_peak_tops()
    units = X * Y * Z * 7 * 10
    ms_step = sum(ms for (_, ms) in prof.values())
    roof = bench._roofline(prof, kernels, DIMS, PEAK, "measured", alu, units, ms_step)
    assert roof["kernel"] == "dd_z_mul" and roof["bound"] == "hbm" and roof["unit"] == "GB/s"
    avg_s = 3.496e-3
    achieved = bench._kernel_bytes(X, Y, Z)["dd_z_mul"] / avg_s / 1e9
    assert roof["achieved"] == pytest.approx(achieved)
    assert roof["frac"] == pytest.approx(achieved / PEAK)
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
        rec = json.load(fh)["dd_z_mul@1024x1024x512"]
    assert roof["traffic"] == int(rec["dram_bytes"])
    assert roof["dram_frac"] == pytest.approx(rec["dram_bytes"] / avg_s / 1e9 / PEAK)
    assert roof["alu_frac"] == pytest.approx(rec["fp32_inst"] / avg_s / 1e12 / alu)
    # the ncu bytes of the committed capture are the algorithmic bytes within 2%
    assert rec["dram_bytes"] == pytest.approx(bench._kernel_bytes(X, Y, Z)["dd_z_mul"], rel=0.02)
    assert roof["update_effective_frac"] == pytest.approx(12.0 * units / (ms_step * 1e-3) / 1e9 / PEAK)


def test_traffic_summary_covers_every_pass_of_the_headline_grid():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
        tr = json.load(fh)
    kb = bench._kernel_bytes(*DIMS)
    for name, bytes_alg in kb.items():
        rec = tr[f"{name}@{DIMS[0]}x{DIMS[1]}x{DIMS[2]}"]
        assert rec["dram_bytes"] == pytest.approx(bytes_alg, rel=0.02), name
        assert rec["fp32_inst"] > 0 and rec["source"]
