"""The aligned double-float arithmetic of the FFT lines (csrc/adf.cuh), compiled
for the CPU and run on Stockham transforms in the GPU lines' stage schedules,
against a direct long-double DFT (no GPU).

What it pins: the butterflies compute the DFT (a wrong constant, sign or index
gives errors of order 1, not 1e-12); the grid invariant (every high part at a
stage input at most 2^19, resp. 2^18, times the stage's quantum, which keeps
the butterfly sums exact); and the error bound the convolution relies on:
below 2^-37 (power-of-two plans) and 2^-34 (mixed plans) of L times the input
bound, for uniform, constant, spiky, eight-decade, alternating, single-tone
and low-part inputs.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1308_0730_gb300", "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    out = str(tmp_path_factory.mktemp("adf") / "adf_host_check")
    # host code only; no FMA contraction, IEEE round-to-nearest adds
    cmd = [nvcc, "-O2", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-ffp-contract=off",
           "-I", CSRC, "-I", INCLUDE, os.path.join(HERE, "native", "adf_host_check.cu"), "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return out


@pytest.mark.parametrize("mode,bound,headroom", [("pow2", 2.0 ** -37, 19), ("mixed", 2.0 ** -34, 18)])
def test_aligned_fft_against_long_double_dft(exe, mode, bound, headroom):
    r = subprocess.run([exe, mode], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    rows = [line.split() for line in r.stdout.strip().splitlines()]
    assert len(rows) >= 40
    for L, pat, err, gap in rows:
        assert float(err) < bound, f"L={L} pattern {pat}: error {float(err):.3e} of L x bound"
        assert int(gap) <= headroom, f"L={L} pattern {pat}: a stage input reached 2^{gap} q"
