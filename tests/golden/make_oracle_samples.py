"""Writes stored FP64-oracle values for workloads whose full oracle run takes
minutes to hours (too slow to repeat inside the GPU tests).

Calls only the oracle (oracle/) and the seeded input generator (synth/). For
each workload it records a checksum of the generated inputs, then the oracle's
final estimate at a fixed seeded sample of voxels (flat index and value), so a
GPU test can regenerate the same inputs, run the CUDA path and compare the
same voxels element by element.

Usage: python tests/golden/make_oracle_samples.py mid   # 256x256x128, 20 iterations
"""
import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

N_SAMPLES = 4096


def input_digest(w) -> str:
    h = hashlib.sha256()
    for v in w.views:
        h.update(np.ascontiguousarray(v, dtype=np.float32).tobytes())
    for p in w.psfs:
        h.update(np.ascontiguousarray(p, dtype=np.float32).tobytes())
    return h.hexdigest()


def sample_indices(n_voxels: int, seed: int = 7) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n_voxels, N_SAMPLES, replace=False))


def write(name: str, w, variant: str = "efficient"):
    t0 = time.time()
    psi, eps = oracle.deconvolve(w.views, w.psfs, w.n_iter, variant)
    dt = time.time() - t0
    idx = sample_indices(w.voxels)
    path = os.path.join(HERE, f"oracle_samples_{name}.txt")
    with open(path, "w") as fh:
        fh.write(f"# FP64 oracle ({variant}, {w.n_iter} iterations) on workload {w.name}\n")
        fh.write(f"# written by tests/golden/make_oracle_samples.py {name}; oracle time {dt:.0f} s on "
                 f"{oracle.num_threads()} threads\n")
        fh.write(f"inputs_sha256 {input_digest(w)}\n")
        fh.write(f"eps {eps!r}\n")
        fh.write(f"max_abs {float(np.abs(psi).max())!r}\n")
        for i in idx:
            fh.write(f"{int(i)} {float(psi.ravel()[i])!r}\n")
    print(path, dt)


def read(name: str):
    """Returns (inputs digest, eps, max|psi|, indices, values)."""
    meta, idx, val = {}, [], []
    with open(os.path.join(HERE, f"oracle_samples_{name}.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            a, b = line.split()
            if a.isdigit():
                idx.append(int(a))
                val.append(float(b))
            else:
                meta[a] = b
    return meta["inputs_sha256"], float(meta["eps"]), float(meta["max_abs"]), np.array(idx), np.array(val)


WORKLOADS = {"mid": synth.config2}

if __name__ == "__main__":
    for name in sys.argv[1:] or ["mid"]:
        write(name, WORKLOADS[name]())
