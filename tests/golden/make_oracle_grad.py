"""Writes stored FP64-oracle gradients of the unrolled deconvolution on the
128x128x96 four-view workload (8 iterations, loss = mean squared error to the
seeded ground truth), too slow to repeat inside the GPU tests.

Calls only the oracle (oracle/) and the seeded input generator (synth/).
PSFs are the Gaussian model at the initial per-view (sigma_xy, sigma_ax),
20 % off the true values. Recorded: a checksum of the inputs, the loss, the
sigma gradients twice over (the oracle's reverse-mode gradient chained through
the Gaussian model by FP64 central differences of the model, and FP64 central
differences of the whole oracle run with step 1e-4), the view gradients at a
seeded sample of voxels and the raw-PSF gradients at a seeded sample of taps.

Usage: python tests/golden/make_oracle_grad.py
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
from synth.workloads import config5_sigmas, gaussian_psf  # noqa: E402

PATH = os.path.join(HERE, "oracle_grad_unrolled_128x128x96.txt")
N_VOX = 2048
N_TAPS = 256
FD_STEP = 1e-4
MODEL_STEP = 1e-6


def model_psfs(w, sigmas):
    return [gaussian_psf(s[0], s[1], w.meta["box"], "z", a) for s, a in zip(sigmas, w.meta["angles"])]


def input_digest(w, psfs) -> str:
    h = hashlib.sha256()
    for v in w.views:
        h.update(np.ascontiguousarray(v, dtype=np.float32).tobytes())
    h.update(np.ascontiguousarray(w.truth, dtype=np.float32).tobytes())
    for p in psfs:
        h.update(np.ascontiguousarray(p, dtype=np.float32).tobytes())
    return h.hexdigest()


def samples(n: int, k: int, seed: int) -> np.ndarray:
    return np.sort(np.random.default_rng(seed).choice(n, min(k, n), replace=False))


def sigma_chain(w, sigmas, grad_psfs):
    """dL/dsigma from dL/dPSF through the Gaussian model (central differences of the model)."""
    out = np.zeros((len(sigmas), 2))
    for v, s in enumerate(sigmas):
        for k in range(2):
            sp, sm = list(s), list(s)
            sp[k] += MODEL_STEP
            sm[k] -= MODEL_STEP
            a = w.meta["angles"][v]
            dP = (gaussian_psf(sp[0], sp[1], w.meta["box"], "z", a)
                  - gaussian_psf(sm[0], sm[1], w.meta["box"], "z", a)) / (2 * MODEL_STEP)
            out[v, k] = float(np.sum(grad_psfs[v] * dP))
    return out


def sigma_fd(w, sigmas, truth64):
    def loss(sig):
        psi, _ = oracle.deconvolve(w.views, model_psfs(w, sig), w.n_iter)
        return float(np.mean((psi - truth64) ** 2))

    out = np.zeros((len(sigmas), 2))
    for v in range(len(sigmas)):
        for k in range(2):
            sp = [list(s) for s in sigmas]
            sm = [list(s) for s in sigmas]
            sp[v][k] += FD_STEP
            sm[v][k] -= FD_STEP
            out[v, k] = (loss(sp) - loss(sm)) / (2 * FD_STEP)
    return out


def write(w):
    sig = config5_sigmas(w.n_views)
    psfs = model_psfs(w, sig)
    t0 = time.time()
    loss, gv, gp, _ = oracle.unrolled_grad(w.views, psfs, w.n_iter, w.truth)
    t_adj = time.time() - t0
    chain = sigma_chain(w, sig, gp)
    t0 = time.time()
    fd = sigma_fd(w, sig, w.truth.astype(np.float64))
    t_fd = time.time() - t0
    with open(PATH, "w") as fh:
        fh.write(f"# FP64 oracle gradients, {w.n_iter} unrolled iterations on workload {w.name}\n")
        fh.write(f"# written by tests/golden/make_oracle_grad.py; reverse mode {t_adj:.0f} s, finite differences "
                 f"{t_fd:.0f} s on {oracle.num_threads()} threads\n")
        fh.write(f"inputs_sha256 {input_digest(w, psfs)}\n")
        fh.write(f"loss {float(loss)!r}\n")
        for v in range(w.n_views):
            fh.write(f"sigma {v} {float(sig[v][0])!r} {float(sig[v][1])!r}\n")
            fh.write(f"dsigma_adjoint {v} {float(chain[v, 0])!r} {float(chain[v, 1])!r}\n")
            fh.write(f"dsigma_fd {v} {float(fd[v, 0])!r} {float(fd[v, 1])!r}\n")
            fh.write(f"max_abs_dview {v} {float(np.abs(gv[v]).max())!r}\n")
            fh.write(f"max_abs_dpsf {v} {float(np.abs(gp[v]).max())!r}\n")
            for i in samples(gv[v].size, N_VOX, 100 + v):
                fh.write(f"dview {v} {int(i)} {float(gv[v].ravel()[i])!r}\n")
            for i in samples(gp[v].size, N_TAPS, 200 + v):
                fh.write(f"dpsf {v} {int(i)} {float(gp[v].ravel()[i])!r}\n")
    print(PATH, t_adj, t_fd)


def read():
    """Returns a dict: digest, loss, sigma/dsigma_adjoint/dsigma_fd (N x 2), max_abs_dview/max_abs_dpsf (N),
    dview/dpsf (per view: indices, values)."""
    out = {"sigma": {}, "dsigma_adjoint": {}, "dsigma_fd": {}, "max_abs_dview": {}, "max_abs_dpsf": {},
           "dview": {}, "dpsf": {}}
    with open(PATH) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            f = line.split()
            if f[0] == "inputs_sha256":
                out["digest"] = f[1]
            elif f[0] == "loss":
                out["loss"] = float(f[1])
            elif f[0] in ("sigma", "dsigma_adjoint", "dsigma_fd"):
                out[f[0]][int(f[1])] = (float(f[2]), float(f[3]))
            elif f[0] in ("max_abs_dview", "max_abs_dpsf"):
                out[f[0]][int(f[1])] = float(f[2])
            else:
                out[f[0]].setdefault(int(f[1]), []).append((int(f[2]), float(f[3])))
    n = len(out["sigma"])
    for k in ("sigma", "dsigma_adjoint", "dsigma_fd"):
        out[k] = np.array([out[k][v] for v in range(n)])
    for k in ("max_abs_dview", "max_abs_dpsf"):
        out[k] = np.array([out[k][v] for v in range(n)])
    for k in ("dview", "dpsf"):
        out[k] = {v: (np.array([a for a, _ in out[k][v]]), np.array([b for _, b in out[k][v]])) for v in range(n)}
    return out


if __name__ == "__main__":
    write(synth.config5())
