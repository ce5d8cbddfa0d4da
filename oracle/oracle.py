"""ctypes front end of the FP64 C oracle (``mvd_oracle.c``).

TEST INFRASTRUCTURE ONLY (see the package docstring). Every function takes and
returns float64 numpy arrays shaped ``[z][y][x]`` (kernels ``[Kz][Ky][Kx]``);
the C file states which equation of the paper each step follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

PLAIN, EFFICIENT, OPT1, OPT2 = 0, 1, 2, 3
VARIANTS = {"plain": PLAIN, "efficient": EFFICIENT, "opt1": OPT1, "opt2": OPT2}

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mvd_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libmvd_oracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O3, OpenMP) if the library is missing or stale."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O3", "-fPIC", "-shared", "-fopenmp", "-std=c11", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.mvdo_conv.argtypes = [_D, _I, _D, _I, _D]
            lib.mvdo_mirror.argtypes = [_D, _I, _D]
            lib.mvdo_kconv.argtypes = [_D, _I, _D, _I, _D, _I]
            lib.mvdo_compound.argtypes = [ctypes.c_int, ctypes.POINTER(_D), _I, ctypes.c_int,
                                          ctypes.c_int, _D]
            lib.mvdo_compound.restype = ctypes.c_int
            lib.mvdo_update.argtypes = [_D, _D, _D, _I, _D, _I, _I, ctypes.c_double, _D, _D, _D]
            lib.mvdo_mean_views.argtypes = [ctypes.c_int, ctypes.POINTER(_D), _I]
            lib.mvdo_mean_views.restype = ctypes.c_double
            lib.mvdo_deconvolve.argtypes = [ctypes.c_int, ctypes.POINTER(_D), ctypes.POINTER(_D), _I,
                                            _I, ctypes.c_int, ctypes.c_int, _I, ctypes.c_int,
                                            ctypes.c_double, ctypes.c_int, _D]
            lib.mvdo_deconvolve.restype = ctypes.c_double
            lib.mvdo_deconvolve_combined.argtypes = [ctypes.c_int, ctypes.POINTER(_D), ctypes.POINTER(_D), _I, _I,
                                                     ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                                     ctypes.c_int, _D]
            lib.mvdo_deconvolve_combined.restype = ctypes.c_double
            lib.mvdo_deconvolve_combined_bounded.argtypes = [ctypes.c_int, ctypes.POINTER(_D),
                                                             ctypes.POINTER(_D), _I, _I, ctypes.c_int,
                                                             ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                             ctypes.c_double, ctypes.c_int, _D]
            lib.mvdo_deconvolve_combined_bounded.restype = ctypes.c_double
            lib.mvdo_normalize_weights.argtypes = [ctypes.c_int, ctypes.POINTER(_D), _I, ctypes.c_int,
                                                   ctypes.c_double, ctypes.POINTER(_D)]
            lib.mvdo_normalize_weights.restype = ctypes.c_double
            lib.mvdo_deconvolve_weighted.argtypes = [ctypes.c_int, ctypes.POINTER(_D), ctypes.POINTER(_D), _I, _I,
                                                     ctypes.c_int, ctypes.c_int, ctypes.POINTER(_D),
                                                     ctypes.c_double, ctypes.c_double, ctypes.c_int, _D]
            lib.mvdo_deconvolve_weighted.restype = ctypes.c_double
            lib.mvdo_conv_zero.argtypes = [_D, _I, _D, _I, _D]
            lib.mvdo_deconvolve_zero.argtypes = [ctypes.c_int, ctypes.POINTER(_D), ctypes.POINTER(_D), _I, _I,
                                                 ctypes.c_int, ctypes.c_int, ctypes.POINTER(_D), ctypes.c_double,
                                                 ctypes.c_double, ctypes.c_int, _D]
            lib.mvdo_deconvolve_zero.restype = ctypes.c_double
            lib.mvdo_conv_mirror.argtypes = [_D, _I, _D, _I, _D]
            lib.mvdo_backproject_mirror.argtypes = [_D, _I, _D, _I, _D]
            lib.mvdo_deconvolve_mirror.argtypes = [ctypes.c_int, ctypes.POINTER(_D), ctypes.POINTER(_D), _I, _I,
                                                   ctypes.c_int, ctypes.c_int, ctypes.POINTER(_D), ctypes.c_double,
                                                   ctypes.c_double, ctypes.c_int, _D]
            lib.mvdo_deconvolve_mirror.restype = ctypes.c_double
            lib.mvdo_update_at.argtypes = [_D, _D, _D, _I, _D, _I, _I, ctypes.c_double,
                                           ctypes.POINTER(ctypes.c_long), ctypes.c_int, _D]
            lib.mvdo_num_threads.restype = ctypes.c_int
            lib.mvdo_unrolled_grad.argtypes = [ctypes.c_int, ctypes.POINTER(_D), ctypes.POINTER(_D), _I, _I,
                                               ctypes.c_int, ctypes.c_int, _D, ctypes.POINTER(_D),
                                               ctypes.POINTER(_D), _D]
            lib.mvdo_unrolled_grad.restype = ctypes.c_double
            _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _dims_xyz(a: np.ndarray):
    z, y, x = a.shape
    return (ctypes.c_int * 3)(x, y, z)


def num_threads() -> int:
    """Number of OpenMP threads the oracle runs on."""
    return int(_load().mvdo_num_threads())


def conv(vol, k) -> np.ndarray:
    """Periodic convolution ``(vol * k)(x) = sum_d k(d) vol((x-d) mod dims)`` (Eq. 51's ``*``)."""
    vol, k = _f64(vol), _f64(k)
    out = np.empty_like(vol)
    _load().mvdo_conv(_dptr(vol), _dims_xyz(vol), _dptr(k), _dims_xyz(k), _dptr(out))
    return out


def conv_zero(vol, k) -> np.ndarray:
    """Convolution with a zero boundary: ``sum_d k(d) vol(x-d)``, terms outside the grid dropped."""
    vol, k = _f64(vol), _f64(k)
    out = np.empty_like(vol)
    _load().mvdo_conv_zero(_dptr(vol), _dims_xyz(vol), _dptr(k), _dims_xyz(k), _dptr(out))
    return out


def conv_mirror(vol, k) -> np.ndarray:
    """Convolution with a mirror boundary: ``sum_d k(d) vol(reflect(x-d))``, half-sample symmetric reflection."""
    vol, k = _f64(vol), _f64(k)
    out = np.empty_like(vol)
    _load().mvdo_conv_mirror(_dptr(vol), _dims_xyz(vol), _dptr(k), _dims_xyz(k), _dptr(out))
    return out


def backproject_mirror(r, k) -> np.ndarray:
    """Mirror-boundary back-projection ``out(j) = sum_i r(i) sum_{e: reflect(i+e)=j} k(e)``."""
    r, k = _f64(r), _f64(k)
    out = np.empty_like(r)
    _load().mvdo_backproject_mirror(_dptr(r), _dims_xyz(r), _dptr(k), _dims_xyz(k), _dptr(out))
    return out


def mirror(k) -> np.ndarray:
    """Mirrored kernel ``P^*(d) = P(-d)`` (Suppl. Note "Integrating xi and x")."""
    k = _f64(k)
    out = np.empty_like(k)
    _load().mvdo_mirror(_dptr(k), _dims_xyz(k), _dptr(out))
    return out


def kconv(a, b, out_shape_zyx) -> np.ndarray:
    """Linear convolution of two small kernels evaluated on a centred box."""
    a, b = _f64(a), _f64(b)
    out = np.empty(out_shape_zyx, dtype=np.float64)
    _load().mvdo_kconv(_dptr(a), _dims_xyz(a), _dptr(b), _dims_xyz(b), _dptr(out), _dims_xyz(out))
    return out


def _psf_arrays(psfs):
    ps = [_f64(p) for p in psfs]
    arr = (_D * len(ps))(*[_dptr(p) for p in ps])
    pd = (ctypes.c_int * (3 * len(ps)))(*[d for p in ps for d in (p.shape[2], p.shape[1], p.shape[0])])
    return ps, arr, pd


def compound(psfs, v: int, variant="efficient") -> np.ndarray:
    """Back-projection kernel of view ``v`` (Eq. 222 / Eq. 230 / Eq. 240 / Eq. 51), sum 1."""
    var = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    ps, arr, pd = _psf_arrays(psfs)
    out = np.empty_like(ps[v])
    rc = _load().mvdo_compound(len(ps), arr, pd, v, var, _dptr(out))
    if rc != 0:
        raise ValueError("compound kernel sums to zero")
    return out


def update(psi, phi, P, K, eps, intermediates=False):
    """One view update (Eq. 15 with back-projection kernel K); returns the new psi.

    With ``intermediates`` also returns ``(b, r, c)``.
    """
    psi = _f64(psi).copy()
    phi, P, K = _f64(phi), _f64(P), _f64(K)
    b, r, c = (np.empty_like(psi) for _ in range(3))
    _load().mvdo_update(_dptr(psi), _dptr(phi), _dptr(P), _dims_xyz(P), _dptr(K), _dims_xyz(K),
                        _dims_xyz(psi), float(eps), _dptr(b), _dptr(r), _dptr(c))
    if intermediates:
        return psi, (b, r, c)
    return psi


def update_at(psi, phi, P, K, eps, flat_indices) -> np.ndarray:
    """One view update evaluated only at the given flat voxel indices."""
    psi, phi, P, K = _f64(psi), _f64(phi), _f64(P), _f64(K)
    idx = np.ascontiguousarray(flat_indices, dtype=np.int64)
    out = np.empty(idx.shape[0], dtype=np.float64)
    _load().mvdo_update_at(_dptr(psi), _dptr(phi), _dptr(P), _dims_xyz(P), _dptr(K), _dims_xyz(K),
                           _dims_xyz(psi), float(eps), idx.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                           int(idx.shape[0]), _dptr(out))
    return out


def mean_views(views) -> float:
    """Flat initial estimate's value: mean over all voxels of all views."""
    vs = [_f64(v) for v in views]
    arr = (_D * len(vs))(*[_dptr(v) for v in vs])
    return float(_load().mvdo_mean_views(len(vs), arr, _dims_xyz(vs[0])))


def deconvolve(views, psfs, n_iter, variant="efficient", schedule=None, eps=0.0, psi_init=None):
    """Sequential (OSEM-order) efficient Bayesian deconvolution in FP64.

    Returns ``(psi, eps_used)``. ``eps <= 0`` selects ``1e-4 * psi0``.
    """
    var = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    vs = [_f64(v) for v in views]
    ps, parr, pd = _psf_arrays(psfs)
    varr = (_D * len(vs))(*[_dptr(v) for v in vs])
    if psi_init is None:
        psi = np.empty_like(vs[0])
        init = 0
    else:
        psi = _f64(psi_init).copy()
        init = 1
    if schedule is None:
        sched, slen = None, 0
    else:
        sched = (ctypes.c_int * len(schedule))(*[int(s) for s in schedule])
        slen = len(schedule)
    used = _load().mvdo_deconvolve(len(vs), varr, parr, pd, _dims_xyz(vs[0]), var, int(n_iter), sched,
                                   slen, float(eps), init, _dptr(psi))
    if used < 0:
        raise ValueError("oracle deconvolution failed (compound kernel sums to zero)")
    return psi, used


def deconvolve_combined(views, psfs, n_iter, variant="efficient", root=True, eps=0.0, psi_init=None,
                        boundary="periodic"):
    """Combined (simultaneous) update, Eq. 50 / Eq. 220: every view's factor from the same psi,
    their product (or with ``root`` its |V|-th root, the geometric mean) applied at once.
    ``boundary``: "periodic", or "zero" / "mirror" (factors c_v / s_v, as in deconvolve_zero
    and deconvolve_mirror).

    Returns ``(psi, eps_used)``; ``eps <= 0`` selects ``1e-4 * psi0``.
    """
    var = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    vs = [_f64(v) for v in views]
    ps, parr, pd = _psf_arrays(psfs)
    varr = (_D * len(vs))(*[_dptr(v) for v in vs])
    if psi_init is None:
        psi, init = np.empty_like(vs[0]), 0
    else:
        psi, init = _f64(psi_init).copy(), 1
    if boundary == "periodic":
        used = _load().mvdo_deconvolve_combined(len(vs), varr, parr, pd, _dims_xyz(vs[0]), var, int(n_iter),
                                                1 if root else 0, float(eps), init, _dptr(psi))
    else:
        used = _load().mvdo_deconvolve_combined_bounded(len(vs), varr, parr, pd, _dims_xyz(vs[0]), var,
                                                        int(n_iter), 1 if root else 0,
                                                        {"zero": 1, "mirror": 2}[boundary], float(eps), init,
                                                        _dptr(psi))
    if used < 0:
        raise ValueError("oracle deconvolution failed (compound kernel sums to zero)")
    return psi, used


WEIGHT_NORMS = {"sum1": 0, "min_overlap": 1, "avg_overlap": 2, "user": 3}


def normalize_weights(weights, norm="sum1", value=0.0):
    """Per-voxel normalisation of view weights (Suppl. Note "Partially overlapping datasets"):
    scale by min(1, T / sum_v w_v). Returns ``(normalised weights, T)``."""
    ws = [_f64(w) for w in weights]
    out = [np.empty_like(w) for w in ws]
    n = WEIGHT_NORMS[norm] if isinstance(norm, str) else int(norm)
    T = _load().mvdo_normalize_weights(len(ws), (_D * len(ws))(*[_dptr(w) for w in ws]), _dims_xyz(ws[0]), n,
                                       float(value), (_D * len(out))(*[_dptr(o) for o in out]))
    if T < 0:
        raise ValueError("bad weight normalisation")
    return out, T


def deconvolve_weighted(views, psfs, n_iter, weights=None, variant="efficient", eps=0.0, psi_init=None,
                        lam=0.0):
    """Sequential deconvolution where view v's update applies the fraction weights[v] (normalised;
    None = all 1) of the change, with the Tikhonov regularisation ``lam`` in Green's one-step-late
    form (factor c / (1 + lam psi)). Returns ``(psi, eps_used)``."""
    var = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    vs = [_f64(v) for v in views]
    ps, parr, pd = _psf_arrays(psfs)
    varr = (_D * len(vs))(*[_dptr(v) for v in vs])
    if weights is None:
        ws, warr = [], None
    else:
        ws = [_f64(w) for w in weights]
        warr = (_D * len(ws))(*[_dptr(w) for w in ws])
    if psi_init is None:
        psi, init = np.empty_like(vs[0]), 0
    else:
        psi, init = _f64(psi_init).copy(), 1
    used = _load().mvdo_deconvolve_weighted(len(vs), varr, parr, pd, _dims_xyz(vs[0]), var, int(n_iter), warr,
                                            float(lam), float(eps), init, _dptr(psi))
    if used < 0:
        raise ValueError("oracle deconvolution failed (compound kernel sums to zero)")
    return psi, used


def _deconvolve_bounded(fn, views, psfs, n_iter, variant, eps, psi_init, weights, lam):
    var = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    vs = [_f64(v) for v in views]
    ps, parr, pd = _psf_arrays(psfs)
    varr = (_D * len(vs))(*[_dptr(v) for v in vs])
    if weights is None:
        ws, warr = [], None
    else:
        ws = [_f64(w) for w in weights]
        warr = (_D * len(ws))(*[_dptr(w) for w in ws])
    if psi_init is None:
        psi, init = np.empty_like(vs[0]), 0
    else:
        psi, init = _f64(psi_init).copy(), 1
    used = fn(len(vs), varr, parr, pd, _dims_xyz(vs[0]), var, int(n_iter), warr, float(lam), float(eps), init,
              _dptr(psi))
    if used < 0:
        raise ValueError("oracle deconvolution failed (compound kernel sums to zero)")
    return psi, used


def deconvolve_zero(views, psfs, n_iter, variant="efficient", eps=0.0, psi_init=None, weights=None, lam=0.0):
    """Sequential deconvolution whose image convolutions use a zero boundary, optionally with
    view weights and Tikhonov ``lam`` (as in deconvolve_weighted). Returns ``(psi, eps)``."""
    return _deconvolve_bounded(_load().mvdo_deconvolve_zero, views, psfs, n_iter, variant, eps, psi_init, weights,
                               lam)


def deconvolve_mirror(views, psfs, n_iter, variant="efficient", eps=0.0, psi_init=None, weights=None, lam=0.0):
    """Sequential deconvolution whose image convolutions use a mirror boundary, optionally with
    view weights and Tikhonov ``lam``. Returns ``(psi, eps)``."""
    return _deconvolve_bounded(_load().mvdo_deconvolve_mirror, views, psfs, n_iter, variant, eps, psi_init, weights,
                               lam)


def unrolled_grad(views, psfs, n_iter, truth, variant="efficient"):
    """Loss mean((psi_K - truth)^2) of n_iter iterations from the flat start and its
    gradients with respect to every view and every raw PSF (reverse mode, FP64).

    Returns ``(loss, grad_views, grad_psfs, psi_K)``.
    """
    var = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    vs = [_f64(v) for v in views]
    ps, parr, pd = _psf_arrays(psfs)
    varr = (_D * len(vs))(*[_dptr(v) for v in vs])
    t = _f64(truth)
    gv = [np.empty_like(v) for v in vs]
    gp = [np.empty_like(p) for p in ps]
    psik = np.empty_like(vs[0])
    loss = _load().mvdo_unrolled_grad(len(vs), varr, parr, pd, _dims_xyz(vs[0]), var, int(n_iter), _dptr(t),
                                      (_D * len(gv))(*[_dptr(g) for g in gv]),
                                      (_D * len(gp))(*[_dptr(g) for g in gp]), _dptr(psik))
    return loss, gv, gp, psik


# ---------------------------------------------------------------------------
# The same sequential deconvolution with every image convolution evaluated
# through FP64 FFTs (the Convolution Theorem, Suppl. Note "Expression in
# convolution algebra": a periodic convolution is a pointwise product of
# spectra). The FFT is a library step (scipy.fft, else numpy.fft); the
# compound kernels, the flat start and the floor come from the C oracle, and
# the update is Eq. 15 with the compound kernel of Eq. 222 applied view by
# view. Rounding stays far below the 1e-4 parity bar (FP64 FFT error is about
# 1e-16 of the volume's norm), and it finishes full-size workloads in
# seconds where the direct sums take hours. Pinned against `deconvolve` in
# tests/test_oracle_fft.py.
# ---------------------------------------------------------------------------

def _fft_mod():
    try:
        import scipy.fft as sf

        workers = os.cpu_count() or 1
        return (lambda a: sf.rfftn(a, workers=workers)), (lambda s, shape: sf.irfftn(s, s=shape, workers=workers))
    except Exception:  # pragma: no cover
        return np.fft.rfftn, (lambda s, shape: np.fft.irfftn(s, s=shape))


def grid_spectrum(k, shape_zyx):
    """Spectrum of kernel ``k`` placed on the periodic grid: tap offset ``d`` at index ``d mod dims``
    (so that ``irfftn(rfftn(f) * grid_spectrum(k)) = f * k`` of Eq. 51)."""
    rfftn, _ = _fft_mod()
    k = _f64(k)
    Kz, Ky, Kx = k.shape
    big = np.zeros(shape_zyx)
    zi = (np.arange(Kz) - (Kz - 1) // 2) % shape_zyx[0]
    yi = (np.arange(Ky) - (Ky - 1) // 2) % shape_zyx[1]
    xi = (np.arange(Kx) - (Kx - 1) // 2) % shape_zyx[2]
    np.add.at(big, np.ix_(zi, yi, xi), k)  # wrapped taps add up, as in the direct sum
    return rfftn(big)


def conv_fft(vol, k) -> np.ndarray:
    """Periodic convolution ``sum_d k(d) vol((x-d) mod dims)`` through FP64 FFTs."""
    rfftn, irfftn = _fft_mod()
    vol = _f64(vol)
    return irfftn(rfftn(vol) * grid_spectrum(k, vol.shape), vol.shape)


def deconvolve_fft(views, psfs, n_iter, variant="efficient", schedule=None, eps=0.0, psi_init=None,
                   kernels=None):
    """`deconvolve` (sequential efficient Bayesian deconvolution, FP64) with the two image
    convolutions of every view update evaluated through FFTs instead of direct sums.

    Per update of view v (Eq. 15 with the back-projection kernel of Eq. 222):
    ``b = psi * P_v``, ``r = phi_v / max(b, eps)``, ``c = r * K_v``, ``psi = max(psi c, eps)``.
    PSFs are normalised to sum 1 (Eq. 3), K_v = `compound` of the normalised PSFs, psi0 is the
    mean over all views (`mean_views`), ``eps <= 0`` selects ``1e-4 psi0``. ``kernels``: the
    compound kernels `compound` returns for these PSFs and this variant, when the caller has
    them already (they depend on the PSFs only). Returns ``(psi, eps_used)``.
    """
    rfftn, irfftn = _fft_mod()
    shape = np.asarray(views[0]).shape
    pn = [_f64(p) / _f64(p).sum() for p in psfs]
    comp = [compound(pn, v, variant) for v in range(len(pn))] if kernels is None else [_f64(k) for k in kernels]
    # psi0: FP64 sum over all voxels of all views (one view converted at a time)
    psi0 = sum(float(np.sum(v, dtype=np.float64)) for v in views) / (float(np.prod(shape)) * len(views))
    if eps <= 0.0:
        eps = 1e-4 * psi0
    psi = np.full(shape, psi0) if psi_init is None else _f64(psi_init).copy()
    order = list(range(len(views))) if schedule is None else [int(s) for s in schedule]
    # kernel spectra are kept only when a view recurs (full-size volumes hold a few GB each)
    keep = int(n_iter) * len(order) > len(set(order))
    spectra = {}

    def spec(v, which):
        key = (v, which)
        if key in spectra:
            return spectra[key]
        s = grid_spectrum(pn[v] if which == 0 else comp[v], shape)
        if keep:
            spectra[key] = s
        return s

    for _ in range(int(n_iter)):
        for v in order:
            b = irfftn(rfftn(psi) * spec(v, 0), shape)
            r = _f64(views[v]) / np.maximum(b, eps)
            del b
            c = irfftn(rfftn(r) * spec(v, 1), shape)
            del r
            psi *= c
            np.maximum(psi, eps, out=psi)
            del c
    return psi, eps
