"""Thin Python binding of libmvd.so (the C ABI in include/mvd.h).

Argument marshalling only: every step of the deconvolution runs in the
library's CUDA kernels. Host inputs are numpy float32 arrays; device inputs
are CUDA tensors (anything with ``data_ptr()``), passed as raw pointers.
There is no CPU fallback: if the library is missing, loading fails.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmvd.so")

MVD_OK, MVD_ERR_ARG, MVD_ERR_SHAPE, MVD_ERR_STATE, MVD_ERR_OOM, MVD_ERR_CUDA, MVD_ERR_TIMEOUT, \
    MVD_ERR_UNSUPPORTED = range(8)
STATUS_NAMES = ["MVD_OK", "MVD_ERR_ARG", "MVD_ERR_SHAPE", "MVD_ERR_STATE", "MVD_ERR_OOM", "MVD_ERR_CUDA",
                "MVD_ERR_TIMEOUT", "MVD_ERR_UNSUPPORTED"]
MVD_PLAIN, MVD_EFFICIENT, MVD_OPT1, MVD_OPT2 = range(4)
VARIANTS = {"plain": MVD_PLAIN, "efficient": MVD_EFFICIENT, "opt1": MVD_OPT1, "opt2": MVD_OPT2}
MVD_PATH_AUTO, MVD_PATH_DIRECT, MVD_PATH_FFT = range(3)
PATHS = {"auto": MVD_PATH_AUTO, "direct": MVD_PATH_DIRECT, "fft": MVD_PATH_FFT}

# every symbol include/mvd.h declares
EXPORTS = ["mvd_default_options", "mvd_create", "mvd_precompute_kernels", "mvd_set_estimate", "mvd_iterate",
           "mvd_result", "mvd_result_device", "mvd_synchronize", "mvd_destroy", "mvd_last_error",
           "mvd_get_eps", "mvd_get_psi0", "mvd_get_path", "mvd_get_compound_kernel", "mvd_launch_count",
           "mvd_profile_enable", "mvd_profile_read", "mvd_update_direct_noalloc", "mvd_batch_create",
           "mvd_batch_run", "mvd_batch_wait", "mvd_batch_tasks", "mvd_batch_destroy", "mvd_unrolled_forward",
           "mvd_unrolled_backward", "mvd_gaussian_psf", "mvd_gaussian_psf_vjp", "mvd_autotune",
           "mvd_batch_create_mode", "mvd_batch_mode", "mvd_iterate_combined",
           "mvd_set_weights", "mvd_get_weights", "mvd_set_regularization", "mvd_set_views", "mvd_fft_plan"]


class MvdError(RuntimeError):
    def __init__(self, status: int, message: str):
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {message}")
        self.status = status


MVD_PRECISE, MVD_FAST, MVD_MIXED = 0, 1, 2
PRECISIONS = {"precise": MVD_PRECISE, "fast": MVD_FAST, "mixed": MVD_MIXED}
MVD_BOUNDARY_PERIODIC, MVD_BOUNDARY_ZERO, MVD_BOUNDARY_MIRROR = 0, 1, 2
BOUNDARIES = {"periodic": MVD_BOUNDARY_PERIODIC, "zero": MVD_BOUNDARY_ZERO, "mirror": MVD_BOUNDARY_MIRROR}


class TuneResult(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int), ("direct_tile_y", ctypes.c_int), ("fft_engine", ctypes.c_int),
                ("from_cache", ctypes.c_int), ("ms_per_update", ctypes.c_double)]


class Options(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_float), ("path", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("views_on_device", ctypes.c_int), ("device", ctypes.c_int), ("precision", ctypes.c_int),
                ("boundary", ctypes.c_int)]


_lib = None
_FP = ctypes.POINTER(ctypes.c_float)


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads libmvd.so (built by ``paper_1308_0730_gb300.build``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    vp, ci, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
    lib.mvd_default_options.argtypes = [ctypes.POINTER(Options)]
    lib.mvd_default_options.restype = None
    lib.mvd_create.argtypes = [ctypes.POINTER(vp), ci, ctypes.POINTER(vp), ctypes.POINTER(ci),
                               ctypes.POINTER(ci), ctypes.POINTER(Options), ctypes.POINTER(vp)]
    lib.mvd_precompute_kernels.argtypes = [vp, ci]
    lib.mvd_set_estimate.argtypes = [vp, vp, ci]
    lib.mvd_iterate.argtypes = [vp, ci, ctypes.POINTER(ci), ci]
    lib.mvd_iterate_combined.argtypes = [vp, ci, ci]
    lib.mvd_iterate_combined.restype = ci
    lib.mvd_set_weights.argtypes = [vp, ctypes.POINTER(vp), ci, ci, ctypes.c_float, _FP]
    lib.mvd_set_weights.restype = ci
    lib.mvd_set_views.argtypes = [vp, ctypes.POINTER(vp), ci]
    lib.mvd_set_views.restype = ci
    lib.mvd_fft_plan.argtypes = [ci, ci, ctypes.POINTER(ci), ci]
    lib.mvd_fft_plan.restype = ci
    lib.mvd_get_weights.argtypes = [vp, ci, _FP, sz]
    lib.mvd_set_regularization.argtypes = [vp, ctypes.c_float]
    lib.mvd_set_regularization.restype = ci
    lib.mvd_get_weights.restype = ci
    lib.mvd_result.argtypes = [vp, _FP, sz]
    lib.mvd_result_device.argtypes = [vp, ctypes.POINTER(vp)]
    lib.mvd_synchronize.argtypes = [vp]
    lib.mvd_destroy.argtypes = [vp]
    lib.mvd_destroy.restype = None
    lib.mvd_last_error.restype = ctypes.c_char_p
    lib.mvd_get_eps.argtypes = [vp]
    lib.mvd_get_eps.restype = ctypes.c_float
    lib.mvd_get_psi0.argtypes = [vp]
    lib.mvd_get_psi0.restype = ctypes.c_float
    lib.mvd_get_path.argtypes = [vp]
    lib.mvd_get_path.restype = ci
    lib.mvd_get_compound_kernel.argtypes = [vp, ci, _FP, sz]
    lib.mvd_launch_count.restype = ctypes.c_ulonglong
    lib.mvd_profile_enable.argtypes = [ci]
    lib.mvd_profile_enable.restype = None
    lib.mvd_profile_read.argtypes = [ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_ulonglong),
                                     ctypes.POINTER(ctypes.c_double), ci]
    lib.mvd_profile_read.restype = ci
    lib.mvd_update_direct_noalloc.argtypes = [vp, vp, vp, vp, ctypes.POINTER(ci), ctypes.POINTER(ci),
                                              ctypes.c_float, vp]
    lib.mvd_update_direct_noalloc.restype = ci
    lib.mvd_batch_create.argtypes = [ctypes.POINTER(vp), ci, ci, ctypes.POINTER(vp)]
    lib.mvd_batch_create.restype = ci
    lib.mvd_batch_create_mode.argtypes = [ctypes.POINTER(vp), ci, ci, ci, ctypes.POINTER(vp)]
    lib.mvd_batch_create_mode.restype = ci
    lib.mvd_batch_mode.argtypes = [vp]
    lib.mvd_batch_mode.restype = ci
    lib.mvd_batch_run.argtypes = [vp]
    lib.mvd_batch_run.restype = ci
    lib.mvd_batch_wait.argtypes = [vp]
    lib.mvd_batch_wait.restype = ci
    lib.mvd_batch_tasks.argtypes = [vp]
    lib.mvd_batch_tasks.restype = ctypes.c_longlong
    lib.mvd_batch_destroy.argtypes = [vp]
    lib.mvd_batch_destroy.restype = None
    lib.mvd_autotune.argtypes = [vp, ctypes.c_char_p, ctypes.POINTER(TuneResult)]
    lib.mvd_unrolled_forward.argtypes = [vp, ci]
    lib.mvd_unrolled_backward.argtypes = [vp, vp, ctypes.POINTER(vp), ctypes.POINTER(vp)]
    _DP = ctypes.POINTER(ctypes.c_double)
    lib.mvd_gaussian_psf.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, ci, ctypes.POINTER(ci), _FP]
    lib.mvd_gaussian_psf_vjp.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, ci, ctypes.POINTER(ci),
                                         _FP, _DP]
    for name in ("mvd_autotune", "mvd_unrolled_forward", "mvd_unrolled_backward", "mvd_gaussian_psf", "mvd_gaussian_psf_vjp",
                 "mvd_create", "mvd_precompute_kernels", "mvd_set_estimate", "mvd_iterate", "mvd_result",
                 "mvd_result_device", "mvd_synchronize", "mvd_get_compound_kernel"):
        getattr(lib, name).restype = ci
    _lib = lib
    return lib


def _check(status: int):
    if status != MVD_OK:
        raise MvdError(status, (_lib.mvd_last_error() or b"").decode())


def _is_device(a) -> bool:
    return hasattr(a, "data_ptr") and getattr(a, "is_cuda", False)


def _host_f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


def _check_volumes(vols, shape, what, count=None):
    """The library reads X*Y*Z floats behind every volume pointer, so each volume must have
    exactly ``shape`` ([Z][Y][X]); device tensors are read as they are and must also be
    contiguous float32. Raises ValueError otherwise."""
    if count is not None and len(vols) != count:
        raise ValueError(f"expected {count} {what}s, got {len(vols)}")
    for i, v in enumerate(vols):
        if tuple(v.shape) != tuple(shape):
            raise ValueError(f"{what} {i} has shape {tuple(v.shape)}, expected {tuple(shape)}")
        if _is_device(v) and (str(v.dtype) != "torch.float32" or not v.is_contiguous()):
            raise ValueError(f"{what} {i}: a device tensor must be contiguous float32")


def mvd_last_error() -> str:
    return (load().mvd_last_error() or b"").decode()


def mvd_launch_count() -> int:
    return int(load().mvd_launch_count())


def mvd_profile_enable(on: bool = True):
    load().mvd_profile_enable(1 if on else 0)


def mvd_profile_read() -> dict:
    """{class name: (timed launches, total ms)} of the launches recorded since enabling."""
    n = 16
    names = (ctypes.c_char_p * n)()
    cnt = (ctypes.c_ulonglong * n)()
    ms = (ctypes.c_double * n)()
    k = load().mvd_profile_read(names, cnt, ms, n)
    return {names[i].decode(): (int(cnt[i]), float(ms[i])) for i in range(k)}


def mvd_create(views, psfs, dims=None, eps: float = 0.0, path="auto", stream=None, device: int = -1,
               precision="precise", boundary="periodic"):
    """Creates a context (see mvd_create in include/mvd.h); returns its handle.

    ``views``: list of float32 arrays ``[Z][Y][X]`` (numpy on the host, or CUDA
    tensors on the device, contiguous). ``psfs``: list of float32 host arrays
    ``[Kz][Ky][Kx]``. ``stream``: a ``torch.cuda.Stream`` or a raw handle.
    ``boundary``: ``"periodic"``, ``"zero"`` or ``"mirror"`` (see mvd_boundary).
    """
    lib = load()
    on_dev = _is_device(views[0])
    expect = tuple(views[0].shape) if dims is None else (int(dims[2]), int(dims[1]), int(dims[0]))
    _check_volumes(views, expect, "view")
    keep = []
    if on_dev:
        ptrs = [ctypes.c_void_p(int(v.data_ptr())) for v in views]
        shape = tuple(views[0].shape)
    else:
        hv = [_host_f32(v) for v in views]
        keep += hv
        ptrs = [ctypes.c_void_p(v.ctypes.data) for v in hv]
        shape = hv[0].shape
    if dims is None:
        dims = (shape[2], shape[1], shape[0])
    hp = [_host_f32(p) for p in psfs]
    keep += hp
    pd = [d for p in hp for d in (p.shape[2], p.shape[1], p.shape[0])]
    opt = Options()
    lib.mvd_default_options(ctypes.byref(opt))
    opt.eps = float(eps)
    opt.path = PATHS[path] if isinstance(path, str) else int(path)
    if stream is not None:
        opt.stream = ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))
    opt.views_on_device = 1 if on_dev else 0
    opt.device = int(device)
    opt.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    opt.boundary = BOUNDARIES[boundary] if isinstance(boundary, str) else int(boundary)
    h = ctypes.c_void_p()
    _check(lib.mvd_create((ctypes.c_void_p * len(ptrs))(*ptrs), len(ptrs),
                          (ctypes.c_void_p * len(hp))(*[ctypes.c_void_p(p.ctypes.data) for p in hp]),
                          (ctypes.c_int * len(pd))(*pd), (ctypes.c_int * 3)(*[int(d) for d in dims]),
                          ctypes.byref(opt), ctypes.byref(h)))
    return h


def mvd_precompute_kernels(ctx, variant="efficient"):
    _check(load().mvd_precompute_kernels(ctx, VARIANTS[variant] if isinstance(variant, str) else int(variant)))


def mvd_set_estimate(ctx, psi=None):
    lib = load()
    if psi is None:
        _check(lib.mvd_set_estimate(ctx, None, 0))
    elif _is_device(psi):
        _check(lib.mvd_set_estimate(ctx, ctypes.c_void_p(int(psi.data_ptr())), 1))
    else:
        h = _host_f32(psi)
        _check(lib.mvd_set_estimate(ctx, ctypes.c_void_p(h.ctypes.data), 0))


def mvd_set_views(ctx, views):
    """Loads the next time point's views (numpy arrays or CUDA tensors, the context's shape)."""
    lib = load()
    on_dev = _is_device(views[0])
    keep = [v if on_dev else _host_f32(v) for v in views]
    ptrs = (ctypes.c_void_p * len(keep))(*[ctypes.c_void_p(int(v.data_ptr()) if on_dev else v.ctypes.data)
                                            for v in keep])
    _check(lib.mvd_set_views(ctx, ptrs, 1 if on_dev else 0))


def mvd_fft_plan(L: int, precision="precise") -> list:
    """Stage radices of the Stockham passes for an axis of length L ([] if L is not {2,3,5}-smooth)."""
    buf = (ctypes.c_int * 64)()
    n = load().mvd_fft_plan(int(L), PRECISIONS[precision] if isinstance(precision, str) else int(precision), buf, 64)
    if n < 0:
        raise ValueError("mvd_fft_plan: bad precision")
    return list(buf[:n])


def mvd_iterate(ctx, n_iter: int, schedule=None):
    lib = load()
    if schedule is None or len(schedule) == 0:
        _check(lib.mvd_iterate(ctx, int(n_iter), None, 0))
    else:
        s = (ctypes.c_int * len(schedule))(*[int(v) for v in schedule])
        _check(lib.mvd_iterate(ctx, int(n_iter), s, len(schedule)))


def mvd_iterate_combined(ctx, n_iter: int, root: bool = True):
    """Combined update (all views' factors from the same estimate); ``root`` takes their geometric mean."""
    _check(load().mvd_iterate_combined(ctx, int(n_iter), 1 if root else 0))


WEIGHT_NORMS = {"sum1": 0, "min_overlap": 1, "avg_overlap": 2, "user": 3}


def mvd_set_weights(ctx, weights, norm="sum1", value: float = 0.0) -> float:
    """Per-view weight images in [0, 1] (partial overlap), normalised on the device; returns the
    normalisation target T. ``weights=None`` removes them."""
    lib = load()
    if weights is None:
        _check(lib.mvd_set_weights(ctx, None, 0, 0, 0.0, None))
        return 0.0
    n = WEIGHT_NORMS[norm] if isinstance(norm, str) else int(norm)
    on_dev = _is_device(weights[0])
    keep = [w if on_dev else _host_f32(w) for w in weights]
    ptrs = (ctypes.c_void_p * len(keep))(*[ctypes.c_void_p(int(w.data_ptr()) if on_dev else w.ctypes.data)
                                            for w in keep])
    T = ctypes.c_float()
    _check(lib.mvd_set_weights(ctx, ptrs, 1 if on_dev else 0, n, float(value), ctypes.byref(T)))
    return float(T.value)


def mvd_set_regularization(ctx, lam: float):
    """Tikhonov regularisation of the sequential update (one-step-late form, factor c / (1 + lam psi))."""
    _check(load().mvd_set_regularization(ctx, float(lam)))


def mvd_get_weights(ctx, v: int, shape_zyx) -> np.ndarray:
    out = np.empty(shape_zyx, dtype=np.float32)
    _check(load().mvd_get_weights(ctx, int(v), out.ctypes.data_as(_FP), out.size))
    return out


def mvd_result(ctx, out: np.ndarray):
    """Copies psi into the float32 host array ``out`` (synchronises)."""
    assert out.dtype == np.float32 and out.flags["C_CONTIGUOUS"]
    _check(load().mvd_result(ctx, out.ctypes.data_as(_FP), out.size))
    return out


def mvd_result_device(ctx) -> int:
    p = ctypes.c_void_p()
    _check(load().mvd_result_device(ctx, ctypes.byref(p)))
    return int(p.value or 0)


def mvd_synchronize(ctx):
    _check(load().mvd_synchronize(ctx))


def mvd_destroy(ctx):
    if ctx:
        load().mvd_destroy(ctx)


def mvd_get_eps(ctx) -> float:
    return float(load().mvd_get_eps(ctx))


def mvd_get_psi0(ctx) -> float:
    return float(load().mvd_get_psi0(ctx))


def mvd_get_path(ctx) -> int:
    return int(load().mvd_get_path(ctx))


def mvd_get_compound_kernel(ctx, v: int, shape_zyx) -> np.ndarray:
    out = np.empty(shape_zyx, dtype=np.float32)
    _check(load().mvd_get_compound_kernel(ctx, int(v), out.ctypes.data_as(_FP), out.size))
    return out


def mvd_update_direct_noalloc(psi, phi, psf, comp, eps: float, stream=None):
    """One view update without any device allocation (see include/mvd.h).

    ``psi`` (updated in place), ``phi``, ``psf`` and ``comp`` are contiguous
    float32 CUDA tensors on one device; ``psi``/``phi`` shaped ``[Z][Y][X]``,
    ``psf``/``comp`` shaped ``[Kz][Ky][Kx]``. Anything else raises ValueError
    before the library sees a pointer (it reads X*Y*Z and Kx*Ky*Kz floats behind
    them). The call runs with psi's device current.
    """
    for name, t in (("psi", psi), ("phi", phi), ("psf", psf), ("comp", comp)):
        if not _is_device(t) or str(t.dtype) != "torch.float32" or not t.is_contiguous() or t.dim() != 3:
            raise ValueError(f"{name} must be a contiguous 3D float32 CUDA tensor")
    if len({t.device for t in (psi, phi, psf, comp)}) != 1:
        raise ValueError("psi, phi, psf and comp must live on one device")
    _check_volumes([phi], psi.shape, "view")
    _check_volumes([comp], psf.shape, "kernel")
    dims = (ctypes.c_int * 3)(int(psi.shape[2]), int(psi.shape[1]), int(psi.shape[0]))
    kd = (ctypes.c_int * 3)(int(psf.shape[2]), int(psf.shape[1]), int(psf.shape[0]))
    st = None if stream is None else ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))
    ptr = lambda t: ctypes.c_void_p(int(t.data_ptr()))  # noqa: E731
    import torch

    with torch.cuda.device(psi.device):  # the C entry point works on the current device
            _check(load().mvd_update_direct_noalloc(ptr(psi), ptr(phi), ptr(psf), ptr(comp), dims, kd, float(eps),
                                                st))


BATCH_MODES = {"auto": 0, "persistent": 1, "branches": 2}


def mvd_batch_create(ctxs, n_iter: int, mode="auto"):
    """Batch over contexts (one device, one stream); mode "auto", "persistent" or "branches"."""
    arr = (ctypes.c_void_p * len(ctxs))(*[c if isinstance(c, ctypes.c_void_p) else c.ctx for c in ctxs])
    h = ctypes.c_void_p()
    m = BATCH_MODES[mode] if isinstance(mode, str) else int(mode)
    _check(load().mvd_batch_create_mode(arr, len(ctxs), int(n_iter), m, ctypes.byref(h)))
    return h


def mvd_batch_mode(batch) -> str:
    return {1: "persistent", 2: "branches"}.get(int(load().mvd_batch_mode(batch)), "none")


def mvd_batch_run(batch):
    _check(load().mvd_batch_run(batch))


def mvd_batch_wait(batch):
    _check(load().mvd_batch_wait(batch))


def mvd_batch_tasks(batch) -> int:
    return int(load().mvd_batch_tasks(batch))


def mvd_batch_destroy(batch):
    if batch:
        load().mvd_batch_destroy(batch)


def mvd_autotune(ctx, cache_path=None) -> dict:
    """Times the engine candidates on this context and keeps the fastest (see include/mvd.h)."""
    r = TuneResult()
    cp = None if cache_path is None else os.fsencode(cache_path)
    _check(load().mvd_autotune(ctx, cp, ctypes.byref(r)))
    return {"path": {MVD_PATH_DIRECT: "direct", MVD_PATH_FFT: "fft"}[r.path], "direct_tile_y": r.direct_tile_y,
            "fft_engine": {1: "register", 0: "stockham", -1: None}[r.fft_engine], "from_cache": bool(r.from_cache),
            "ms_per_update": r.ms_per_update}


def mvd_unrolled_forward(ctx, n_iter: int):
    """n_iter iterations from the flat start, keeping per-iteration checkpoints."""
    _check(load().mvd_unrolled_forward(ctx, int(n_iter)))


def mvd_unrolled_backward(ctx, grad_psi, grad_views, psf_shapes):
    """Reverse pass of the last unrolled forward run.

    ``grad_psi``: contiguous float32 CUDA tensor ``[Z][Y][X]``; ``grad_views``:
    CUDA tensors of the same shape, overwritten with dL/dphi_v. Returns the
    raw-PSF gradients as float32 numpy arrays shaped ``psf_shapes``.
    """
    gp = [np.empty(sh, dtype=np.float32) for sh in psf_shapes]
    gv = (ctypes.c_void_p * len(grad_views))(*[ctypes.c_void_p(int(g.data_ptr())) for g in grad_views])
    gpp = (ctypes.c_void_p * len(gp))(*[ctypes.c_void_p(g.ctypes.data) for g in gp])
    _check(load().mvd_unrolled_backward(ctx, ctypes.c_void_p(int(grad_psi.data_ptr())), gv, gpp))
    return gp


_AXES = {"x": 0, "y": 1, "z": 2}


def mvd_gaussian_psf(sigma_xy: float, sigma_ax: float, box_xyz, angle_deg: float = 0.0, axis="z") -> np.ndarray:
    """Gaussian PSF model sampled on the centred box ``box_xyz`` (Kx, Ky, Kz); shaped ``[Kz][Ky][Kx]``."""
    box = (ctypes.c_int * 3)(*[int(b) for b in box_xyz])
    out = np.empty((box_xyz[2], box_xyz[1], box_xyz[0]), dtype=np.float32)
    _check(load().mvd_gaussian_psf(float(sigma_xy), float(sigma_ax), float(angle_deg), _AXES.get(axis, axis), box,
                                   out.ctypes.data_as(_FP)))
    return out


def mvd_gaussian_psf_vjp(sigma_xy: float, sigma_ax: float, box_xyz, grad_psf, angle_deg: float = 0.0,
                         axis="z") -> np.ndarray:
    """(dL/dsigma_xy, dL/dsigma_ax) for dL/dPSF ``grad_psf`` (``[Kz][Ky][Kx]``)."""
    box = (ctypes.c_int * 3)(*[int(b) for b in box_xyz])
    g = _host_f32(grad_psf)
    out = np.zeros(2, dtype=np.float64)
    _check(load().mvd_gaussian_psf_vjp(float(sigma_xy), float(sigma_ax), float(angle_deg), _AXES.get(axis, axis), box,
                                       g.ctypes.data_as(_FP), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return out


class Deconvolver:
    """Owns one context: ``with Deconvolver(views, psfs) as d: d.iterate(10); psi = d.result()``.

    ``variant``: "plain", "efficient", "opt1", "opt2" (mvd_variant). ``path``: "auto", "direct",
    "fft". ``precision``: "precise", "mixed", "fast" (mvd_precision). ``boundary``: "periodic",
    "zero", "mirror" (mvd_boundary). Volumes are ``[Z][Y][X]`` float32 (numpy, or contiguous
    CUDA tensors); the setters check their shapes against the context's.
    """

    def __init__(self, views, psfs, variant="efficient", eps=0.0, path="auto", stream=None, device=-1,
                 precision="precise", boundary="periodic"):
        self.shape = tuple(views[0].shape)
        self.n_views = len(views)
        self.psf_shapes = [tuple(p.shape) for p in psfs]
        self.ctx = mvd_create(views, psfs, eps=eps, path=path, stream=stream, device=device, precision=precision,
                              boundary=boundary)
        try:
            mvd_precompute_kernels(self.ctx, variant)
        except Exception:
            self.close()
            raise

    def iterate(self, n_iter, schedule=None):
        mvd_iterate(self.ctx, n_iter, schedule)

    def set_weights(self, weights, norm="sum1", value=0.0) -> float:
        if weights is not None:
            _check_volumes(weights, self.shape, "weight image", self.n_views)
        return mvd_set_weights(self.ctx, weights, norm, value)

    def set_regularization(self, lam):
        mvd_set_regularization(self.ctx, lam)

    def weights(self, v):
        return mvd_get_weights(self.ctx, v, self.shape)

    def iterate_combined(self, n_iter, root=True):
        mvd_iterate_combined(self.ctx, n_iter, root)

    def set_estimate(self, psi=None):
        if psi is not None:
            _check_volumes([psi], self.shape, "estimate")
        mvd_set_estimate(self.ctx, psi)

    def set_views(self, views):
        _check_volumes(views, self.shape, "view", self.n_views)
        mvd_set_views(self.ctx, views)

    def result(self, out=None) -> np.ndarray:
        if out is None:
            out = np.empty(self.shape, dtype=np.float32)
        return mvd_result(self.ctx, out)

    def autotune(self, cache_path=None) -> dict:
        return mvd_autotune(self.ctx, cache_path)

    def compound_kernel(self, v):
        return mvd_get_compound_kernel(self.ctx, v, self.psf_shapes[v])

    @property
    def eps(self):
        return mvd_get_eps(self.ctx)

    @property
    def psi0(self):
        return mvd_get_psi0(self.ctx)

    @property
    def path(self):
        return {MVD_PATH_DIRECT: "direct", MVD_PATH_FFT: "fft"}.get(mvd_get_path(self.ctx), "none")

    def synchronize(self):
        mvd_synchronize(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            mvd_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
