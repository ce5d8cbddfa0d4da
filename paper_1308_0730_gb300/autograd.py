"""torch.autograd front end of the unrolled deconvolution and the Gaussian PSF model.

``unrolled_deconvolve(views, psfs, n_iter)`` runs n_iter iterations of the
sequential update (Eq. 15 with the compound kernels of Eq. 222) from the flat
start and returns psi_K; its backward is the library's hand-written adjoint
(mvd_unrolled_backward), giving gradients for the views and the raw PSFs.
``gaussian_psf(sigma, box)`` samples the PSF model with the library and
back-propagates into (sigma_xy, sigma_ax). Argument marshalling only: the
forward iterations and the adjoint run in libmvd.so.
"""
from __future__ import annotations

import numpy as np
import torch

from . import mvd as _m


class _DeviceVolume:
    """Borrowed view of a device buffer through the CUDA array interface."""

    def __init__(self, ptr: int, shape):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<f4", "data": (int(ptr), False),
                                         "version": 2, "strides": None}


class _Holder:
    def __init__(self, ctx):
        self.ctx = ctx

    def close(self):
        if self.ctx:
            _m.mvd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class UnrolledDeconvolution(torch.autograd.Function):
    """psi_K = K iterations of the default schedule from psi0 = mean of the views."""

    @staticmethod
    def forward(ctx, views, n_iter, variant, path, *psfs):
        if not views.is_cuda:
            raise ValueError("views must be a CUDA tensor [N][Z][Y][X]")
        views = views.detach().to(torch.float32).contiguous()
        psf_host = [p.detach().to("cpu", torch.float32).contiguous().numpy() for p in psfs]
        stream = torch.cuda.current_stream(views.device)
        h = _m.mvd_create([views[v] for v in range(views.shape[0])], psf_host, path=path, stream=stream,
                          device=views.device.index)
        holder = _Holder(h)
        _m.mvd_precompute_kernels(h, variant)
        _m.mvd_unrolled_forward(h, n_iter)
        ptr = _m.mvd_result_device(h)
        psi = torch.as_tensor(_DeviceVolume(ptr, views.shape[1:]), device=views.device).clone()
        ctx.holder = holder
        ctx.psf_meta = [(tuple(p.shape), p.device, p.dtype) for p in psfs]
        ctx.n_views = views.shape[0]
        return psi

    @staticmethod
    def backward(ctx, grad_psi):
        holder = ctx.holder
        if holder.ctx is None:
            raise RuntimeError("unrolled deconvolution: backward called twice")
        g = grad_psi.detach().to(torch.float32).contiguous()
        grad_views = torch.empty((ctx.n_views,) + tuple(g.shape), dtype=torch.float32, device=g.device)
        gp = _m.mvd_unrolled_backward(holder.ctx, g, [grad_views[v] for v in range(ctx.n_views)],
                                      [m[0] for m in ctx.psf_meta])
        holder.close()
        grads_psf = [torch.from_numpy(a).to(dev, dt) for a, (_, dev, dt) in zip(gp, ctx.psf_meta)]
        return (grad_views, None, None, None, *grads_psf)


def unrolled_deconvolve(views: torch.Tensor, psfs, n_iter: int, variant: str = "efficient", path: str = "auto"):
    """Differentiable K-iteration deconvolution; ``views`` CUDA ``[N][Z][Y][X]``, ``psfs`` ``[Kz][Ky][Kx]`` tensors."""
    return UnrolledDeconvolution.apply(views, int(n_iter), variant, path, *psfs)


class GaussianPSF(torch.autograd.Function):
    """Normalised anisotropic Gaussian on a centred box, differentiable in (sigma_xy, sigma_ax)."""

    @staticmethod
    def forward(ctx, sigma, box_xyz, angle_deg, axis):
        s = sigma.detach().to("cpu", torch.float64).numpy()
        out = _m.mvd_gaussian_psf(float(s[0]), float(s[1]), box_xyz, angle_deg, axis)
        ctx.args = (float(s[0]), float(s[1]), tuple(box_xyz), angle_deg, axis)
        ctx.sigma_meta = (sigma.device, sigma.dtype)
        return torch.from_numpy(out)

    @staticmethod
    def backward(ctx, grad_psf):
        sxy, sax, box, angle, axis = ctx.args
        gp = grad_psf.detach().to("cpu", torch.float32).contiguous().numpy()
        gs = _m.mvd_gaussian_psf_vjp(sxy, sax, box, gp, angle, axis)
        dev, dt = ctx.sigma_meta
        return torch.from_numpy(np.asarray(gs)).to(dev, dt), None, None, None


def gaussian_psf(sigma: torch.Tensor, box_xyz, angle_deg: float = 0.0, axis: str = "z") -> torch.Tensor:
    """PSF ``[Kz][Ky][Kx]`` (float32, CPU) from ``sigma = (sigma_xy, sigma_ax)``; rotation about y by angle_deg."""
    return GaussianPSF.apply(sigma, tuple(box_xyz), float(angle_deg), axis)
