"""Seeded synthetic workloads generated on a CUDA device with PyTorch.

The recipe is that of ``synth.workloads.config3`` (the 1024x1024x512 seven-view
specimen): ellipsoids drawn at twice the resolution and box-downsampled, the
periodic blur of the objects with each view's PSF, scaled so that the
brightest blurred voxel of any view holds 200 photons, a uniform background of
5, and a Poisson draw per voxel. The CPU generator takes minutes and tens of GB
of host memory at that size; here the object parameters come from the same
numpy draws (``ellipsoid_params``), the rasterisation and the FP64 FFT blur run
on the device, and the noise is PyTorch's Poisson sampler with a seeded device
generator.

The views are therefore not bit-identical to the CPU generator's (FFT rounding
and a different Poisson sampler); every consumer takes the views generated
here, host copies included. Nothing here belongs to the deconvolution method:
it is input generation only.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .workloads import _as_stored, _fine_offsets, _spim_psfs, ellipsoid_params


@dataclass
class DeviceWorkload:
    """Views resident on a CUDA device (float32 tensors [Z][Y][X]) and their PSFs (numpy)."""

    name: str
    dims: tuple  # (X, Y, Z)
    views: list  # torch.float32 CUDA tensors
    psfs: list  # numpy float32 [Kz][Ky][Kx]
    n_iter: int
    variant: str = "efficient"
    meta: dict = field(default_factory=dict)

    @property
    def n_views(self) -> int:
        return len(self.psfs)

    @property
    def voxels(self) -> int:
        X, Y, Z = self.dims
        return X * Y * Z

    def host_views(self, pinned: bool = False) -> list:
        """Host copies of the views (numpy float32; page-locked with ``pinned``)."""
        out = []
        for v in self.views:
            h = v.cpu()
            if pinned:
                h = h.pin_memory()
            out.append(h.numpy())
        return out


def _rasterise(torch, dev, dims, h, centres, radii, inten, rots, chunk=512):
    """Sum of the ellipsoids on the periodic grid (FP64): each coarse voxel of an ellipsoid's
    (2h+1)^3 block takes the fraction of its 2x2x2 fine samples inside it times its intensity."""
    X, Y, Z = dims
    nb = 2 * h + 1
    f = torch.tensor(_fine_offsets(h), dtype=torch.float64, device=dev)
    FZ, FY, FX = torch.meshgrid(f, f, f, indexing="ij")
    P = torch.stack([FX.reshape(-1), FY.reshape(-1), FZ.reshape(-1)], dim=1)  # (2nb)^3 x 3, z slowest
    base = torch.arange(nb, device=dev, dtype=torch.long) - h
    vol = torch.zeros(Z * Y * X, dtype=torch.float64, device=dev)
    ci_all = np.floor(centres).astype(np.int64)
    frac_all = centres - ci_all
    R_all = np.stack(rots)  # n x 3 x 3
    for a in range(0, len(centres), chunk):
        b = min(len(centres), a + chunk)
        fr = torch.tensor(frac_all[a:b], dtype=torch.float64, device=dev)
        r = torch.tensor(radii[a:b], dtype=torch.float64, device=dev)
        Rt = torch.tensor(R_all[a:b], dtype=torch.float64, device=dev).transpose(1, 2)
        rel = P.unsqueeze(0) - fr.unsqueeze(1)  # n x S x 3
        body = torch.einsum("nij,nsj->nsi", Rt, rel) / r.unsqueeze(1)
        inside = (body * body).sum(-1) <= 1.0
        del rel, body
        cnt = inside.reshape(b - a, nb, 2, nb, 2, nb, 2).sum(dim=(2, 4, 6)).to(torch.float64)
        val = cnt * (torch.tensor(inten[a:b], dtype=torch.float64, device=dev) / 8.0).view(-1, 1, 1, 1)
        ci = torch.tensor(ci_all[a:b], dtype=torch.long, device=dev)
        xi = (ci[:, 0:1] + base.view(1, -1)) % X
        yi = (ci[:, 1:2] + base.view(1, -1)) % Y
        zi = (ci[:, 2:3] + base.view(1, -1)) % Z
        flat = (zi.view(-1, nb, 1, 1) * Y + yi.view(-1, 1, nb, 1)) * X + xi.view(-1, 1, 1, nb)
        vol.index_add_(0, flat.reshape(-1), val.reshape(-1))
    return vol.view(Z, Y, X)


def _psf_grid_spectrum(torch, psf, shape, dev):
    Kz, Ky, Kx = psf.shape
    big = torch.zeros(shape, dtype=torch.float64, device=dev)
    zi = torch.tensor((np.arange(Kz) - (Kz - 1) // 2) % shape[0], device=dev)
    yi = torch.tensor((np.arange(Ky) - (Ky - 1) // 2) % shape[1], device=dev)
    xi = torch.tensor((np.arange(Kx) - (Kx - 1) // 2) % shape[2], device=dev)
    big[zi.view(-1, 1, 1), yi.view(1, -1, 1), xi.view(1, 1, -1)] = torch.tensor(psf, dtype=torch.float64,
                                                                                   device=dev)
    return torch.fft.rfftn(big)


def config3_device(seed: int = 1003, dims=(1024, 1024, 512), n_objects: int = 150_000, device="cuda:0",
                   n_iter: int = 10) -> DeviceWorkload:
    """The 1024x1024x512 seven-view specimen (150k ellipsoids, radii 3-6, intensity 0.5-1; PSFs
    sigma 1.5/5, box 19x19x51 rotated by k*51.43 deg about y; peak 200 photons + background 5;
    10 iterations), generated on ``device``."""
    import torch

    dev = torch.device(device)
    rng = np.random.default_rng(seed)
    centres, radii, inten, rots = ellipsoid_params(rng, dims, n_objects, (3.0, 6.0), (0.5, 1.0))
    h = int(math.ceil(6.0)) + 1
    X, Y, Z = dims
    shape = (Z, Y, X)
    objects = _rasterise(torch, dev, dims, h, centres, radii, inten, rots)
    psfs64, angles = _spim_psfs(7, 1.5, 5.0, (19, 19, 51))
    spec = torch.fft.rfftn(objects)
    del objects
    blurred = []
    for p in psfs64:
        b = torch.fft.irfftn(spec * _psf_grid_spectrum(torch, _as_stored(p), shape, dev), s=shape)
        blurred.append(b.clamp_(min=0.0).to(torch.float32))
        del b
    del spec
    scale = 200.0 / max(float(b.max()) for b in blurred)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    views = []
    for i in range(len(blurred)):
        lam = blurred[i].mul_(scale).add_(5.0)
        blurred[i] = None
        views.append(torch.poisson(lam, generator=gen))
        del lam
    if dev.type == "cuda":
        torch.cuda.synchronize(dev)
    name = f"ellipsoids-{X}x{Y}x{Z}-7views"
    return DeviceWorkload(name=name, dims=tuple(dims), views=views, psfs=[p.astype(np.float32) for p in psfs64],
                          n_iter=n_iter, meta=dict(angles=angles, box=(19, 19, 51), peak=200.0, background=5.0,
                                                   objects=n_objects, scale=scale, generator="device"))
