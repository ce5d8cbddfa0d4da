"""Synthetic light-sheet workloads: objects, PSFs, blur, Poisson noise.

Arrays are C-ordered ``[z][y][x]`` (x fastest). Dimensions are quoted as
``(X, Y, Z)``; PSF boxes as ``(Kx, Ky, Kz)``, odd, centre at ``(K-1)/2``.

Object model: many small objects of random location, size and intensity,
drawn at twice the resolution and box-downsampled (the paper's simulated
specimen, Suppl. Note "Biological object simulation"). The microscope blur is
the circular convolution of the truth with each view's PSF, evaluated here
with an FP64 FFT (scipy/numpy), then a Poisson draw per voxel (Suppl. Note
"Sampling and noise"). Attenuation, anisotropic sampling and rotation of the
volume are not simulated: the views are already on one registered grid.

Seeds: the workload of the k-th configuration uses ``default_rng(1000 + k)``.
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass, field

import numpy as np

try:  # multithreaded FFT where scipy is present; numpy otherwise
    import scipy.fft as _fft

    def _rfftn(a):
        return _fft.rfftn(a, workers=-1)

    def _irfftn(a, shape):
        return _fft.irfftn(a, s=shape, workers=-1)
except Exception:  # pragma: no cover
    def _rfftn(a):
        return np.fft.rfftn(a)

    def _irfftn(a, shape):
        return np.fft.irfftn(a, s=shape)


@dataclass
class Workload:
    """One deconvolution problem: registered views, PSFs and ground truth."""

    name: str
    dims: tuple  # (X, Y, Z)
    views: list  # float32 [Z][Y][X], photon counts
    psfs: list  # float32 [Kz][Ky][Kx], each sums to 1 (normalised in FP64)
    truth: np.ndarray  # float32 [Z][Y][X], photon units
    n_iter: int
    variant: str = "efficient"
    meta: dict = field(default_factory=dict)

    @property
    def n_views(self) -> int:
        return len(self.views)

    @property
    def voxels(self) -> int:
        X, Y, Z = self.dims
        return X * Y * Z

    def psf_dims(self):
        return [(p.shape[2], p.shape[1], p.shape[0]) for p in self.psfs]


# ----------------------------------------------------------------------------
# geometry helpers
# ----------------------------------------------------------------------------

def smooth235(n: int) -> int:
    """Nearest integer >= 8 whose only prime factors are 2, 3 and 5 (ties: smaller)."""
    def is_smooth(m):
        for p in (2, 3, 5):
            while m % p == 0:
                m //= p
        return m == 1

    best = None
    for d in range(0, n):
        for m in (n - d, n + d):
            if m >= 8 and is_smooth(m):
                best = m
                break
        if best is not None:
            return best
    return 8


def _rot_y(angle_deg: float) -> np.ndarray:
    t = math.radians(angle_deg)
    c, s = math.cos(t), math.sin(t)
    # x' = c x + s z ; z' = -s x + c z  (rotation about y)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def rotated_box(box_xyz, angle_deg: float):
    """Odd axis-aligned bounding box of an odd (Kx,Ky,Kz) box rotated about y."""
    R = _rot_y(angle_deg)
    h = np.array([(k - 1) / 2.0 for k in box_xyz])
    ext = np.abs(R) @ h
    # guard against cos/sin rounding just above an integer
    return tuple(int(2 * math.floor(e + 1e-9) + 1) for e in ext)


def gaussian_psf(sigma_xy: float, sigma_ax: float, box_xyz, axis: str = "z",
                 angle_y_deg: float = 0.0, rotate_box: bool = True) -> np.ndarray:
    """Point-sampled anisotropic Gaussian PSF, FP64, normalised to sum 1.

    ``exp(-d^T S^-1 d / 2)`` at integer offsets ``d`` from the box centre, with
    ``S = R diag(.) R^T``; the axial sigma sits on ``axis`` and ``R`` rotates
    about y by ``angle_y_deg``. ``box_xyz`` is the box of the unrotated PSF;
    with ``rotate_box`` the sampled box is its rotated odd bounding box.
    Returns an array shaped ``[Kz][Ky][Kx]``.
    """
    var = {"x": sigma_xy ** 2, "y": sigma_xy ** 2, "z": sigma_xy ** 2}
    var[axis] = sigma_ax ** 2
    D = np.diag([var["x"], var["y"], var["z"]])
    R = _rot_y(angle_y_deg)
    S = R @ D @ R.T
    Si = np.linalg.inv(S)
    box = rotated_box(box_xyz, angle_y_deg) if rotate_box else tuple(box_xyz)
    Kx, Ky, Kz = box
    dz, dy, dx = np.meshgrid(np.arange(Kz) - (Kz - 1) / 2, np.arange(Ky) - (Ky - 1) / 2,
                             np.arange(Kx) - (Kx - 1) / 2, indexing="ij")
    d = np.stack([dx, dy, dz], axis=-1)
    q = np.einsum("...i,ij,...j->...", d, Si, d)
    p = np.exp(-0.5 * q)
    return p / p.sum()


def _random_rotation(rng) -> np.ndarray:
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([
        [a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
        [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
        [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d],
    ])


# ----------------------------------------------------------------------------
# objects (2x supersampled, box-downsampled)
# ----------------------------------------------------------------------------

def _fine_offsets(h: int):
    """Fine-grid sample positions (coarse units) for a (2h+1)^3 coarse block."""
    n = 2 * h + 1
    f = (np.arange(2 * n) + 0.5) / 2.0 - 0.5 - h  # relative to block centre voxel
    return f


def blobs_truth(rng, dims, n, sigma_range, peak_range, background) -> np.ndarray:
    """Gaussian blobs on a periodic grid, plus a constant background (FP64)."""
    X, Y, Z = dims
    fx = (np.arange(2 * X) + 0.5) / 2.0 - 0.5
    fy = (np.arange(2 * Y) + 0.5) / 2.0 - 0.5
    fz = (np.arange(2 * Z) + 0.5) / 2.0 - 0.5
    fine = np.zeros((2 * Z, 2 * Y, 2 * X))
    centres = rng.uniform(0, 1, size=(n, 3)) * np.array([X, Y, Z])
    sigmas = rng.uniform(*sigma_range, size=n)
    peaks = rng.uniform(*peak_range, size=n)

    def pdist(f, c, L):
        d = f - c
        return d - L * np.round(d / L)

    for (cx, cy, cz), s, pk in zip(centres, sigmas, peaks):
        ex = np.exp(-0.5 * (pdist(fx, cx, X) / s) ** 2)
        ey = np.exp(-0.5 * (pdist(fy, cy, Y) / s) ** 2)
        ez = np.exp(-0.5 * (pdist(fz, cz, Z) / s) ** 2)
        fine += pk * ez[:, None, None] * ey[None, :, None] * ex[None, None, :]
    coarse = fine.reshape(Z, 2, Y, 2, X, 2).mean(axis=(1, 3, 5))
    return coarse + background


def _ellipsoid_counts(args):
    """Fine samples inside each ellipsoid, summed over the 2x2x2 fine cells of
    every coarse voxel of its (2h+1)^3 block (0..8, uint8)."""
    h, frac, radii, rots = args
    nb = 2 * h + 1
    f = _fine_offsets(h)
    FZ, FY, FX = np.meshgrid(f, f, f, indexing="ij")
    P = np.stack([FX.ravel(), FY.ravel(), FZ.ravel()], axis=0)  # 3 x (2nb)^3
    out = np.empty((len(frac), nb, nb, nb), dtype=np.uint8)
    for k, (fr, r, Rm) in enumerate(zip(frac, radii, rots)):
        # fine points relative to the ellipsoid centre, in its body frame
        rel = P - fr[:, None]
        body = (Rm.T @ rel) / r[:, None]
        inside = (np.einsum("ij,ij->j", body, body) <= 1.0).reshape(2 * nb, 2 * nb, 2 * nb)
        out[k] = inside.reshape(nb, 2, nb, 2, nb, 2).sum(axis=(1, 3, 5))
    return out


def ellipsoid_params(rng, dims, n, radii_range, intensity_range):
    """Random centres (x, y, z), per-axis radii, intensities and orientations of n ellipsoids,
    drawn in this order from ``rng``."""
    X, Y, Z = dims
    centres = rng.uniform(0, 1, size=(n, 3)) * np.array([X, Y, Z])
    radii = rng.uniform(*radii_range, size=(n, 3))
    inten = rng.uniform(*intensity_range, size=n)
    rots = [_random_rotation(rng) for _ in range(n)]
    return centres, radii, inten, rots


def ellipsoids_truth(rng, dims, n, radii_range, intensity_range, workers: int = 1) -> np.ndarray:
    """Solid ellipsoids (random radii, orientation, intensity), additive, periodic.

    Each coarse voxel takes the fraction of its 2x2x2 fine samples inside the
    ellipsoid times the intensity. ``workers > 1`` rasterises chunks in a
    spawned process pool (the calling program's main module must be
    import-safe, i.e. guarded by ``if __name__ == "__main__"``); the result is
    identical.
    """
    X, Y, Z = dims
    h = int(math.ceil(radii_range[1])) + 1
    nb = 2 * h + 1
    vol = np.zeros((Z, Y, X))
    centres, radii, inten, rots = ellipsoid_params(rng, dims, n, radii_range, intensity_range)
    base = np.arange(nb) - h
    ci_all = np.floor(centres).astype(int)
    frac_all = centres - ci_all  # centre offset within its voxel
    chunk = 2048
    jobs = [(h, frac_all[a:a + chunk], radii[a:a + chunk], rots[a:a + chunk]) for a in range(0, n, chunk)]
    if workers > 1 and len(jobs) > 1:
        import multiprocessing as mp

        with mp.get_context("spawn").Pool(workers) as pool:
            counts = pool.map(_ellipsoid_counts, jobs)
    else:
        counts = [_ellipsoid_counts(j) for j in jobs]
    k = 0
    for cnt in counts:
        for c8 in cnt:
            ci = ci_all[k]
            block = (c8 / 8.0) * inten[k]
            xi = (ci[0] + base) % X
            yi = (ci[1] + base) % Y
            zi = (ci[2] + base) % Z
            vol[np.ix_(zi, yi, xi)] += block
            k += 1
    return vol


def blend_weights(dims, lo, hi, border) -> np.ndarray:
    """Blending image of a view that covers the box [lo, hi) of the volume
    (x, y, z): 1 inside, rising from 0 over `border` voxels at each face of the
    box following half a cosine period, 0 outside; the product over the axes.
    Returns float32 [Z][Y][X]."""
    axes = []
    for n, a, b, w in zip(dims, lo, hi, border):
        i = np.arange(n)
        d = np.minimum(i - a, b - 1 - i).astype(np.float64)  # voxels from the nearest face, inside
        ramp = 0.5 * (1.0 - np.cos(np.pi * (d + 1.0) / (w + 1.0))) if w > 0 else np.ones(n)
        axes.append(np.where(d < 0, 0.0, np.where(d < w, ramp, 1.0)))
    wx, wy, wz = axes
    return (wz[:, None, None] * wy[None, :, None] * wx[None, None, :]).astype(np.float32)


# ----------------------------------------------------------------------------
# imaging model
# ----------------------------------------------------------------------------

def _psf_volume_spectrum(psf: np.ndarray, shape_zyx):
    """Spectrum of a PSF placed on the periodic grid with its centre at the origin."""
    Kz, Ky, Kx = psf.shape
    big = np.zeros(shape_zyx)
    zi = (np.arange(Kz) - (Kz - 1) // 2) % shape_zyx[0]
    yi = (np.arange(Ky) - (Ky - 1) // 2) % shape_zyx[1]
    xi = (np.arange(Kx) - (Kx - 1) // 2) % shape_zyx[2]
    big[np.ix_(zi, yi, xi)] = psf
    return _rfftn(big)


def blur_circular(vol: np.ndarray, psf: np.ndarray) -> np.ndarray:
    """Microscope image formation: periodic convolution of ``vol`` with ``psf`` (FP64 FFT)."""
    s = _rfftn(vol) * _psf_volume_spectrum(psf, vol.shape)
    out = _irfftn(s, vol.shape)
    return np.maximum(out, 0.0)


def _as_stored(p):
    """The PSF as the deconvolution receives it: rounded to FP32 (the FP64
    samples' last bits depend on the platform's exp)."""
    return np.asarray(p, dtype=np.float32).astype(np.float64)


# fixed-point scales of the exact image formation below
_VOL_BITS, _PSF_BITS = 14, 22


def image_exact(vol: np.ndarray, psf: np.ndarray) -> np.ndarray:
    """Periodic blur ``vol * psf`` that is bit-identical on every platform.

    ``vol`` and ``psf`` are rounded to the fixed-point grids 2^-14 and 2^-22;
    their integer convolution is computed with an FP64 FFT and rounded to the
    nearest integer, which recovers the exact integer sum because the FFT's
    error stays far below 0.5 at these scales (for the volumes used here the
    integers stay below 2^53 and the error bound is about 1e-2). The result is
    that exact sum times 2^-36. Last-bit differences between FFT libraries
    therefore cannot reach the Poisson sampler that consumes it.
    """
    t = np.rint(np.asarray(vol, np.float64) * 2.0 ** _VOL_BITS)
    k = np.rint(np.asarray(psf, np.float64) * 2.0 ** _PSF_BITS)
    s = _rfftn(t) * _psf_volume_spectrum(k, t.shape)
    out = np.rint(_irfftn(s, t.shape))
    return np.maximum(out, 0.0) * 2.0 ** -(_VOL_BITS + _PSF_BITS)


def _observe(rng, truth, psfs):
    blurred = [image_exact(truth, _as_stored(p)) for p in psfs]
    views = [rng.poisson(b).astype(np.float32) for b in blurred]
    return views


def time_series(w: "Workload", n_points: int, seed: int) -> list:
    """Views of ``n_points`` later time points of workload ``w``: the object drifts by one voxel
    along x per time point, recorded with the same PSFs and fresh Poisson noise."""
    psfs = [p.astype(np.float64) for p in w.psfs]
    out = []
    for t in range(n_points):
        rng = np.random.default_rng(seed + t)
        out.append(_observe(rng, np.roll(w.truth.astype(np.float64), t, axis=2), psfs))
    return out


def _finish(name, dims, truth, psfs64, views, n_iter, variant="efficient", **meta):
    return Workload(name=name, dims=tuple(dims), views=views,
                    psfs=[p.astype(np.float32) for p in psfs64],
                    truth=truth.astype(np.float32), n_iter=n_iter, variant=variant,
                    meta=dict(meta))


def _spim_psfs(n_views, sigma_xy, sigma_ax, box, angles=None):
    if angles is None:
        angles = [k * 360.0 / n_views for k in range(n_views)]
    return [gaussian_psf(sigma_xy, sigma_ax, box, "z", a) for a in angles], list(angles)


def _scale_to_peak(truth, psfs, peak):
    m = max(image_exact(truth, _as_stored(p)).max() for p in psfs)
    return truth * (peak / m)


# ----------------------------------------------------------------------------
# the five configurations
# ----------------------------------------------------------------------------

def config1(seed: int = 1001) -> Workload:
    """32^3, 40 Gaussian blobs + background 1, 3 views elongated along x, y, z."""
    rng = np.random.default_rng(seed)
    dims = (32, 32, 32)
    truth = blobs_truth(rng, dims, 40, (1.0, 2.0), (50.0, 200.0), 1.0)
    psfs = [gaussian_psf(1.0, 2.5, (13, 7, 7), "x"),
            gaussian_psf(1.0, 2.5, (7, 13, 7), "y"),
            gaussian_psf(1.0, 2.5, (7, 7, 13), "z")]
    views = _observe(rng, truth, psfs)
    return _finish("blobs-32x32x32-3views", dims, truth, psfs, views, 10)


def config2(seed: int = 1002) -> Workload:
    """256x256x128, 3000 ellipsoids, 4 views at 0/90/180/270 deg about y, peak 100."""
    rng = np.random.default_rng(seed)
    dims = (256, 256, 128)
    truth = ellipsoids_truth(rng, dims, 3000, (3.0, 6.0), (0.5, 1.0))
    psfs, angles = _spim_psfs(4, 1.2, 4.0, (15, 15, 41))
    truth = _scale_to_peak(truth, psfs, 100.0)
    views = _observe(rng, truth, psfs)
    return _finish("ellipsoids-256x256x128-4views", dims, truth, psfs, views, 20,
                   angles=angles)


def config3(seed: int = 1003, dims=(1024, 1024, 512), n_objects=150_000) -> Workload:
    """1024x1024x512, 150k ellipsoids, 7 views at k*51.43 deg, peak 200 + background 5.

    Every view is blurred once: with B_v the exact blur of the unscaled
    objects, the truth is s * objects + 5 (s puts the brightest blurred
    voxel of any view at 200 photons) and its image is s * B_v + 5 (the PSFs
    sum to 1), drawn as Poisson counts.
    """
    rng = np.random.default_rng(seed)
    objects = ellipsoids_truth(rng, dims, n_objects, (3.0, 6.0), (0.5, 1.0), workers=os.cpu_count() or 1)
    psfs, angles = _spim_psfs(7, 1.5, 5.0, (19, 19, 51))
    blurred = [image_exact(objects, _as_stored(p)).astype(np.float32) for p in psfs]
    scale = 200.0 / max(float(b.max()) for b in blurred)
    views = []
    for i in range(len(blurred)):
        lam = blurred[i].astype(np.float64) * scale + 5.0
        blurred[i] = None
        views.append(rng.poisson(lam).astype(np.float32))
        del lam
    truth = objects * scale + 5.0
    return _finish("ellipsoids-1024x1024x512-7views", dims, truth, psfs, views, 10,
                   angles=angles, box=(19, 19, 51))


def config4_layout(seed: int = 1004, n_volumes: int = 48):
    """Sizes, view counts and peak photon counts of the batched volumes.

    Each axis is drawn log-uniformly (x, y in [48, 320], z in [48, 192]) and
    rounded to the nearest {2,3,5}-smooth integer; views U{2..6}; peak
    U(50, 300) photons.
    """
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_volumes):
        X = smooth235(int(round(math.exp(rng.uniform(math.log(48), math.log(320))))))
        Y = smooth235(int(round(math.exp(rng.uniform(math.log(48), math.log(320))))))
        Z = smooth235(int(round(math.exp(rng.uniform(math.log(48), math.log(192))))))
        out.append(((X, Y, Z), int(rng.integers(2, 7)), float(rng.uniform(50.0, 300.0))))
    return out


def _batch_volume(args):
    seed, b, dims, n_views, peak = args
    rng = np.random.default_rng([seed, b])
    X, Y, Z = dims
    # object density as in the 256x256x128 case (3000 per 8.4e6 voxels)
    n_obj = max(8, int(round(3000 * X * Y * Z / (256 * 256 * 128))))
    truth = ellipsoids_truth(rng, dims, n_obj, (3.0, 6.0), (0.5, 1.0))
    psfs, angles = _spim_psfs(n_views, 1.2, 4.0, (15, 15, 41))
    truth = _scale_to_peak(truth, psfs, peak)
    views = _observe(rng, truth, psfs)
    return _finish(f"batch{b:02d}-{X}x{Y}x{Z}-{n_views}views", dims, truth, psfs,
                   views, 15, angles=angles, peak=peak)


def config4(seed: int = 1004, n_volumes: int = 48, only=None, workers: int = 1):
    """48 independent volumes: log-uniform sizes, 2-6 views, peak 50-300 photons.

    ``only``: indices of the volumes to generate (default all); volume b's
    objects and noise use ``default_rng([seed, b])`` so any subset is
    reproducible on its own. ``workers > 1`` generates the volumes in a
    spawned process pool (the calling program's main module must be
    import-safe); the result is identical.
    """
    jobs = [(seed, b, dims, n_views, peak) for b, (dims, n_views, peak) in enumerate(config4_layout(seed, n_volumes))
            if only is None or b in only]
    if workers > 1 and len(jobs) > 1:
        import multiprocessing as mp

        # largest volumes first, so the pool's tail is short
        order = sorted(range(len(jobs)), key=lambda i: -int(np.prod(jobs[i][2])))
        with mp.get_context("spawn").Pool(min(workers, len(jobs))) as pool:
            done = pool.map(_batch_volume, [jobs[i] for i in order], chunksize=1)
        out = [None] * len(jobs)
        for i, w in zip(order, done):
            out[i] = w
        return out
    return [_batch_volume(j) for j in jobs]


SIGMA_TRUE = (1.2, 4.0)


def config5_sigmas(n_views: int = 4):
    """Initial learnable (sigma_xy, sigma_ax) per view: 0.8x / 1.2x of the truth, alternating."""
    f = [0.8 if v % 2 == 0 else 1.2 for v in range(n_views)]
    return [(SIGMA_TRUE[0] * s, SIGMA_TRUE[1] * s) for s in f]


def config5(seed: int = 1005) -> Workload:
    """128x128x96, 800 ellipsoids, 4 views as the 256x256x128 case, 8 unrolled iterations."""
    rng = np.random.default_rng(seed)
    dims = (128, 128, 96)
    truth = ellipsoids_truth(rng, dims, 800, (3.0, 6.0), (0.5, 1.0))
    psfs, angles = _spim_psfs(4, *SIGMA_TRUE, (15, 15, 41))
    truth = _scale_to_peak(truth, psfs, 100.0)
    views = _observe(rng, truth, psfs)
    return _finish("ellipsoids-128x128x96-4views-unrolled", dims, truth, psfs, views, 8,
                   angles=angles, box=(15, 15, 41), sigma_true=SIGMA_TRUE)


def config5_crop(seed: int = 1055) -> Workload:
    """24^3 copy for finite differences: 20 ellipsoids, 4 views, box 7x7x13."""
    rng = np.random.default_rng(seed)
    dims = (24, 24, 24)
    truth = ellipsoids_truth(rng, dims, 20, (3.0, 6.0), (0.5, 1.0))
    psfs, angles = _spim_psfs(4, *SIGMA_TRUE, (7, 7, 13))
    truth = _scale_to_peak(truth, psfs, 100.0)
    views = _observe(rng, truth, psfs)
    return _finish("ellipsoids-24x24x24-4views-unrolled", dims, truth, psfs, views, 8,
                   angles=angles, box=(7, 7, 13), sigma_true=SIGMA_TRUE)


def small_case(seed: int, dims=(16, 12, 10), n_views=2, boxes=None, n_iter=3,
               peak=80.0, asymmetric=False) -> Workload:
    """Small random problem for parity sweeps (any dims, any odd boxes).

    With ``asymmetric`` the PSFs are Gaussians with shifted means, so that the
    mirror ``P(-x)`` differs from ``P(x)``.
    """
    rng = np.random.default_rng(seed)
    X, Y, Z = dims
    n_obj = max(3, X * Y * Z // 400)
    truth = blobs_truth(rng, dims, n_obj, (0.8, 1.6), (20.0, 100.0), 0.5)
    if boxes is None:
        boxes = [(5, 3, 7), (3, 5, 5), (7, 3, 3), (5, 5, 3)][:n_views]
    psfs = []
    for v, b in enumerate(boxes):
        Kx, Ky, Kz = b
        dz, dy, dx = np.meshgrid(np.arange(Kz) - (Kz - 1) / 2, np.arange(Ky) - (Ky - 1) / 2,
                                 np.arange(Kx) - (Kx - 1) / 2, indexing="ij")
        mu = rng.uniform(-0.6, 0.6, size=3) if asymmetric else np.zeros(3)
        s = rng.uniform(0.7, 1.6, size=3)
        p = np.exp(-0.5 * (((dx - mu[0]) / s[0]) ** 2 + ((dy - mu[1]) / s[1]) ** 2
                           + ((dz - mu[2]) / s[2]) ** 2))
        psfs.append(p / p.sum())
    truth = _scale_to_peak(truth, psfs, peak)
    views = _observe(rng, truth, psfs)
    return _finish(f"small-{X}x{Y}x{Z}-{n_views}views", dims, truth, psfs, views, n_iter)
