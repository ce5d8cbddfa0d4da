"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-types the oracle's own formula: each compares it with an
independent computation (brute-force DFT, a library convolution, a Gaussian
closed form, a hand-worked example) or with an invariant the paper's
derivation implies (conservation, fixed point, non-negativity, EM monotone
likelihood, the single-view reduction).
"""
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_kernel(rng, shape, asym=True):
    k = rng.uniform(0.0, 1.0, size=shape)
    if asym:
        k[0, 0, 0] += 3.0  # break central symmetry
    return k / k.sum()


def _place_centred(k, shape):
    """Kernel on the periodic grid with its box centre at the origin."""
    big = np.zeros(shape)
    Kz, Ky, Kx = k.shape
    zi = (np.arange(Kz) - (Kz - 1) // 2) % shape[0]
    yi = (np.arange(Ky) - (Ky - 1) // 2) % shape[1]
    xi = (np.arange(Kx) - (Kx - 1) // 2) % shape[2]
    big[np.ix_(zi, yi, xi)] = k
    return big


def _dft_matrix(n):
    j = np.arange(n)
    return np.exp(-2j * np.pi * np.outer(j, j) / n)


def _dft3(a):
    Fz, Fy, Fx = (_dft_matrix(n) for n in a.shape)
    return np.einsum("az,by,cx,zyx->abc", Fz, Fy, Fx, a)


def _idft3(a):
    Fz, Fy, Fx = (np.conj(_dft_matrix(n)) / n for n in a.shape)
    return np.einsum("az,by,cx,zyx->abc", Fz, Fy, Fx, a)


# ---------------------------------------------------------------------------
# convolution (Eq. 51's "*")
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("shape,kshape", [((8, 8, 8), (3, 5, 7)), ((5, 6, 8), (3, 3, 5))])
def test_conv_matches_bruteforce_dft(shape, kshape):
    """Circular convolution equals IDFT(DFT(f) . DFT(k)) with explicit DFT matrices."""
    rng = np.random.default_rng(1)
    f = rng.uniform(0.0, 2.0, size=shape)
    k = _rand_kernel(rng, kshape)
    want = np.real(_idft3(_dft3(f) * _dft3(_place_centred(k, shape))))
    got = oracle.conv(f, k)
    assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(want))


def test_conv_matches_numpy_fft_nonsquare():
    rng = np.random.default_rng(2)
    shape = (9, 10, 12)
    f = rng.uniform(0.0, 1.0, size=shape)
    k = _rand_kernel(rng, (5, 3, 7))
    want = np.fft.irfftn(np.fft.rfftn(f) * np.fft.rfftn(_place_centred(k, shape)), s=shape,
                         axes=(0, 1, 2))
    assert np.allclose(oracle.conv(f, k), want, rtol=0, atol=1e-13)


def test_conv_separable_gaussian_equals_three_1d_convs():
    """An axis-aligned Gaussian is separable: 3D conv = 1D periodic convs along x, y, z."""
    rng = np.random.default_rng(3)
    shape = (10, 12, 14)
    f = rng.uniform(0.0, 1.0, size=shape)
    gx, gy, gz = (np.exp(-0.5 * (np.arange(n) - (n - 1) / 2) ** 2 / s ** 2) for n, s in
                  ((7, 1.3), (5, 0.9), (9, 2.0)))
    gx, gy, gz = gx / gx.sum(), gy / gy.sum(), gz / gz.sum()
    k = gz[:, None, None] * gy[None, :, None] * gx[None, None, :]

    def conv1d(a, g, axis):
        h = (len(g) - 1) // 2
        out = np.zeros_like(a)
        for i, w in enumerate(g):
            out += w * np.roll(a, i - h, axis=axis)
        return out

    want = conv1d(conv1d(conv1d(f, gx, 2), gy, 1), gz, 0)
    assert np.allclose(oracle.conv(f, k), want, rtol=0, atol=1e-13)


def test_mirror_is_adjoint_kernel():
    """<f * P, r> = <f, r * P^*>: integration over x is convolution with P(-x)."""
    rng = np.random.default_rng(4)
    shape = (7, 8, 9)
    f, r = rng.uniform(size=shape), rng.uniform(size=shape)
    P = _rand_kernel(rng, (3, 5, 5))
    lhs = np.sum(oracle.conv(f, P) * r)
    rhs = np.sum(f * oracle.conv(r, oracle.mirror(P)))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # and the un-mirrored kernel is NOT the adjoint for an asymmetric P
    wrong = np.sum(f * oracle.conv(r, P))
    assert abs(lhs - wrong) > 1e-6 * abs(lhs)


def test_kernel_linear_convolution_matches_scipy():
    signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(5)
    a = _rand_kernel(rng, (3, 5, 7))
    b = _rand_kernel(rng, (5, 3, 3))
    full = signal.convolve(a, b, mode="full", method="direct")
    got = oracle.kconv(a, b, full.shape)
    assert np.allclose(got, full, rtol=0, atol=1e-15)
    # centred crop to a's box
    crop = oracle.kconv(a, b, a.shape)
    oz, oy, ox = [(F - A) // 2 for F, A in zip(full.shape, a.shape)]
    assert np.allclose(crop, full[oz:oz + 3, oy:oy + 5, ox:ox + 7], atol=1e-15)


# ---------------------------------------------------------------------------
# compound kernels (Eq. 222, Eq. 230, Eq. 240)
# ---------------------------------------------------------------------------

def _hand_golden():
    vals = {}
    with open(os.path.join(GOLDEN, "hand_update_4x1x1.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            name, *nums = line.split()
            vals[name] = np.array([float(x) for x in nums])
    return vals


def _k1d(taps):
    return np.array(taps, dtype=np.float64).reshape(1, 1, 3)


def test_compound_hand_worked_example():
    g = _hand_golden()
    psfs = [_k1d([0.2, 0.8, 0.0]), _k1d([0.25, 0.5, 0.25])]
    assert np.allclose(oracle.compound(psfs, 0, "efficient").ravel(), g["efficient_comp0"], atol=1e-15)
    assert np.allclose(oracle.compound(psfs, 1, "efficient").ravel(), g["efficient_comp1"], atol=1e-15)
    assert np.allclose(oracle.compound(psfs, 0, "plain").ravel(), [0.0, 0.8, 0.2], atol=1e-16)


def test_update_hand_worked_example():
    """Two sequential RL updates on a 4x1x1 grid, worked out by hand (golden file)."""
    g = _hand_golden()
    P0, P1 = _k1d([0.2, 0.8, 0.0]), _k1d([0.25, 0.5, 0.25])
    phi0 = np.array([2.0, 0.0, 1.0, 1.0]).reshape(1, 1, 4)
    phi1 = np.ones((1, 1, 4))
    psi = np.ones((1, 1, 4))
    psi = oracle.update(psi, phi0, P0, oracle.mirror(P0), 1e-12)
    assert np.allclose(psi.ravel(), g["plain_view0"], atol=1e-15)
    psi2, _ = oracle.deconvolve([phi0, phi1], [P0, P1], 1, "plain", eps=1e-12,
                                psi_init=np.ones((1, 1, 4)))
    assert np.allclose(psi2.ravel(), g["plain_iter1"], atol=1e-14)


def test_compound_single_view_is_mirrored_psf():
    """With one view W is empty, so every variant's kernel is P^* (the RL back-projection)."""
    rng = np.random.default_rng(6)
    P = _rand_kernel(rng, (3, 5, 7))
    for var in ("plain", "efficient", "opt1", "opt2"):
        assert np.allclose(oracle.compound([P], 0, var), oracle.mirror(P), atol=1e-16)


def _sampled_gaussian(mu, cov, box):
    Kx, Ky, Kz = box
    dz, dy, dx = np.meshgrid(np.arange(Kz) - (Kz - 1) / 2, np.arange(Ky) - (Ky - 1) / 2,
                             np.arange(Kx) - (Kx - 1) / 2, indexing="ij")
    d = np.stack([dx - mu[0], dy - mu[1], dz - mu[2]], axis=-1)
    q = np.einsum("...i,ij,...j->...", d, np.linalg.inv(cov), d)
    p = np.exp(-0.5 * q)
    return p / p.sum()


def _moments(k):
    Kz, Ky, Kx = k.shape
    dz, dy, dx = np.meshgrid(np.arange(Kz) - (Kz - 1) / 2, np.arange(Ky) - (Ky - 1) / 2,
                             np.arange(Kx) - (Kx - 1) / 2, indexing="ij")
    D = np.stack([dx, dy, dz], axis=-1).reshape(-1, 3)
    w = k.ravel() / k.sum()
    mean = w @ D
    C = (D - mean).T @ ((D - mean) * w[:, None])
    return mean, C


@pytest.mark.parametrize("variant", ["efficient", "opt1", "opt2"])
def test_compound_gaussian_closed_form(variant):
    """For Gaussian PSFs N(mu_v, S_v): mirror -> N(-mu_v, S_v); convolutions add means and
    covariances; pointwise products add precisions. Hence the compound kernel of view v is
    Gaussian with precision L = S_v^-1 + sum_w A_w^-1 and mean L^-1 (S_v^-1 (-mu_v) + sum_w
    A_w^-1 m_w), where (A_w, m_w) = (S_v + 2 S_w, -mu_v) for Eq. 222, (S_v + S_w, mu_w - mu_v)
    for Eq. 230 and (S_v, -mu_v) for Eq. 240. Sampled Gaussians with sigma >= 1 reproduce the
    continuous moments to ~1e-8, so the moments must match closely."""
    rng = np.random.default_rng(7)
    box = (19, 19, 21)  # >= 5 sigma on every axis: truncation below 1e-5
    mus = [rng.uniform(-0.5, 0.5, 3) for _ in range(3)]
    covs = []
    for _ in range(3):
        A = rng.normal(size=(3, 3)) * 0.15
        S = np.diag(rng.uniform(1.5, 1.7, 3) ** 2) + A @ A.T
        covs.append(S)
    psfs = [_sampled_gaussian(m, S, box) for m, S in zip(mus, covs)]
    v = 0
    Lv = np.linalg.inv(covs[v])
    prec = Lv.copy()
    lin = Lv @ (-mus[v])
    for w in (1, 2):
        if variant == "efficient":
            A, m = covs[v] + 2 * covs[w], -mus[v]
        elif variant == "opt1":
            A, m = covs[v] + covs[w], mus[w] - mus[v]
        else:
            A, m = covs[v], -mus[v]
        Ai = np.linalg.inv(A)
        prec += Ai
        lin += Ai @ m
    cov_want = np.linalg.inv(prec)
    mean_want = cov_want @ lin
    mean, C = _moments(oracle.compound(psfs, v, variant))
    assert np.allclose(mean, mean_want, atol=2e-4)
    assert np.allclose(C, cov_want, rtol=0, atol=2e-4 * np.max(np.abs(cov_want)))


# ---------------------------------------------------------------------------
# the update and the schedule (Eq. 15, Eq. 51, Eq. 220, sequential order)
# ---------------------------------------------------------------------------

def _fft_blur(f, k):
    shape = f.shape
    return np.fft.irfftn(np.fft.rfftn(f) * np.fft.rfftn(_place_centred(k, shape)), s=shape,
                        axes=(0, 1, 2))


@pytest.mark.parametrize("variant", ["plain", "efficient", "opt1", "opt2"])
def test_noise_free_truth_is_fixed_point(variant):
    """phi_v = psi* * P_v exactly => ratio 1 => back-projection of ones is 1 => psi* fixed."""
    w = synth.small_case(11, dims=(12, 10, 14), n_views=3, asymmetric=True)
    truth = w.truth.astype(np.float64)
    psfs = [p.astype(np.float64) / p.astype(np.float64).sum() for p in w.psfs]
    views = [_fft_blur(truth, p) for p in psfs]
    psi, eps = oracle.deconvolve(views, psfs, 2, variant, psi_init=truth, eps=1e-9)
    assert np.max(np.abs(psi - truth) / truth) < 1e-11


def test_plain_update_conserves_total_intensity():
    """Sum psi after an update with view v equals sum phi_v (normalised P, exact adjoint)."""
    w = synth.small_case(12, dims=(11, 9, 13), n_views=3, asymmetric=True)
    psfs = [p.astype(np.float64) for p in w.psfs]
    psi = np.full(w.truth.shape, 7.0)
    for v in (0, 2, 1):
        psi = oracle.update(psi, w.views[v], psfs[v], oracle.mirror(psfs[v]), 1e-12)
        assert abs(psi.sum() - w.views[v].sum()) < 1e-10 * w.views[v].sum()


def test_estimate_stays_positive_and_floored():
    rng = np.random.default_rng(13)
    w = synth.small_case(13, dims=(10, 10, 10), n_views=2)
    views = [v * (rng.uniform(size=v.shape) > 0.5) for v in w.views]  # many exact zeros
    psi, eps = oracle.deconvolve(views, w.psfs, 4, "efficient")
    assert np.all(psi >= eps) and eps > 0


def test_delta_psfs_pin_the_schedule():
    """With identity (delta) PSFs every variant's update sets psi to max(phi_v, eps), so the
    result after any number of iterations is the last scheduled view."""
    rng = np.random.default_rng(14)
    shape = (6, 5, 4)
    views = [rng.uniform(1.0, 5.0, size=shape) for _ in range(3)]
    delta = np.zeros((3, 3, 3))
    delta[1, 1, 1] = 1.0
    for variant in ("plain", "efficient"):
        for sched in ([0, 1, 2], [2, 0, 1], [1, 1, 0, 2, 1]):
            psi, _ = oracle.deconvolve(views, [delta] * 3, 2, variant, schedule=sched)
            assert np.allclose(psi, views[sched[-1]], atol=1e-14)


def test_flat_initial_estimate_is_mean_of_views():
    w = synth.small_case(15, dims=(8, 9, 10), n_views=3)
    want = np.mean([v.astype(np.float64).mean() for v in w.views])
    assert abs(oracle.mean_views(w.views) - want) < 1e-12 * want
    psi, eps = oracle.deconvolve(w.views, w.psfs, 0)
    assert np.allclose(psi, want, rtol=1e-14) and abs(eps - 1e-4 * want) < 1e-16 * want


def test_single_view_rl_likelihood_is_monotone():
    """Single-view RL is an EM algorithm: the Poisson log-likelihood sum(phi log b - b)
    never decreases from one update to the next."""
    w = synth.small_case(16, dims=(10, 12, 9), n_views=1, asymmetric=True)
    P = w.psfs[0].astype(np.float64)
    phi = w.views[0].astype(np.float64)
    psi = np.full(phi.shape, phi.mean())
    prev = -np.inf
    for _ in range(12):
        b = _fft_blur(psi, P)
        ll = np.sum(np.where(phi > 0, phi * np.log(b), 0.0) - b)
        assert ll >= prev - 1e-9 * abs(ll)
        prev = ll
        psi = oracle.update(psi, phi, P, oracle.compound([P], 0, "efficient"), 1e-12)


def test_single_view_efficient_equals_plain():
    w = synth.small_case(17, dims=(9, 9, 9), n_views=1)
    a, _ = oracle.deconvolve(w.views, w.psfs, 3, "efficient")
    b, _ = oracle.deconvolve(w.views, w.psfs, 3, "plain")
    assert np.array_equal(a, b)


def test_update_at_matches_full_update():
    w = synth.small_case(18, dims=(10, 8, 12), n_views=2, asymmetric=True)
    psfs = [p.astype(np.float64) for p in w.psfs]
    K = oracle.compound(psfs, 1, "efficient")
    rng = np.random.default_rng(0)
    psi = rng.uniform(1.0, 3.0, size=w.truth.shape)
    full = oracle.update(psi, w.views[1], psfs[1], K, 1e-3)
    idx = rng.choice(psi.size, 40, replace=False)
    at = oracle.update_at(psi, w.views[1], psfs[1], K, 1e-3, idx)
    assert np.allclose(at, full.ravel()[idx], rtol=1e-13)


def test_deconvolution_improves_correlation_with_truth():
    """Qualitative smoke check (not parity): deconvolution sharpens towards the truth."""
    w = synth.config1()
    psi, _ = oracle.deconvolve(w.views, w.psfs, w.n_iter, "efficient")
    r_in = np.corrcoef(w.views[0].ravel(), w.truth.ravel())[0, 1]
    r_out = np.corrcoef(psi.ravel(), w.truth.ravel())[0, 1]
    assert r_out > r_in + 0.05


def test_psf_scale_is_irrelevant():
    """PSFs are probability distributions (Eq. 3): scaling a PSF must not change the result."""
    w = synth.small_case(19, dims=(10, 9, 8), n_views=2, asymmetric=True)
    a, _ = oracle.deconvolve(w.views, w.psfs, 2, "efficient")
    b, _ = oracle.deconvolve(w.views, [w.psfs[0] * 4.0, w.psfs[1] * 0.25], 2, "efficient")  # exact scales
    assert np.allclose(a, b, rtol=1e-12)
