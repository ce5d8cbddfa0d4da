"""FP64 CPU oracle for efficient Bayesian multi-view deconvolution.

TEST INFRASTRUCTURE ONLY: tests, the smoke check and the benchmark's
CPU-baseline leg may import this package; the product path never does. It
shares no code with the CUDA path.
"""
from .oracle import (  # noqa: F401
    PLAIN,
    EFFICIENT,
    OPT1,
    OPT2,
    VARIANTS,
    build,
    conv,
    conv_zero,
    conv_mirror,
    backproject_mirror,
    mirror,
    kconv,
    compound,
    update,
    update_at,
    deconvolve,
    deconvolve_fft,
    conv_fft,
    grid_spectrum,
    deconvolve_combined,
    deconvolve_zero,
    deconvolve_mirror,
    deconvolve_weighted,
    normalize_weights,
    WEIGHT_NORMS,
    mean_views,
    num_threads,
    unrolled_grad,
)
