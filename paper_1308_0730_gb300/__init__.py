"""GB300 (sm_103a) efficient Bayesian multi-view deconvolution.

The compute path is libmvd.so (CUDA, C ABI in include/mvd.h); ``mvd`` is its
thin Python binding.
"""
from .mvd import (  # noqa: F401
    Deconvolver,
    MvdError,
    load,
    mvd_create,
    mvd_precompute_kernels,
    mvd_set_estimate,
    mvd_iterate,
    mvd_iterate_combined,
    mvd_result,
    mvd_result_device,
    mvd_synchronize,
    mvd_destroy,
    mvd_last_error,
    mvd_launch_count,
    mvd_get_eps,
    mvd_get_psi0,
    mvd_get_path,
    mvd_get_compound_kernel,
    mvd_profile_enable,
    mvd_profile_read,
    mvd_batch_create,
    mvd_batch_run,
    mvd_batch_wait,
    mvd_batch_tasks,
    mvd_batch_destroy,
    mvd_batch_mode,
    mvd_autotune,
    mvd_unrolled_forward,
    mvd_unrolled_backward,
    mvd_gaussian_psf,
    mvd_gaussian_psf_vjp,
)
