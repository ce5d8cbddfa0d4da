"""Seeded synthetic inputs for multi-view deconvolution workloads.

This package holds the imaging model only (ground-truth objects, Gaussian
PSFs, the microscope's blur and Poisson photon noise). It holds none of the
deconvolution method's arithmetic; both the FP64 oracle and the CUDA path
consume what it produces.
"""
from .workloads import (  # noqa: F401
    Workload,
    gaussian_psf,
    rotated_box,
    smooth235,
    config1,
    config2,
    config3,
    config4,
    config5,
    config5_crop,
    small_case,
)
from .device import DeviceWorkload, config3_device  # noqa: F401
