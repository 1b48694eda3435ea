"""Seeded synthetic inputs for the BST filtered-backprojection path.

This package holds the input generators shared by the CPU oracle, the GPU
parity tests and the benchmark: ellipse phantoms (the paper's workload is an
analytic ellipsoid, Sec. 4 footnote, following Kak & Slaney), their
closed-form parallel-beam sinograms (Eq. 1 applied to an ellipse), angle
lists and measurement noise (Lambert-Beer law, Sec. 1 "Description of the
problem").  It contains none of the backprojection method's arithmetic.
"""
from .phantom import (  # noqa: F401
    BASE_SEED,
    Ellipse,
    uniform_angles,
    shepp_style_ellipses,
    random_ellipses,
    ellipse_sinogram,
    ellipse_image,
    gaussian_blob_sinogram,
    gaussian_blob_image,
    poisson_log_noise,
    gaussian_noise,
    slice_seed,
    ellipse_table,
    detector_coords,
)
from .workloads import WORKLOADS, workload_slices, ragged_sizes  # noqa: F401
