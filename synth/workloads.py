"""The five synthetic workloads of this repository, by name and size.

Each slice is seeded independently (``slice_seed``), so any subset of slices
of a large workload can be regenerated on the host without the rest.

    single-256     1 slice,   256 angles x 256 rays, ten-ellipse head-like
                   phantom with +-5 % jitter, noiseless analytic sinogram
    volume-512     512 slices x 512 x 512, 5-20 random ellipses per slice,
                   Poisson noise at 1e4 photons/ray then -log
    volume-2048    2048 slices x 2048 x 2048, 5-20 random ellipses per slice,
                   additive Gaussian noise sigma = 1 % of the slice maximum
    ragged-64      64 sinograms, rays drawn from {256..2048}, angles = rays
    autograd-1024  16 slices x 1024 x 1024, ellipses kept inside the field of
                   view, Poisson noise; the targets are the phantom images
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .phantom import (
    ellipse_image,
    ellipse_sinogram,
    gaussian_noise,
    poisson_log_noise,
    random_ellipses,
    shepp_style_ellipses,
    slice_seed,
    uniform_angles,
)


@dataclass(frozen=True)
class Workload:
    name: str
    index: int          # seed offset of this workload
    slices: int
    angles: int
    rays: int
    noise: str          # "none" | "poisson" | "gaussian"
    fov_safe: bool


WORKLOADS = {
    "single-256": Workload("single-256", 0, 1, 256, 256, "none", True),
    "volume-512": Workload("volume-512", 1, 512, 512, 512, "poisson", False),
    "volume-2048": Workload("volume-2048", 2, 2048, 2048, 2048, "gaussian", False),
    "ragged-64": Workload("ragged-64", 3, 64, 0, 0, "poisson", False),
    "autograd-1024": Workload("autograd-1024", 4, 16, 1024, 1024, "poisson", True),
}


def slice_ellipses(w: Workload, s: int):
    rng = np.random.default_rng(slice_seed(w.index, s))
    if w.name == "single-256":
        return rng, shepp_style_ellipses(rng)
    return rng, random_ellipses(rng, fov_safe=w.fov_safe)


def workload_slices(name: str, indices, rays: int | None = None, angles: int | None = None,
                    with_images: bool = False, supersample: int = 4):
    """Host-generated slices of a workload: (theta[V] float32, sino[len][V][N] float32
    [, images[len][N][N] float64]).  ``rays``/``angles`` override the sizes."""
    w = WORKLOADS[name]
    N = rays or w.rays
    V = angles or w.angles
    theta = uniform_angles(V)
    sinos = np.zeros((len(indices), V, N), dtype=np.float32)
    imgs = np.zeros((len(indices), N, N), dtype=np.float64) if with_images else None
    for n, s in enumerate(indices):
        rng, ells = slice_ellipses(w, s)
        y = ellipse_sinogram(ells, theta, N)
        if w.noise == "poisson":
            y = poisson_log_noise(y, rng)
        elif w.noise == "gaussian":
            y = gaussian_noise(y, rng)
        sinos[n] = y.astype(np.float32)
        if with_images:
            imgs[n] = ellipse_image(ells, N, supersample)
    return theta, sinos, imgs


def ragged_sizes(count: int = 64, choices=(256, 512, 768, 1024, 1536, 2048)) -> list[int]:
    """Seeded ray counts of the ragged batch (angles = rays for each item)."""
    rng = np.random.default_rng(slice_seed(WORKLOADS["ragged-64"].index, 999_999))
    return [int(x) for x in rng.choice(np.asarray(choices), size=count)]
