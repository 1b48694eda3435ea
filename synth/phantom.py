"""Seeded ellipse phantoms, closed-form sinograms and noise (FP64, numpy).

Geometry shared by every part of this repository:

* detector samples  t_i = (i - N/2) * dt,  i = 0..N-1,  dt = 2/N  (t in [-1, 1));
* image samples     volume[r][c] at u = (u1, u2) = ((c - N/2) * d, (r - N/2) * d),
  d = dt, so the column index follows u1 and the row index follows u2;
* projection angle  theta with direction xi = (cos theta, sin theta); at
  theta = 0 the detector coordinate is t = u1 (Eq. 1).

The paper evaluates on an analytic ellipsoid whose Radon transform is known in
closed form (Sec. 4 footnote, Kak & Slaney).  For one ellipse with centre c,
semi-axes (a, b), rotation psi and density rho the parallel projection is

    y(t, theta) = 2 rho a b sqrt(a_th^2 - s^2) / a_th^2   for |s| < a_th, else 0,
    s = t - c . xi(theta),  a_th^2 = a^2 cos^2(theta - psi) + b^2 sin^2(theta - psi).

Measurement noise follows the Lambert-Beer law I = I0 exp(-y) of Sec. 1
(Poisson photon counts, then -log), or is additive Gaussian.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

BASE_SEED = 1704083640


def slice_seed(config_index: int, slice_index: int) -> int:
    """Seed of one slice of one workload: base + config * 10^6 + slice."""
    return BASE_SEED + int(config_index) * 10**6 + int(slice_index)


@dataclass(frozen=True)
class Ellipse:
    cx: float
    cy: float
    a: float
    b: float
    psi: float
    rho: float


def uniform_angles(V: int) -> np.ndarray:
    """theta_j = j*pi/V, j = 0..V-1, rounded to float32 (the C-ABI's type)."""
    return (np.arange(V, dtype=np.float64) * (np.pi / V)).astype(np.float32)


def shepp_style_ellipses(rng: np.random.Generator) -> list[Ellipse]:
    """Ten-ellipse head-like phantom built by a seeded rule of this repository.

    One outer shell, one inner negative shell and eight small features on a
    ring, every parameter jittered by +-5 %.  The layout is a rule written
    here, not a transcription of any published table.
    """
    def jit(x: float) -> float:
        return float(x) * (1.0 + 0.05 * rng.uniform(-1.0, 1.0))

    out = [
        Ellipse(0.0, 0.0, jit(0.70), jit(0.90), 0.0, jit(1.0)),
        Ellipse(0.0, jit(-0.015), jit(0.66), jit(0.86), 0.0, jit(-0.8)),
    ]
    for k in range(8):
        phi = 2.0 * np.pi * k / 8.0 + np.pi / 16.0
        r = 0.22 + 0.06 * (k % 3)
        a = 0.05 + 0.02 * (k % 4)
        b = 0.08 + 0.02 * ((k + 1) % 3)
        psi = k * np.pi / 8.0
        sign = -1.0 if k % 2 else 1.0
        dens = sign * 0.1 * (1 + k % 3)
        out.append(Ellipse(jit(r * np.cos(phi)), jit(r * np.sin(phi)), jit(a), jit(b),
                           psi + 0.05 * np.pi * rng.uniform(-1.0, 1.0), jit(dens)))
    return out


def random_ellipses(rng: np.random.Generator, fov_safe: bool = False,
                    kmin: int = 5, kmax: int = 20) -> list[Ellipse]:
    """K ~ U{kmin..kmax} ellipses: centres uniform in the unit disk, semi-axes
    U[0.05, 0.4], rotation U[0, pi), density U[-0.5, 1].

    With ``fov_safe`` the centre radius is scaled by (0.95 - max(a, b)) so that
    every ellipse lies inside the detector's field of view (used where the
    reconstruction is compared with the phantom image itself).
    """
    K = int(rng.integers(kmin, kmax + 1))
    out = []
    for _ in range(K):
        r = np.sqrt(rng.uniform(0.0, 1.0))
        phi = rng.uniform(0.0, 2.0 * np.pi)
        a = rng.uniform(0.05, 0.4)
        b = rng.uniform(0.05, 0.4)
        psi = rng.uniform(0.0, np.pi)
        rho = rng.uniform(-0.5, 1.0)
        if fov_safe:
            r *= 0.95 - max(a, b)
        out.append(Ellipse(r * np.cos(phi), r * np.sin(phi), a, b, psi, rho))
    return out


def detector_coords(N: int) -> np.ndarray:
    return (np.arange(N, dtype=np.float64) - N // 2) * (2.0 / N)


def ellipse_sinogram(ellipses, angles, N: int) -> np.ndarray:
    """Closed-form parallel-beam sinogram [V][N] (FP64) of a sum of ellipses."""
    th = np.asarray(angles, dtype=np.float64)[:, None]
    t = detector_coords(N)[None, :]
    y = np.zeros((th.shape[0], N), dtype=np.float64)
    for e in ellipses:
        s = t - (e.cx * np.cos(th) + e.cy * np.sin(th))
        a2 = (e.a * np.cos(th - e.psi)) ** 2 + (e.b * np.sin(th - e.psi)) ** 2
        inside = s * s < a2
        chord = np.where(inside, np.sqrt(np.maximum(a2 - s * s, 0.0)), 0.0)
        y += 2.0 * e.rho * e.a * e.b * chord / a2
    return y


def ellipse_image(ellipses, N: int, supersample: int = 1) -> np.ndarray:
    """Phantom image [N][N] sampled at pixel centres (cell-averaged when
    ``supersample`` > 1, over an s x s grid inside each pixel)."""
    d = 2.0 / N
    img = np.zeros((N, N), dtype=np.float64)
    offs = ((np.arange(supersample) + 0.5) / supersample - 0.5) * d
    base = (np.arange(N, dtype=np.float64) - N // 2) * d
    for oy in offs:
        for ox in offs:
            u1 = (base + ox)[None, :]
            u2 = (base + oy)[:, None]
            for e in ellipses:
                x = u1 - e.cx
                yv = u2 - e.cy
                cp, sp = np.cos(e.psi), np.sin(e.psi)
                p = (x * cp + yv * sp) / e.a
                q = (-x * sp + yv * cp) / e.b
                img += np.where(p * p + q * q <= 1.0, e.rho, 0.0)
    return img / (supersample * supersample)


def gaussian_blob_sinogram(centre, width: float, amp: float, angles, N: int) -> np.ndarray:
    """Projection of amp*exp(-|u-a|^2/(2 s^2)): amp*sqrt(2 pi)*s*exp(-(t-a.xi)^2/(2 s^2))."""
    th = np.asarray(angles, dtype=np.float64)[:, None]
    t = detector_coords(N)[None, :]
    s0 = centre[0] * np.cos(th) + centre[1] * np.sin(th)
    return amp * np.sqrt(2.0 * np.pi) * width * np.exp(-((t - s0) ** 2) / (2.0 * width * width))


def gaussian_blob_image(centre, width: float, amp: float, N: int) -> np.ndarray:
    base = (np.arange(N, dtype=np.float64) - N // 2) * (2.0 / N)
    u1 = base[None, :]
    u2 = base[:, None]
    return amp * np.exp(-((u1 - centre[0]) ** 2 + (u2 - centre[1]) ** 2) / (2.0 * width * width))


def poisson_log_noise(y: np.ndarray, rng: np.random.Generator, photons: float = 1e4) -> np.ndarray:
    """Counts ~ Poisson(I0 exp(-y)) clamped to >= 1, then y = -log(count / I0)."""
    lam = photons * np.exp(-np.asarray(y, dtype=np.float64))
    counts = np.maximum(rng.poisson(lam), 1).astype(np.float64)
    return -np.log(counts / photons)


def gaussian_noise(y: np.ndarray, rng: np.random.Generator, frac: float = 0.01) -> np.ndarray:
    """Additive Gaussian noise with sigma = frac * max|y| of this slice."""
    sigma = frac * float(np.max(np.abs(y))) if y.size else 0.0
    return y + rng.normal(0.0, sigma, size=y.shape)


def ellipse_table(ellipse_lists, kmax: int = 20) -> tuple[np.ndarray, np.ndarray]:
    """Pack per-slice ellipse lists into float32 [S][kmax][6] plus int32 counts
    (cx, cy, a, b, psi, rho) for the device-side sinogram generator."""
    S = len(ellipse_lists)
    tab = np.zeros((S, kmax, 6), dtype=np.float32)
    cnt = np.zeros((S,), dtype=np.int32)
    for s, lst in enumerate(ellipse_lists):
        cnt[s] = len(lst)
        for k, e in enumerate(lst):
            tab[s, k] = (e.cx, e.cy, e.a, e.b, e.psi, e.rho)
    return tab, cnt
