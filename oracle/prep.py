"""Pre-reconstruction stages in front of the BST path (FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Normalization (Sec. 1 (a)): the sinogram from photon counts I, flat field
I0 and dark field D, y = -log[(I - D) / (I0 - D)].  Reading: numerator and
denominator are clamped to at least 1e-6 before the ratio (the paper is
silent on non-positive differences).

Centering (Sec. 1 (b)): the measured sinogram is y(t - beta, theta) for an
unknown rotation-axis offset beta; with beta known (in detector samples) the
centered sinogram y(t) = y_meas(t + beta) is formed as the exact band-limited
shift on the padded ray grid: the P3 spectrum is multiplied by
exp(+2 pi i k beta / M) (k the signed frequency).  For integer beta this is a
circular shift of the padded ray by beta samples.

Window (stage P1 of Sec. 2): the centered rays are multiplied by a
Kaiser-Bessel window w(t) = I0(b sqrt(1 - (t/h)^2)) / I0(b) for |t| <= h
(0 outside), shape b and half-width h in detector units (the paper names the
window but gives no parameters).  Because the window acts on the centered
coordinate, it is applied to the measured rays as w(t - beta dt).
"""
from __future__ import annotations

import numpy as np

from . import bst as ob

CLAMP = 1e-6


def normalize(counts, flat, dark=None) -> np.ndarray:
    """y = -log[(I - D) / (I0 - D)] with both differences clamped to >= 1e-6."""
    counts = np.asarray(counts, dtype=np.float64)
    flat = np.asarray(flat, dtype=np.float64)
    dark = 0.0 if dark is None else np.asarray(dark, dtype=np.float64)
    return -np.log(np.maximum(counts - dark, CLAMP) / np.maximum(flat - dark, CLAMP))


def kaiser_bessel(t, beta: float, half: float) -> np.ndarray:
    """w(t) = I0(beta sqrt(1 - (t/half)^2)) / I0(beta) on |t| <= half, else 0 (stage P1)."""
    t = np.asarray(t, dtype=np.float64)
    inside = np.abs(t) <= half
    arg = beta * np.sqrt(np.maximum(1.0 - (t / half) ** 2, 0.0))
    return np.where(inside, np.i0(arg) / np.i0(beta), 0.0)


def window_on_measured(N: int, shift: float, beta: float, half: float) -> np.ndarray:
    """The P1 window at the measured detector samples t_i = (i - N/2) dt.

    The window is centred on the rotation axis (Sec. 1 (b)): a measured
    sample at t_i sits at t_i - shift*dt in centred coordinates, so it is
    weighted by w(t_i - shift*dt)."""
    t = (np.arange(N) - N // 2) * (2.0 / N)
    return kaiser_bessel(t - shift * (2.0 / N), beta, half)


def prepared_fbp(sino, angles, pad_factor: int = 2, g=None, flat=None, dark=None, shift: float = 0.0,
                 kb_beta: float = 0.0, kb_half: float = 1.0, mode: str = ob.FILTER, grid_width: int = 0):
    """BST FBP of one slice after the pre-reconstruction stages.

    sino: counts [V][N] when ``flat`` (I0, broadcast to [V][N]) is given, else y.
    ``flat``/``dark`` may be per-detector [N] rows (one slice's detector row).
    grid_width > 0: stage P5 by Kaiser-Bessel gridding of that width (oracle.kb)."""
    s = np.asarray(sino, dtype=np.float64)
    V, N = s.shape
    M = pad_factor * N
    y = normalize(s, flat, dark) if flat is not None else s
    if kb_beta > 0.0:
        y = y * window_on_measured(N, shift, kb_beta, kb_half)[None, :]
    Y = ob.ray_spectrum(y, M)
    if shift != 0.0:
        Y = Y * np.exp(2j * np.pi * ob.signed_index(M) * shift / M)[None, :]
    if grid_width > 0:
        from . import kb
        return kb.kb_from_spectrum(Y, angles, N, mode, g, grid_width)
    return ob.bst_from_spectrum(Y, angles, N, mode, g)
