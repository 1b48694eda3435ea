"""Pins of the pre-reconstruction oracle: normalization (Sec. 1 (a)) inverts
the Lambert-Beer law exactly, integer centering shifts (Sec. 1 (b)) equal
array shifts, a fractional shift undoes a rotation-axis offset of a closed-
form projection, and the window (P1) with b = 0 over the whole detector is
the identity."""
import numpy as np

import synth
from oracle import bst as ob
from oracle import prep


def test_normalization_inverts_lambert_beer(rng):
    y = rng.uniform(0.0, 3.0, (8, 32))
    flat = rng.uniform(900, 1100, 32)
    dark = rng.uniform(5, 20, 32)
    counts = (flat - dark) * np.exp(-y) + dark      # I = D + (I0 - D) e^{-y}
    np.testing.assert_allclose(prep.normalize(counts, flat, dark), y, rtol=0, atol=1e-12)


def test_integer_shift_equals_array_shift(rng):
    N, V, beta = 32, 24, 3
    th = synth.uniform_angles(V)
    y = rng.standard_normal((V, N))
    y[:, :beta] = 0.0   # samples shifted past t = -1 stay on the padded grid; none here
    shifted = np.zeros_like(y)
    shifted[:, : N - beta] = y[:, beta:]             # y_c[i] = y[i + beta]
    a = prep.prepared_fbp(y, th, shift=beta)
    b = ob.fbp(shifted, th)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


def test_fractional_shift_recovers_offset_projection():
    """Measured rays y(t - beta dt) of a Gaussian blob; centering by beta
    reconstructs the blob as well as the unshifted data does."""
    N = 128
    th = synth.uniform_angles(N)
    beta = 2.37
    ref = synth.gaussian_blob_image((0.3, -0.2), 0.08, 1.0, N)
    t = synth.detector_coords(N)
    c = 0.3 * np.cos(th.astype(np.float64))[:, None] - 0.2 * np.sin(th.astype(np.float64))[:, None]
    meas = np.sqrt(2 * np.pi) * 0.08 * np.exp(-((t[None, :] - beta * 2.0 / N) - c) ** 2 / (2 * 0.08 ** 2))
    x = prep.prepared_fbp(meas, th, shift=beta)
    x0 = ob.fbp(synth.gaussian_blob_sinogram((0.3, -0.2), 0.08, 1.0, th, N), th)
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < 0.025
    assert np.linalg.norm(x - x0) / np.linalg.norm(ref) < 2e-3
    bad = ob.fbp(meas, th)                           # uncorrected offset is visibly wrong
    assert np.linalg.norm(bad - ref) / np.linalg.norm(ref) > 0.2


def test_flat_window_is_identity(rng):
    N, V = 32, 20
    th = synth.uniform_angles(V)
    y = rng.standard_normal((V, N))
    a = prep.prepared_fbp(y, th, kb_beta=1e-12, kb_half=10.0)
    np.testing.assert_allclose(a, ob.fbp(y, th), rtol=0, atol=1e-9 * np.abs(a).max())
    w = prep.kaiser_bessel(np.array([0.0, 0.5, 1.0, 1.5]), 4.0, 1.0)
    assert w[0] == 1.0 and 0 < w[2] < w[1] < 1 and w[3] == 0.0
