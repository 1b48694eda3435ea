"""Pins of the pre-reconstruction oracle: normalization (Sec. 1 (a)) inverts
the Lambert-Beer law exactly, integer centering shifts (Sec. 1 (b)) equal
array shifts, a fractional shift undoes a rotation-axis offset of a closed-
form projection, and the window (P1) with b = 0 over the whole detector is
the identity.

The Kaiser-Bessel window of stage P1 (Sec. 2) is pinned by mathematics that
does not use the oracle's formula: its continuous Fourier transform has the
closed form 2h sinh(sqrt(b^2 - (2 pi h f)^2)) / sqrt(b^2 - (2 pi h f)^2)
divided by I0(b) (sin in place of sinh past the main lobe), evaluated here
with I0 from its power series; its peak is 1; it vanishes past h.  Its
placement on measured rays under a centering shift (Sec. 1 (b)) is pinned
by the integer-shift identity: windowing the measured rays at w(t - beta dt)
and shifting back equals shifting first and windowing at the centred
coordinate."""
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


def i0_series(x: float) -> float:
    """Modified Bessel function I0 from its defining power series
    sum_k (x^2/4)^k / (k!)^2 (Abramowitz and Stegun 9.6.12)."""
    total, term, k = 0.0, 1.0, 0
    while term > 1e-18 * (total + term):
        total += term
        k += 1
        term *= (x * x / 4.0) / (k * k)
    return total + term


def window_transform_error() -> float:
    """Largest deviation of the window's Fourier transform (Gauss-Legendre
    quadrature of the oracle's window; the integrand is analytic in t, since
    I0 is even) from its closed form, relative to the transform at f = 0."""
    xg, wg = np.polynomial.legendre.leggauss(200)
    worst = 0.0
    for b in (2.0, 6.5, 12.0):
        for h in (0.5, 0.9):
            norm = 2 * h * np.sinh(b) / b / i0_series(b)
            for f in (0.0, 0.3, 1.0, b / (2 * np.pi * h) * 0.999, 3.0, 7.5):
                t = h * xg
                got = h * np.sum(wg * prep.kaiser_bessel(t, b, h) * np.exp(-2j * np.pi * f * t))
                a2 = b * b - (2 * np.pi * h * f) ** 2
                a = np.sqrt(abs(a2))
                ref = 2 * h * (np.sinh(a) if a2 > 0 else np.sin(a)) / a / i0_series(b)
                worst = max(worst, abs(got - ref) / norm)
    return worst


def window_peak_error() -> float:
    """|w(0) - 1| + the largest |w| past the half-width, over several shapes."""
    err = 0.0
    for b, h in ((2.0, 0.5), (6.5, 0.9), (12.0, 1.0)):
        w = prep.kaiser_bessel(np.array([0.0, h * 1.0001, -h * 1.5, 3.0 * h]), b, h)
        err += abs(w[0] - 1.0) + np.abs(w[1:]).max()
    return err


def shifted_window_error(seed: int = 5) -> float:
    """Integer centering shift with a window: the oracle windows the measured
    rays at w(t_i - beta dt) and then shifts them back by beta; this must equal
    the plain FBP of the rays shifted first, y_c[i] = y[i + beta], windowed at
    the centred coordinate w(t_i).  Relative max error."""
    rng = np.random.default_rng(seed)
    N, V, beta, b, h = 32, 20, 3, 6.0, 0.7
    th = synth.uniform_angles(V)
    y = rng.standard_normal((V, N))
    y[:, :beta] = 0.0
    shifted = np.zeros_like(y)
    shifted[:, : N - beta] = y[:, beta:]
    wc = prep.kaiser_bessel((np.arange(N) - N // 2) * (2.0 / N), b, h)
    a = prep.prepared_fbp(y, th, shift=beta, kb_beta=b, kb_half=h)
    ref = ob.fbp(shifted * wc[None, :], th)
    return np.abs(a - ref).max() / np.abs(ref).max()


def test_window_fourier_transform_matches_closed_form():
    assert window_transform_error() < 1e-12


def test_window_peak_is_one_and_support_is_the_half_width():
    assert window_peak_error() < 1e-15


def test_window_is_even_and_monotone_on_the_half_width():
    t = np.linspace(0.0, 0.8, 41)
    w = prep.kaiser_bessel(t, 7.0, 0.8)
    np.testing.assert_array_equal(w, prep.kaiser_bessel(-t, 7.0, 0.8))
    assert np.all(np.diff(w) < 0)


def test_window_sits_on_the_centred_coordinate_under_integer_shift():
    assert shifted_window_error() < 1e-12


def test_window_with_fractional_shift_matches_windowed_centred_projection():
    """A Gaussian blob measured with a fractional rotation-axis offset, windowed
    and centred by the oracle, reconstructs like the centred closed-form
    projection windowed at the centred coordinate."""
    N, beta, b, h = 128, 2.37, 8.0, 0.9
    th = synth.uniform_angles(N)
    t = synth.detector_coords(N)
    th64 = th.astype(np.float64)[:, None]
    c = 0.3 * np.cos(th64) - 0.2 * np.sin(th64)
    blob = lambda tt: np.sqrt(2 * np.pi) * 0.08 * np.exp(-(tt - c) ** 2 / (2 * 0.08 ** 2))
    meas = blob(t[None, :] - beta * 2.0 / N)
    x = prep.prepared_fbp(meas, th, shift=beta, kb_beta=b, kb_half=h)
    ref = ob.fbp(blob(t[None, :]) * prep.kaiser_bessel(t, b, h)[None, :], th)
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < 2e-3
