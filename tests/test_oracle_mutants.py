"""Planted mistakes in the oracle must be caught by its pins.

Each case patches one plausible mistake into a stage of oracle.bst (on the
CPU, inside the test only) and checks that a pin which passes on the real
oracle fails on the mutant."""
import numpy as np
import pytest

import synth
from oracle import bst as ob


def _blob_error(N=64):
    th = synth.uniform_angles(N)
    y = synth.gaussian_blob_sinogram((0.3, -0.2), 0.08, 1.0, th, N)
    ref = synth.gaussian_blob_image((0.3, -0.2), 0.08, 1.0, N)
    return np.linalg.norm(ob.fbp(y, th) - ref) / np.linalg.norm(ref)


def _bilinear_error():
    M, V = 64, 24
    th = synth.uniform_angles(V)
    t64 = th.astype(np.float64)
    k = ob.signed_index(M).astype(np.float64)
    Z = 0.7 - 0.03 * k[None, :] + 0.4 * t64[:, None] + 0.011 * k[None, :] * t64[:, None]
    X = ob.grid(Z.astype(np.complex128), th)
    C, R = np.meshgrid(k, k)
    rho = np.hypot(C, R)
    up = (R > 0) | ((R == 0) & (C >= 0))
    theta = np.arctan2(np.where(up, R, -R), np.where(up, C, -C))
    kappa = np.where(up, rho, -rho)
    ok = (rho < M / 2 - 1) & (theta >= t64[0]) & (theta < t64[-1])
    expect = 0.7 - 0.03 * kappa + 0.4 * theta + 0.011 * kappa * theta
    return np.abs(X[ok].real - expect[ok]).max()


def _imag_ratio():
    rng = np.random.default_rng(2)
    V, N = 28, 32
    th = np.sort(rng.uniform(0.05, 3.1, V)).astype(np.float32)
    _, xp = ob.bst(rng.standard_normal((V, N)), th, 2, ob.FILTER, return_pad=True)
    return np.abs(xp.imag).max() / np.abs(xp.real).max()


def _disk_level():
    N = 64
    th = synth.uniform_angles(N)
    x = ob.fbp(synth.ellipse_sinogram([synth.Ellipse(0, 0, 0.3, 0.3, 0, 1.0)], th, N), th)
    base = (np.arange(N) - N // 2) * (2.0 / N)
    m = np.hypot(base[None, :], base[:, None]) <= 0.15
    return abs(x[m].mean() - 1.0)


def test_pins_pass_on_the_real_oracle():
    assert _blob_error() < 0.025
    assert _bilinear_error() < 1e-11
    assert _imag_ratio() < 1e-13
    assert _disk_level() < 0.01
    from test_oracle_bst import linear_spectrum_error
    th = np.sort(np.random.default_rng(2).uniform(0.03, 3.1, 40)).astype(np.float32)
    assert linear_spectrum_error(th) <= 0.0
    from test_oracle_prep import shifted_window_error, window_peak_error, window_transform_error
    assert window_transform_error() < 1e-12
    assert window_peak_error() < 1e-15
    assert shifted_window_error() < 1e-12


def _swap_taps(pairs):
    real = ob.polar_taps

    def patched(M, angles, rows=None):
        jr, kb, w = real(M, angles, rows)
        w = w.copy()
        for a, b in pairs:
            w[[a, b]] = w[[b, a]]
        return jr, kb, w
    return patched


@pytest.mark.parametrize("name", ["angle_fraction_reversed", "radial_fraction_reversed",
                                  "image_transposed", "exponent_sign_flipped",
                                  "dt_dropped", "seam_without_negation"])
def test_planted_mistake_is_caught(name, monkeypatch):
    if name == "angle_fraction_reversed":
        monkeypatch.setattr(ob, "polar_taps", _swap_taps([(0, 2), (1, 3)]))
        assert _bilinear_error() > 1e-3
    elif name == "radial_fraction_reversed":
        monkeypatch.setattr(ob, "polar_taps", _swap_taps([(0, 1), (2, 3)]))
        assert _bilinear_error() > 1e-3
    elif name == "image_transposed":
        real = ob.image_from_grid
        monkeypatch.setattr(ob, "image_from_grid", lambda X, N, direct=False: (real(X, N, direct)[0].T, None))
        assert _blob_error() > 0.5
    elif name == "exponent_sign_flipped":
        real = ob.ray_spectrum
        monkeypatch.setattr(ob, "ray_spectrum", lambda y, M, direct=False: np.conj(real(y, M, direct)))
        assert _blob_error() > 0.5
    elif name == "dt_dropped":
        real = ob.ray_spectrum
        monkeypatch.setattr(ob, "ray_spectrum", lambda y, M, direct=False: real(y, M, direct) * (y.shape[-1] / 2.0))
        assert _disk_level() > 0.5
    elif name == "seam_without_negation":
        real = ob.polar_taps

        def patched(M, angles, rows=None):
            jr, kb, w = real(M, angles, rows)
            V = ob.angles64(angles).size
            # pretend the seam rows were read at +k instead of -k: undo the flip on row 0 / V-1
            # taps whose virtual row was V or -1 (the last two taps of bracket V-1, the first two of -1)
            r_idx = np.arange(M) if rows is None else np.asarray(rows)
            sg = ob.signed_index(M)
            R = sg[r_idx][:, None] * np.ones((1, M))
            C = np.ones((r_idx.size, 1)) * sg[None, :]
            up = (R > 0) | ((R == 0) & (C >= 0))
            theta = np.arctan2(np.where(up, R, -R), np.where(up, C, -C))
            J = np.searchsorted(ob.angles64(angles), theta, side="right") - 1
            kb = kb.copy()
            kb[2:][:, J == V - 1] *= -1
            kb[:2][:, J == -1] *= -1
            return jr, kb, w
        monkeypatch.setattr(ob, "polar_taps", patched)
        from test_oracle_bst import linear_spectrum_error
        th = np.sort(np.random.default_rng(2).uniform(0.03, 3.1, 40)).astype(np.float32)
        assert linear_spectrum_error(th) > 1.0


@pytest.mark.parametrize("name", ["window_sqrt_dropped", "window_shift_sign_flipped",
                                  "window_normalised_twice"])
def test_planted_window_mistake_is_caught(name, monkeypatch):
    """Stage P1 (Sec. 2) and its placement under centering (Sec. 1 (b))."""
    from oracle import prep
    from test_oracle_prep import shifted_window_error, window_peak_error, window_transform_error
    if name == "window_sqrt_dropped":
        def mutant(t, beta, half):
            t = np.asarray(t, dtype=np.float64)
            arg = beta * np.maximum(1.0 - (t / half) ** 2, 0.0)
            return np.where(np.abs(t) <= half, np.i0(arg) / np.i0(beta), 0.0)
        monkeypatch.setattr(prep, "kaiser_bessel", mutant)
        assert window_transform_error() > 1e-3
    elif name == "window_shift_sign_flipped":
        def mutant(N, shift, beta, half):
            t = (np.arange(N) - N // 2) * (2.0 / N)
            return prep.kaiser_bessel(t + shift * (2.0 / N), beta, half)
        monkeypatch.setattr(prep, "window_on_measured", mutant)
        assert shifted_window_error() > 1e-2
    elif name == "window_normalised_twice":
        real = prep.kaiser_bessel
        monkeypatch.setattr(prep, "kaiser_bessel", lambda t, beta, half: real(t, beta, half) / np.i0(beta))
        assert window_peak_error() > 0.1
        assert window_transform_error() > 1e-3
