"""Pins of the step-by-step BST oracle (Theorem 2.1 / Eq. 3, stages P0-P8)."""
import numpy as np
import pytest

import synth
from oracle import brute
from oracle import bst as ob


def _radius(N):
    base = (np.arange(N) - N // 2) * (2.0 / N)
    return np.hypot(base[None, :], base[:, None])


def _nonuniform(rng, V, lo=0.05):
    return np.sort(rng.uniform(lo, np.pi - 0.01, V)).astype(np.float32)


@pytest.mark.parametrize("N,V,alpha", [(8, 6, 2), (16, 12, 2), (12, 10, 2), (16, 16, 1)])
def test_fft_path_equals_direct_dft(N, V, alpha, rng):
    """Brute force on tiny inputs: explicit O(M^2) DFT sums replace both FFTs."""
    for th in (synth.uniform_angles(V), _nonuniform(rng, V)):
        y = rng.standard_normal((V, N))
        for mode, g in ((ob.FILTER, None), (ob.FILTER, rng.uniform(0.2, 2, alpha * N // 2)),
                        (ob.BACKPROJECT, None)):
            a = ob.bst(y, th, alpha, mode, g)
            b = ob.bst(y, th, alpha, mode, g, direct=True)
            assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


@pytest.mark.parametrize("uniform", [True, False])
def test_gridding_reproduces_bilinear_polar_data(uniform, rng):
    """P5 is bilinear in (signed radius, angle): data that is bilinear in (k, theta_j)
    must be reproduced exactly at every Cartesian point away from the seam."""
    M, V = 64, 24
    th = synth.uniform_angles(V) if uniform else _nonuniform(rng, V, lo=0.02)
    t64 = th.astype(np.float64)
    a, b, c, d = 0.7, -0.03, 0.4, 0.011
    k = ob.signed_index(M).astype(np.float64)
    Z = a + b * k[None, :] + c * t64[:, None] + d * k[None, :] * t64[:, None]
    X = ob.grid(Z.astype(np.complex128), th)
    kk = ob.signed_index(M).astype(np.float64)
    C, R = np.meshgrid(kk, kk)
    rho = np.hypot(C, R)
    up = (R > 0) | ((R == 0) & (C >= 0))
    theta = np.arctan2(np.where(up, R, -R), np.where(up, C, -C))
    kappa = np.where(up, rho, -rho)
    ok = (rho < M / 2 - 1) & (theta >= t64[0]) & (theta < t64[-1])
    expect = a + b * kappa + c * theta + d * kappa * theta
    assert ok.sum() > 1000
    np.testing.assert_allclose(X[ok].real, expect[ok], rtol=0, atol=1e-11)
    assert np.all(X[rho >= M / 2] == 0)


def linear_spectrum_error(th, M=64, a=0.8, b=-0.45):
    """Max excess of |grid(Z) - F| over the linear-interpolation error bound, for
    the polar samples Z_j[k] = F(k xi_j) of the linear function F(w) = a w1 + b w2.
    Z is consistent with the seam identity Z(theta + pi, k) = Z(theta, -k), so
    every Cartesian point, seam brackets included, must come out within
    |kappa| (|a| + |b|) dtheta^2 / 8 of F."""
    t64 = np.asarray(th, dtype=np.float32).astype(np.float64)
    k = ob.signed_index(M).astype(np.float64)
    Z = k[None, :] * (a * np.cos(t64)[:, None] + b * np.sin(t64)[:, None])
    X = ob.grid(Z.astype(np.complex128), th)
    C, R = np.meshgrid(k, k)
    rho = np.hypot(C, R)
    ok = rho < M / 2 - 1
    ext = np.concatenate(([t64[-1] - np.pi], t64, [t64[0] + np.pi]))
    dmax = np.diff(ext).max()
    bound = rho * (abs(a) + abs(b)) * dmax * dmax / 8.0 + 1e-12
    return np.max(np.abs(X.real - (a * C + b * R))[ok] - bound[ok])


@pytest.mark.parametrize("uniform", [True, False])
def test_gridding_of_linear_spectrum_within_interpolation_bound(uniform, rng):
    th = synth.uniform_angles(40) if uniform else _nonuniform(rng, 40, lo=0.03)
    assert linear_spectrum_error(th) <= 0.0


@pytest.mark.parametrize("mode", [ob.FILTER, ob.BACKPROJECT])
@pytest.mark.parametrize("uniform", [True, False])
def test_output_is_real(mode, uniform, rng):
    """For a real sinogram the gridded spectrum is Hermitian, so the padded
    image has no imaginary part (pins the signed-radius and seam rules)."""
    N, V = 32, 28
    th = synth.uniform_angles(V) if uniform else _nonuniform(rng, V)
    y = rng.standard_normal((V, N))
    _, xp = ob.bst(y, th, 2, mode, return_pad=True)
    assert np.abs(xp.imag).max() <= 1e-13 * np.abs(xp.real).max()


@pytest.mark.parametrize("N", [64, 128])
def test_fbp_reconstructs_gaussian_blob(N):
    """Eq. 3 with the ramp (g = 1) inverts the closed-form projection of an
    off-centre Gaussian (pins scale, orientation and transform signs)."""
    th = synth.uniform_angles(N)
    y = synth.gaussian_blob_sinogram((0.3, -0.2), 0.08, 1.0, th, N)
    ref = synth.gaussian_blob_image((0.3, -0.2), 0.08, 1.0, N)
    x = ob.fbp(y, th)
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < 0.025
    assert np.linalg.norm(x - brute.ss_fbp(y, th)) / np.linalg.norm(ref) < 0.035


def test_fbp_reconstructs_ellipse_phantom():
    """Ellipse phantom of the paper's evaluation (Sec. 4): BST-FBP error against
    the phantom, measured once (0.077 at N=64, 0.059 at N=128) and frozen."""
    for N, tol in ((64, 0.09), (128, 0.07)):
        th = synth.uniform_angles(N)
        ells = synth.random_ellipses(np.random.default_rng(5), fov_safe=True)
        y = synth.ellipse_sinogram(ells, th, N)
        img = synth.ellipse_image(ells, N, 4)
        m = _radius(N) <= 0.9
        x = ob.fbp(y, th)
        assert np.linalg.norm((x - img)[m]) / np.linalg.norm(img[m]) < tol


def test_backprojection_agrees_with_brute_force():
    """Plain BST (W = 1/sigma) approximates Eq. 2 up to an additive constant
    (W[0] = 0); mean-removed agreement measured once (0.074) and frozen."""
    for N in (64, 128):
        th = synth.uniform_angles(N)
        ells = synth.random_ellipses(np.random.default_rng(5), fov_safe=True)
        y = synth.ellipse_sinogram(ells, th, N)
        b1 = ob.backproject(y, th)
        b2 = brute.backproject(y, th)
        m = _radius(N) <= 0.9
        d1 = b1[m] - b1[m].mean()
        d2 = b2[m] - b2[m].mean()
        assert np.linalg.norm(d1 - d2) / np.linalg.norm(d2) < 0.085


def test_fbp_of_a_centred_disk_has_the_right_level():
    """A uniform disk of radius 0.3 and density 1: projection 2 sqrt(r^2 - t^2).
    The reconstructed plateau must be 1 (pins the net constant
    dt * dw^2 = N / (2 M^2) and the DC handling); measured 1.004-1.005."""
    for N in (64, 128):
        th = synth.uniform_angles(N)
        disk = [synth.Ellipse(0.0, 0.0, 0.3, 0.3, 0.0, 1.0)]
        x = ob.fbp(synth.ellipse_sinogram(disk, th, N), th)
        m = _radius(N) <= 0.15
        assert abs(x[m].mean() - 1.0) < 0.01


def test_weights_and_padding_conventions():
    M, N = 16, 8
    W = ob.weight_table(M, N, ob.BACKPROJECT)
    assert W[0] == 0 and W[M // 2] == 0
    np.testing.assert_allclose(W[1:M // 2], M * (2.0 / N) / np.arange(1, M // 2))
    g = np.arange(M // 2, dtype=np.float64) + 1
    W = ob.weight_table(M, N, ob.FILTER, g)
    assert W[M // 2] == 0 and np.all(W[: M // 2] == g)
    p = ob.pad_center(np.arange(N, dtype=np.float64)[None, :] + 1, M)[0].real
    # centre sample (i = N/2, t = 0) lands on m = 0; i = 0 (t = -1) on m = M - N/2
    assert p[0] == N // 2 + 1 and p[M - N // 2] == 1 and p[N // 2 - 1] == N
    assert np.all(p[N // 2: M - N // 2] == 0)


def test_angle_validation():
    with pytest.raises(ValueError):
        ob.angles64(np.array([0.0, 0.5, 0.4], dtype=np.float32))
    with pytest.raises(ValueError):
        ob.angles64(np.array([0.0, 3.2], dtype=np.float32))
    with pytest.raises(ValueError):
        ob.angles64(np.array([-0.1, 1.0], dtype=np.float32))
