"""Pins of the brute-force oracle (Eq. 2 backprojection, its transpose, SS-FBP)."""
import numpy as np
import pytest

import synth
from oracle import brute


def _radius(N):
    base = (np.arange(N) - N // 2) * (2.0 / N)
    return np.hypot(base[None, :], base[:, None])


@pytest.mark.parametrize("N,V", [(16, 12), (33, 20), (64, 64)])
def test_constant_sinogram_backprojects_to_c_pi(N, V):
    # int_0^pi c d theta = c pi wherever every ray sample is inside the detector
    c = 1.7
    th = synth.uniform_angles(V)
    b = brute.backproject(np.full((V, N), c), th)
    m = _radius(N) <= 1.0 - 2.0 / N
    np.testing.assert_allclose(b[m], c * np.pi, rtol=0, atol=1e-12)


def test_constant_invariant_nonuniform_angles(rng):
    th = np.sort(rng.uniform(0.0, np.pi - 1e-3, 17)).astype(np.float32)
    N = 24
    b = brute.backproject(np.full((17, N), 2.0), th)
    m = _radius(N) <= 1.0 - 2.0 / N
    np.testing.assert_allclose(b[m], 2.0 * np.pi, rtol=0, atol=1e-12)


@pytest.mark.parametrize("N,V", [(16, 12), (20, 31)])
def test_adjoint_identity_B_R(N, V, rng):
    th = synth.uniform_angles(V)
    p = rng.standard_normal((V, N))
    f = rng.standard_normal((N, N))
    lhs = np.sum(brute.backproject(p, th) * f)
    rhs = np.sum(p * brute.project(f, th))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_point_rays_land_on_the_right_pixels():
    # a single detector sample at t = t_i for theta = 0 backprojects onto the
    # column u1 = t_i (theta = 0 => t = u1); at theta = pi/2 onto the row u2 = t_i
    N = 16
    th = np.array([0.0, np.pi / 2], dtype=np.float32)
    y = np.zeros((2, N))
    y[0, 11] = 1.0
    b = brute.backproject(y, th)
    w = brute.trapezoid_weights(th)[0]
    assert np.allclose(b[:, 11], w) and np.allclose(np.delete(b, 11, axis=1), 0.0)
    y = np.zeros((2, N))
    y[1, 4] = 1.0
    b = brute.backproject(y, th)
    s = np.float64(np.sin(np.float32(np.pi / 2)))
    c = np.float64(np.cos(np.float32(np.pi / 2)))
    assert abs(s - 1) < 1e-7 and abs(c) < 1e-7
    assert np.allclose(b[4, N // 2], brute.trapezoid_weights(th)[1], atol=1e-5)


@pytest.mark.parametrize("N", [64, 128])
def test_ss_fbp_reconstructs_gaussian_blob(N):
    th = synth.uniform_angles(N)
    y = synth.gaussian_blob_sinogram((0.3, -0.2), 0.08, 1.0, th, N)
    ref = synth.gaussian_blob_image((0.3, -0.2), 0.08, 1.0, N)
    x = brute.ss_fbp(y, th)
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < 0.03


def test_backproject_pixels_matches_full():
    N, V = 24, 18
    th = synth.uniform_angles(V)
    y = np.random.default_rng(4).standard_normal((V, N))
    full = brute.backproject(y, th)
    rows = np.array([0, 5, 12, 23])
    cols = np.array([3, 12, 0, 23])
    np.testing.assert_allclose(brute.backproject_pixels(y, th, rows, cols), full[rows, cols], atol=1e-12)
