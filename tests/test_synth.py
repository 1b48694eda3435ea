"""Pins of the input generators: closed-form ellipse projections (Eq. 1 on an
ellipse, Sec. 4 footnote) against brute-force numerical line integrals."""
import numpy as np

import synth


def _inside(e, u1, u2):
    x, y = u1 - e.cx, u2 - e.cy
    cp, sp = np.cos(e.psi), np.sin(e.psi)
    p = (x * cp + y * sp) / e.a
    q = (-x * sp + y * cp) / e.b
    return p * p + q * q <= 1.0


def test_ellipse_sinogram_matches_line_integrals():
    rng = np.random.default_rng(3)
    ells = synth.random_ellipses(rng, fov_safe=True)
    N = 64
    th = synth.uniform_angles(16)
    y = synth.ellipse_sinogram(ells, th, N)
    t = synth.detector_coords(N)
    s = np.linspace(-1.5, 1.5, 300001)
    ds = s[1] - s[0]
    for j in (0, 3, 7, 12):
        c, sn = np.cos(np.float64(th[j])), np.sin(np.float64(th[j]))
        for i in (10, 25, 32, 40, 55):
            u1 = t[i] * c - s * sn
            u2 = t[i] * sn + s * c
            val = sum(e.rho * _inside(e, u1, u2).sum() * ds for e in ells)
            assert abs(val - y[j, i]) < 2e-3


def test_blob_sinogram_matches_line_integrals():
    N = 32
    th = synth.uniform_angles(8)
    y = synth.gaussian_blob_sinogram((0.2, -0.1), 0.1, 1.5, th, N)
    t = synth.detector_coords(N)
    s = np.linspace(-2, 2, 40001)
    ds = s[1] - s[0]
    for j in range(8):
        c, sn = np.cos(np.float64(th[j])), np.sin(np.float64(th[j]))
        for i in (8, 16, 20):
            u1 = t[i] * c - s * sn
            u2 = t[i] * sn + s * c
            val = np.sum(1.5 * np.exp(-((u1 - 0.2) ** 2 + (u2 + 0.1) ** 2) / 0.02)) * ds
            assert abs(val - y[j, i]) < 1e-9


def test_workloads_are_seeded_and_shaped():
    th, s1, _ = synth.workload_slices("volume-512", [3, 7], rays=64, angles=48)
    th2, s2, _ = synth.workload_slices("volume-512", [7], rays=64, angles=48)
    assert s1.shape == (2, 48, 64) and s1.dtype == np.float32
    np.testing.assert_array_equal(s1[1], s2[0])
    assert np.all(np.diff(th.astype(np.float64)) > 0) and th[-1] < np.pi
    sizes = synth.ragged_sizes()
    assert len(sizes) == 64 and set(sizes) <= {256, 512, 768, 1024, 1536, 2048}


def test_poisson_noise_mean():
    rng = np.random.default_rng(0)
    y = np.full((200, 200), 0.5)
    yn = synth.poisson_log_noise(y, rng)
    assert abs(yn.mean() - 0.5) < 2e-3
    assert 0.005 < yn.std() < 0.03
