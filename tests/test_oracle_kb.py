"""Pins of the Kaiser-Bessel gridding oracle (oracle/kb.py), no GPU.

The direct sum is pinned to the independent slant-stack FBP of oracle/brute.py
(which never touches the 2D Fourier plane) at the points where the two must
coincide; the gridding is pinned to the direct sum within the error of
convolution gridding, which must fall as the kernel widens; the closed-form
kernel transform is pinned to numerical quadrature.  Planted mistakes in each
step must fail one of these pins."""
import numpy as np
import pytest

import synth
from oracle import brute
from oracle import bst as ob
from oracle import kb


def _rand_sino(rng, V, N):
    return rng.standard_normal((V, N))


def _phantom_sino(V, N, seed=3):
    th = synth.uniform_angles(V)
    ell = synth.random_ellipses(np.random.default_rng(seed), fov_safe=True)
    return th, synth.ellipse_sinogram(ell, th, N)


@pytest.mark.filterwarnings("ignore::UserWarning")
def test_kb_transform_matches_quadrature():
    quad = pytest.importorskip("scipy.integrate").quad
    for width, alpha in ((4, 2), (6, 2), (8, 2), (6, 1)):
        beta = kb.kb_beta(width, alpha)
        for nu in (0.0, 0.07, 0.25, 0.5, 0.8, 1.4):
            val = quad(lambda x: float(kb.kb_kernel(x, width, beta)) * np.cos(2 * np.pi * nu * x),
                       -width / 2, width / 2, limit=400, epsabs=1e-14)[0]
            assert abs(val - float(kb.kb_transform(nu, width, beta))) <= 1e-9 * max(abs(val), 1e-3)


def test_kernel_is_normalised_and_even():
    beta = kb.kb_beta(6, 2)
    assert kb.kb_kernel(0.0, 6, beta) == pytest.approx(1.0, abs=1e-15)
    x = np.linspace(0, 3, 37)
    assert np.array_equal(kb.kb_kernel(x, 6, beta), kb.kb_kernel(-x, 6, beta))
    assert kb.kb_kernel(3.0001, 6, beta) == 0.0
    assert kb.kb_kernel(3.0, 6, beta) == 0.0    # no pedestal: ties at the support edge carry no weight


@pytest.mark.parametrize("mode_g", ["ramp", "taps"])
def test_direct_sum_centre_pixel_equals_slant_stack(rng, mode_g):
    # t = u . xi = 0 at the centre pixel for every angle: a detector sample,
    # where the slant stack's linear interpolation is exact
    V, N = 24, 32
    th = np.sort(rng.uniform(0.02, 3.1, V)).astype(np.float32)
    y = _rand_sino(rng, V, N)
    g = None if mode_g == "ramp" else rng.uniform(0.5, 1.5, N)
    ctr = kb.direct_sum(y, th, 2, ob.FILTER, g, pixels=([N // 2], [N // 2]))[0]
    ss = brute.ss_fbp(y, th, 2, g)[N // 2, N // 2]
    assert abs(ctr - ss) <= 1e-12 * np.abs(y).max()


def test_direct_sum_equals_slant_stack_on_the_axes(rng):
    # angles 0 and pi/2: every pixel projects onto a detector sample (up to the
    # float32 rounding of pi/2), so trigonometric and linear interpolation agree
    N = 32
    th = np.array([0.0, np.pi / 2], dtype=np.float32)
    y = _rand_sino(rng, 2, N)
    d = kb.direct_sum(y, th)
    s = brute.ss_fbp(y, th)
    assert np.abs(d - s).max() <= 1e-5 * np.abs(s).max()


@pytest.mark.parametrize("width,bound", [(4, 1e-3), (6, 1e-5), (8, 2e-7)])
def test_gridding_converges_to_the_direct_sum(width, bound):
    N = V = 48
    th, y = _phantom_sino(V, N)
    xe = kb.direct_sum(y, th)
    xk = kb.kb_fbp(y, th, width=width)
    assert np.linalg.norm(xk - xe) / np.linalg.norm(xe) < bound


def test_gridding_nonuniform_angles_taps_and_plain_b(rng):
    V, N = 40, 32
    th = np.sort(rng.uniform(0.01, 3.13, V)).astype(np.float32)
    y = _rand_sino(rng, V, N)
    g = rng.uniform(0.2, 1.2, N)
    for mode, gg in ((ob.FILTER, g), (ob.BACKPROJECT, None)):
        xe = kb.direct_sum(y, th, 2, mode, gg)
        xk = kb.kb_fbp(y, th, 2, mode, gg)
        assert np.linalg.norm(xk - xe) / np.linalg.norm(xe) < 1e-5


def test_pad_factor_one_interior():
    # no guard band at M = N: the edge aliases, the inscribed disk stays accurate
    N = V = 48
    th, y = _phantom_sino(V, N)
    xe = kb.direct_sum(y, th, 1)
    xk = kb.kb_fbp(y, th, 1)
    base = np.arange(N) - N // 2
    m = np.hypot(base[None, :], base[:, None]) < 0.8 * N / 2
    assert np.linalg.norm((xk - xe)[m]) / np.linalg.norm(xe[m]) < 3e-3


def test_kb_is_closer_to_the_discrete_integral_than_bilinear():
    # both approximate the same polar quadrature; bilinear interpolation in
    # (kappa, theta) loses most of the accuracy that the KB kernel keeps
    N = V = 48
    th, y = _phantom_sino(V, N)
    xe = kb.direct_sum(y, th)
    e_kb = np.linalg.norm(kb.kb_fbp(y, th) - xe) / np.linalg.norm(xe)
    e_bl = np.linalg.norm(ob.fbp(y, th) - xe) / np.linalg.norm(xe)
    assert e_kb < 1e-5 and e_bl > 100 * e_kb


def test_blob_reconstruction_matches_closed_form():
    N = 64
    th = synth.uniform_angles(N)
    y = synth.gaussian_blob_sinogram((0.3, -0.2), 0.08, 1.0, th, N)
    ref = synth.gaussian_blob_image((0.3, -0.2), 0.08, 1.0, N)
    assert np.linalg.norm(kb.kb_fbp(y, th) - ref) / np.linalg.norm(ref) < 0.025


# ---- planted mistakes ----------------------------------------------------------

def _pins_hold() -> bool:
    rng = np.random.default_rng(11)
    N, V = 24, 20
    th = np.sort(rng.uniform(0.02, 3.1, V)).astype(np.float32)
    y = _rand_sino(rng, V, N)
    ok = abs(kb.direct_sum(y, th, pixels=([N // 2], [N // 2]))[0] - brute.ss_fbp(y, th)[N // 2, N // 2]) \
        <= 1e-12 * np.abs(y).max()
    th2 = np.array([0.0, np.pi / 2], dtype=np.float32)
    y2 = _rand_sino(rng, 2, N)
    s2 = brute.ss_fbp(y2, th2)
    ok &= np.abs(kb.direct_sum(y2, th2) - s2).max() <= 1e-5 * np.abs(s2).max()
    xe = kb.direct_sum(y, th)
    ok &= np.linalg.norm(kb.kb_fbp(y, th) - xe) / np.linalg.norm(xe) < 1e-5
    return bool(ok)


def test_pins_hold_on_the_real_oracle():
    assert _pins_hold()


class _FFTWithForwardInverse:
    """np.fft with ifft2 replaced by the forward transform (wrong exponent sign)."""

    def __getattr__(self, name):
        return getattr(np.fft, name)

    @staticmethod
    def ifft2(G):
        return np.fft.fft2(G) / G.size


def _mutant(name):
    if name == "no deapodization":
        return "kb_transform", lambda nu, w, b: np.ones_like(np.asarray(nu, dtype=np.float64))
    if name == "positions transposed":
        real = kb.sample_positions
        return "sample_positions", lambda M, angles: real(M, angles)[::-1]
    if name == "DC cell weight dropped":
        real = kb.sample_weights

        def no_dc(M, N, angles, mode=ob.FILTER, g=None):
            w = real(M, N, angles, mode, g).copy()
            w[:, 0] = 0.0
            return w
        return "sample_weights", no_dc
    if name == "kernel shape for the wrong oversampling":
        return "kb_beta", lambda w, a: float(np.pi * np.sqrt(w * w * 0.25 - 0.8))
    if name == "samples spread one bin off":
        real = kb.spread
        return "spread", lambda a, cs, rs, M, w, b: real(a, cs - 1.0, rs, M, w, b)
    raise KeyError(name)


MUTANTS = ["no deapodization", "positions transposed", "DC cell weight dropped",
           "kernel shape for the wrong oversampling", "samples spread one bin off", "forward exponent in P6"]


@pytest.mark.parametrize("name", MUTANTS)
def test_planted_mistake_fails_a_pin(monkeypatch, name):
    if name == "forward exponent in P6":
        monkeypatch.setattr(kb, "np", type("np_with_wrong_ifft", (), {
            "__getattr__": lambda self, k: getattr(np, k), "fft": _FFTWithForwardInverse()})())
    else:
        attr, fn = _mutant(name)
        monkeypatch.setattr(kb, attr, fn)
    assert not _pins_hold()
