"""Pins of the adjoint oracle (the Fourier-slice projector dual to Eq. 3) and of
the filter-tap gradient: adjoint identities and central finite differences."""
import numpy as np
import pytest

import synth
from oracle import adjoint as oa
from oracle import bst as ob


@pytest.mark.parametrize("N,V,alpha", [(16, 12, 2), (32, 40, 2), (16, 20, 1)])
@pytest.mark.parametrize("mode", ["ramp", "taps", ob.BACKPROJECT])
def test_adjoint_identity(N, V, alpha, mode, rng):
    for th in (synth.uniform_angles(V), np.sort(rng.uniform(0.05, 3.1, V)).astype(np.float32)):
        p = rng.standard_normal((V, N))
        f = rng.standard_normal((N, N))
        if mode == ob.BACKPROJECT:
            m, g = ob.BACKPROJECT, None
        else:
            m, g = ob.FILTER, (None if mode == "ramp" else rng.uniform(0.3, 2.0, alpha * N // 2))
        lhs = np.sum(ob.bst(p, th, alpha, m, g) * f)
        rhs = np.sum(p * oa.bst_adjoint(f, th, alpha, m, g))
        assert abs(lhs - rhs) <= 1e-12 * np.sqrt(np.sum(p * p) * np.sum(f * f))


def test_filter_gradient_matches_finite_differences(rng):
    N, V = 16, 12
    th = synth.uniform_angles(V)
    p = rng.standard_normal((V, N))
    f = rng.standard_normal((N, N))
    g = rng.uniform(0.5, 1.5, N)

    def loss(gg):
        return np.sum((ob.fbp(p, th, g=gg) - f) ** 2)

    R = 2.0 * (ob.fbp(p, th, g=g) - f)
    G = oa.filter_grad(p, R, th)
    h = 1e-6
    fd = np.array([(loss(g + h * e) - loss(g - h * e)) / (2 * h) for e in np.eye(N)])
    assert np.abs(G - fd).max() <= 1e-7 * np.abs(fd).max()


def test_sinogram_gradient_matches_finite_differences(rng):
    N, V = 16, 12
    th = np.sort(rng.uniform(0.1, 3.0, V)).astype(np.float32)
    p = rng.standard_normal((V, N))
    f = rng.standard_normal((N, N))
    g = rng.uniform(0.5, 1.5, N)
    R = 2.0 * (ob.fbp(p, th, g=g) - f)
    Gp = oa.bst_adjoint(R, th, g=g)
    h = 1e-6
    for j, i in ((0, 0), (3, 5), (11, 15), (6, 8), (9, 1)):
        e = np.zeros_like(p)
        e[j, i] = h
        fd = (np.sum((ob.fbp(p + e, th, g=g) - f) ** 2) - np.sum((ob.fbp(p - e, th, g=g) - f) ** 2)) / (2 * h)
        assert abs(Gp[j, i] - fd) <= 1e-6 * max(1.0, abs(fd))


def test_grid_transpose_is_the_transpose_of_grid(rng):
    M, V = 32, 14
    th = synth.uniform_angles(V)
    Z = rng.standard_normal((V, M)) + 1j * rng.standard_normal((V, M))
    X = rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))
    lhs = np.sum(ob.grid(Z, th) * X)
    rhs = np.sum(Z * oa.grid_transpose(X, th))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
