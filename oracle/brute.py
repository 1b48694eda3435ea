"""Brute-force backprojection B, its transpose R, and slant-stack FBP (FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Geometry: detector sample i sits at t_i = (i - N/2) dt, dt = 2/N; pixel
(r, c) sits at u = ((c - N/2) d, (r - N/2) d), d = dt.

B follows Eq. 2, b(u) = int_0^pi y(u . xi_theta, theta) d theta, as a Riemann
sum over the supplied angles with trapezoid weights on the half circle,
w_j = (theta_{j+1} - theta_{j-1}) / 2 with theta_V = theta_0 + pi and
theta_{-1} = theta_{V-1} - pi (pi/V for uniform angles), and y(t) taken by
linear interpolation on the fractional index t/dt + N/2, zero outside
[0, N-1].  Summing along every pixel's line for every angle is the
slant-stack (SS) backprojection of Sec. 2, O(N^3) per slice.

R is the exact transpose of that discrete B, written as a scatter (Eq. 1
discretised), so that <B p, f> = <p, R f> holds to rounding.

SS filtered backprojection (x = B[F y], Sec. 1): each angle is filtered
along t with the ramp |sigma| times the filter taps g, on the same padded
FFT grid the BST path uses, then backprojected.
"""
from __future__ import annotations

import numpy as np


def _angles64(angles) -> np.ndarray:
    return np.asarray(angles, dtype=np.float32).astype(np.float64)


def trapezoid_weights(angles) -> np.ndarray:
    """Angular quadrature weights of Eq. 2 on [0, pi) with the pi-periodic wrap."""
    th = _angles64(angles)
    ext = np.concatenate(([th[-1] - np.pi], th, [th[0] + np.pi]))
    return (ext[2:] - ext[:-2]) / 2.0


def _frac_index(N: int, theta: float, rows: np.ndarray, cols: np.ndarray) -> np.ndarray:
    # t / dt + N/2 with t = u1 cos(theta) + u2 sin(theta)
    return (cols - N // 2) * np.cos(theta) + (rows - N // 2) * np.sin(theta) + N // 2


def _interp(yj: np.ndarray, fi: np.ndarray) -> np.ndarray:
    N = yj.shape[0]
    i0 = np.floor(fi).astype(np.int64)
    f = fi - i0
    v0 = np.where((i0 >= 0) & (i0 <= N - 1), yj[np.clip(i0, 0, N - 1)], 0.0)
    v1 = np.where((i0 + 1 >= 0) & (i0 + 1 <= N - 1), yj[np.clip(i0 + 1, 0, N - 1)], 0.0)
    return (1.0 - f) * v0 + f * v1


def backproject(y: np.ndarray, angles) -> np.ndarray:
    """B y for one sinogram y[V][N] -> image [N][N] (Eq. 2, slant-stack sum)."""
    y = np.asarray(y, dtype=np.float64)
    V, N = y.shape
    th = _angles64(angles)
    w = trapezoid_weights(th)
    r = np.arange(N, dtype=np.float64)[:, None]
    c = np.arange(N, dtype=np.float64)[None, :]
    out = np.zeros((N, N), dtype=np.float64)
    for j in range(V):
        out += w[j] * _interp(y[j], _frac_index(N, th[j], r, c))
    return out


def backproject_pixels(y: np.ndarray, angles, rows, cols) -> np.ndarray:
    """B y evaluated only at the listed pixels (rows[i], cols[i])."""
    y = np.asarray(y, dtype=np.float64)
    V, N = y.shape
    th = _angles64(angles)
    w = trapezoid_weights(th)
    rows = np.asarray(rows, dtype=np.float64)
    cols = np.asarray(cols, dtype=np.float64)
    out = np.zeros(rows.shape, dtype=np.float64)
    for j in range(V):
        out += w[j] * _interp(y[j], _frac_index(N, th[j], rows, cols))
    return out


def project(x: np.ndarray, angles, N: int | None = None) -> np.ndarray:
    """R x: the exact transpose of ``backproject`` (a scatter over pixels)."""
    x = np.asarray(x, dtype=np.float64)
    N = N or x.shape[0]
    th = _angles64(angles)
    w = trapezoid_weights(th)
    V = th.shape[0]
    r = np.repeat(np.arange(N, dtype=np.float64), N)
    c = np.tile(np.arange(N, dtype=np.float64), N)
    xv = x.reshape(-1)
    y = np.zeros((V, N), dtype=np.float64)
    for j in range(V):
        fi = _frac_index(N, th[j], r, c)
        i0 = np.floor(fi).astype(np.int64)
        f = fi - i0
        for idx, wt in ((i0, (1.0 - f)), (i0 + 1, f)):
            ok = (idx >= 0) & (idx <= N - 1)
            y[j] += w[j] * np.bincount(idx[ok], weights=(wt * xv)[ok], minlength=N)
    return y


def ramp_taps(M: int, N: int, g=None) -> np.ndarray:
    """h_k for k = 0..M/2: |sigma_k| g[k] with sigma_k = k dsigma, dsigma = 1/(M dt);
    h_0 = (dsigma/4) g[0] (the cell average of |sigma| over the DC bin) and
    h_{M/2} = 0.  g = None is the plain ramp (g = 1)."""
    dt = 2.0 / N
    dsig = 1.0 / (M * dt)
    gg = np.ones(M // 2, dtype=np.float64) if g is None else np.asarray(g, dtype=np.float64)[: M // 2]
    h = np.zeros(M // 2 + 1, dtype=np.float64)
    k = np.arange(M // 2, dtype=np.float64)
    h[: M // 2] = k * dsig * gg
    h[0] = 0.25 * dsig * gg[0]
    return h


def ramp_filter(y: np.ndarray, pad_factor: int = 2, g=None) -> np.ndarray:
    """F y along t (Sec. 1): q_j[i] = dsigma sum_k h_k Y_j[k] e^{+2 pi i k m / M}, with
    Y_j = dt DFT_M of the centre-aligned padded ray and m = (i - N/2) mod M."""
    y = np.asarray(y, dtype=np.float64)
    V, N = y.shape
    M = pad_factor * N
    dt = 2.0 / N
    dsig = 1.0 / (M * dt)
    m = (np.arange(N) - N // 2) % M
    p = np.zeros((V, M), dtype=np.float64)
    p[:, m] = y
    Y = dt * np.fft.fft(p, axis=1)
    k = np.arange(M)
    ak = np.minimum(k, M - k)
    h = ramp_taps(M, N, g)
    q = dsig * M * np.fft.ifft(Y * h[ak][None, :], axis=1)
    return np.real(q[:, m])


def ss_fbp(y: np.ndarray, angles, pad_factor: int = 2, g=None) -> np.ndarray:
    """Slant-stack filtered backprojection x = B[F y]."""
    return backproject(ramp_filter(y, pad_factor, g), angles)
