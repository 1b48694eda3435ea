"""Kaiser-Bessel convolution gridding for stage P5 (FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 2 names the polar-to-Cartesian interpolation of stage P5 but not its
kernel; the plain path uses bilinear interpolation in (signed radius, angle).
This module is the Kaiser-Bessel (KB) alternative, classical convolution
gridding.  It starts from what Eq. 3 says about the image: with
x^(sigma xi_theta) known on the polar grid, the inverse 2D Fourier integral
in polar coordinates, discretised with the angular weights dtheta_j of the
half circle and the radial step dsigma, is the finite sum

    x(u) = sum_{j,k} a_jk exp(2 pi i omega_jk . u),
    a_jk = dtheta_j dsigma |sigma_k| W[|k|] Y_j[k],   omega_jk = sigma_k xi_j,

where Y_j is the P3 spectrum and W the P4 weight (the filter g for FBP,
1/sigma_k for plain B).  The DC cell takes dsigma / 4 for |sigma_0| (the cell
average of |sigma|, as for the slant-stack ramp) and the Nyquist bin is zero.
In bin units (dsigma = dw = 1/(M dt)) the sample sits at
(c_s, r_s) = k (cos theta_j, sin theta_j) and pixel (r, c) at
(c_p, r_p) = (c - N/2, r - N/2), so omega . u = (c_s c_p + r_s r_p) / M.
``direct_sum`` evaluates this sum as written (the quantity gridding
approximates).  ``kb_fbp`` approximates it in O(M^2 log M):

    1. spread: G[r', c'] = sum_s a_s phi(c' - c_s) phi(r' - r_s) on the
       M-periodic grid, phi the KB kernel of width W (in bins) normalised to
       phi(0) = 1, over the W points c' - c_s in (-W/2, W/2];
    2. x_pad[r_p, c_p] = sum G[r', c'] exp(+2 pi i (r' r_p + c' c_p) / M);
    3. volume[r][c] = Re x_pad / (C(c_p / M) C(r_p / M)), C the continuous
       Fourier transform of phi (deapodization).

Readings (the paper gives no kernel): W = 6 by default; shape
beta = pi sqrt((W / alpha)^2 (alpha - 1/2)^2 - 0.8) with alpha = M / N the
grid oversampling (the choice of Beatty, Nishimura and Pauly, 2005);
phi(x) = (I0(beta sqrt(1 - (2x/W)^2)) - 1) / (I0(beta) - 1) for |x| <= W/2,
the KB kernel with its pedestal removed.  The pedestal-free form is zero at
the edge of the support, so a sample whose footprint edge falls exactly on a
grid point (every sample at theta = 0 or pi/2 does) adds nothing there; the
plain KB kernel, 1/I0(beta) at the edge, would make the gridded spectrum of a
real slice depart from Hermitian symmetry by that much at each such tie
(the half-open support keeps one edge point of a sample and drops the
mirrored point of its mirror sample).
"""
from __future__ import annotations

import numpy as np

from . import bst as ob
from .brute import trapezoid_weights


def kb_beta(width: int, pad_factor: float) -> float:
    a = float(pad_factor)
    return float(np.pi * np.sqrt((width / a) ** 2 * (a - 0.5) ** 2 - 0.8))


def kb_kernel(x, width: int, beta: float) -> np.ndarray:
    """phi(x) = (I0(beta sqrt(1 - (2x/W)^2)) - 1) / (I0(beta) - 1) on |x| <= W/2,
    else 0: the KB kernel without its pedestal, so phi(+-W/2) = 0."""
    x = np.asarray(x, dtype=np.float64)
    u = 2.0 * x / width
    inside = np.abs(u) <= 1.0
    v = (np.i0(beta * np.sqrt(np.maximum(1.0 - u * u, 0.0))) - 1.0) / (np.i0(beta) - 1.0)
    return np.where(inside, v, 0.0)


def kb_transform(nu, width: int, beta: float) -> np.ndarray:
    """C(nu) = int phi(x) exp(-2 pi i nu x) dx
             = W (sinh(z) / z - sinc(W nu)) / (I0(beta) - 1),
    z = sqrt(beta^2 - (pi W nu)^2) (sin(|z|)/|z| when z is imaginary),
    sinc(x) = sin(pi x) / (pi x): the transform of I0(beta sqrt(1 - (2x/W)^2))
    minus that of the pedestal 1 on [-W/2, W/2]."""
    nu = np.asarray(nu, dtype=np.float64)
    z2 = beta * beta - (np.pi * width * nu) ** 2
    z = np.sqrt(np.abs(z2))
    small = z < 1e-8
    zs = np.where(small, 1.0, z)
    ratio = np.where(small, 1.0, np.where(z2 >= 0, np.sinh(zs) / zs, np.sin(zs) / zs))
    return width * (ratio - np.sinc(width * nu)) / (np.i0(beta) - 1.0)


def sample_weights(M: int, N: int, angles, mode: str = ob.FILTER, g=None) -> np.ndarray:
    """a_jk / Y_j[k] as an array [V][M] (natural FFT order of k)."""
    dt = 2.0 / N
    dsig = 1.0 / (M * dt)
    W = ob.weight_table(M, N, mode, g)
    k = np.abs(ob.signed_index(M)).astype(np.float64)
    kk = np.where(k == 0, 0.25, k)          # |sigma_k| / dsigma, DC cell average 1/4
    radial = dsig * dsig * kk * W[np.abs(ob.signed_index(M))]
    return trapezoid_weights(angles)[:, None] * radial[None, :]


def sample_positions(M: int, angles):
    """(c_s, r_s) = k (cos theta_j, sin theta_j) in bins, arrays [V][M]."""
    th = ob.angles64(angles)
    k = ob.signed_index(M).astype(np.float64)
    return k[None, :] * np.cos(th)[:, None], k[None, :] * np.sin(th)[:, None]


def weighted_samples(y, angles, pad_factor: int = 2, mode: str = ob.FILTER, g=None):
    """P2-P4 and the quadrature weight: a_s, c_s, r_s as flat arrays."""
    y = np.asarray(y, dtype=np.float64)
    V, N = y.shape
    M = pad_factor * N
    Y = ob.ray_spectrum(y, M)
    a = Y * sample_weights(M, N, angles, mode, g)
    cs, rs = sample_positions(M, angles)
    return a.reshape(-1), cs.reshape(-1), rs.reshape(-1)


def direct_sum(y, angles, pad_factor: int = 2, mode: str = ob.FILTER, g=None, pixels=None) -> np.ndarray:
    """x(u_p) = Re sum_s a_s exp(2 pi i (c_s c_p + r_s r_p) / M), every pixel
    (an [N][N] image) or the listed (rows, cols)."""
    y = np.asarray(y, dtype=np.float64)
    N = y.shape[1]
    M = pad_factor * N
    a, cs, rs = weighted_samples(y, angles, pad_factor, mode, g)
    keep = a != 0
    a, cs, rs = a[keep], cs[keep], rs[keep]
    if pixels is None:
        rr, cc = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
        rows, cols = rr.reshape(-1), cc.reshape(-1)
    else:
        rows, cols = (np.asarray(v).reshape(-1) for v in pixels)
    cp = (cols - N // 2).astype(np.float64)
    rp = (rows - N // 2).astype(np.float64)
    out = np.empty(rows.size, dtype=np.float64)
    step = max(1, 2_000_000 // max(a.size, 1))
    for i0 in range(0, rows.size, step):
        ph = np.outer(cp[i0:i0 + step], cs) + np.outer(rp[i0:i0 + step], rs)
        out[i0:i0 + step] = np.real(np.exp(2j * np.pi * ph / M) @ a)
    return out.reshape(N, N) if pixels is None else out


def spread(a, cs, rs, M: int, width: int, beta: float) -> np.ndarray:
    """Step 1: G[r' mod M, c' mod M] += a phi(c' - c_s) phi(r' - r_s) for the W
    grid points c' - c_s in (-W/2, W/2] of each axis."""
    G = np.zeros(M * M, dtype=np.complex128)
    c0 = np.floor(cs - width / 2.0).astype(np.int64) + 1
    r0 = np.floor(rs - width / 2.0).astype(np.int64) + 1
    for dc in range(width):
        wc = kb_kernel(c0 + dc - cs, width, beta)
        for dr in range(width):
            v = a * wc * kb_kernel(r0 + dr - rs, width, beta)
            idx = ((r0 + dr) % M) * M + (c0 + dc) % M
            G += np.bincount(idx, weights=v.real, minlength=M * M) + 1j * np.bincount(idx, weights=v.imag,
                                                                                       minlength=M * M)
    return G.reshape(M, M)


def kb_from_spectrum(Y, angles, N: int, mode: str = ob.FILTER, g=None, width: int = 6,
                     beta: float | None = None) -> np.ndarray:
    """Steps P4 (weight and cell area), P5 (KB spread), P6 and deapodization,
    from the P3 spectrum Y[V][M]."""
    M = Y.shape[-1]
    beta = kb_beta(width, M / N) if beta is None else beta
    a = (Y * sample_weights(M, N, angles, mode, g)).reshape(-1)
    cs, rs = (v.reshape(-1) for v in sample_positions(M, angles))
    keep = a != 0
    G = spread(a[keep], cs[keep], rs[keep], M, width, beta)      # P5
    xp = (M * M) * np.fft.ifft2(G)                                # P6
    p = np.arange(N) - N // 2
    idx = p % M                                                   # P7 (fftshift in the indices)
    C = kb_transform(p / M, width, beta)
    return np.real(xp[np.ix_(idx, idx)]) / (C[:, None] * C[None, :])


def kb_fbp(y, angles, pad_factor: int = 2, mode: str = ob.FILTER, g=None, width: int = 6,
           beta: float | None = None) -> np.ndarray:
    """BST FBP (or plain B) of one sinogram y[V][N] with KB gridding in P5."""
    y = np.asarray(y, dtype=np.float64)
    N = y.shape[1]
    Y = ob.ray_spectrum(y, pad_factor * N)                        # P2, P3
    return kb_from_spectrum(Y, angles, N, mode, g, width, beta)
