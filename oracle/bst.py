"""The BST backprojection / filtered backprojection, step by step (FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Theorem 2.1 (Eq. 3): the 2D Fourier transform of the backprojection b = B y
on the polar point sigma (cos theta, sin theta) equals y^(sigma, theta) / sigma,
the 1D Fourier transform of the sinogram along t divided by sigma.  With the
ordinary-frequency convention f^(s) = int f(t) e^{-2 pi i s t} dt the constant
in Eq. 3 is exactly 1.  Sec. 2 computes b through the stages

    P0 polar relabelling   (y(-t, theta) = y(t, theta + pi): signed radii)
    P1 window              (omitted: the plain method uses no window)
    P2 zero padding        p_j[(i - N/2) mod M] = y_j[i], M = alpha N
    P3 1D FFT along t      Y_j[k] = dt sum_m p_j[m] e^{-2 pi i k m / M}
    P4 weight              Y_j[k] *= W[|k|]; W = 1/sigma_k for b, W = g for FBP
    P5 polar -> Cartesian  bilinear interpolation in (signed radius, angle)
    P6 2D inverse FFT      x = dw^2 sum X^[r', c'] e^{+2 pi i (r' r_p + c' c_p) / M}
    P7 fftshift            folded into the crop indices
    P8 resample to [-1,1]^2 identity: the grids already live on [-1, 1)^2

For FBP (x = B[F y], Sec. 1) the ramp |sigma| of F cancels the 1/sigma of
Eq. 3, so the weight is the filter in "BST form" g = h^/|sigma| (ramp: g = 1).

Readings taken where the paper is silent (each is a choice of this
repository): pad factor alpha = 2; bilinear interpolation; the Nyquist bin
W[M/2] = 0; the DC bin set to the mean over angles (the Cartesian origin is
single-valued); W[0] = 0 for plain B (b has a divergent mean, so b is defined
up to an additive constant); the seam theta_V = theta_0 + pi with
Y(theta_V, k) = Y(theta_0, -k); points with radius >= M/2 are zero.
"""
from __future__ import annotations

import numpy as np

FILTER = "filter"
BACKPROJECT = "backproject"


def angles64(angles) -> np.ndarray:
    """Angles as given to the C-ABI (float32), validated and widened exactly."""
    th = np.asarray(angles, dtype=np.float32).astype(np.float64)
    if th.ndim != 1 or th.size < 2:
        raise ValueError("need at least two angles")
    if not np.all(np.isfinite(th)) or th[0] < 0.0 or th[-1] >= np.pi or np.any(np.diff(th) <= 0):
        raise ValueError("angles must be finite, strictly increasing and in [0, pi)")
    return th


def signed_index(M: int) -> np.ndarray:
    """Signed frequency of each natural-order FFT index: k for k < M/2, k - M after."""
    k = np.arange(M)
    return np.where(k < M // 2, k, k - M)


# --- P2 + P3 ---------------------------------------------------------------

def pad_center(y: np.ndarray, M: int) -> np.ndarray:
    """P2: centre-aligned zero padding, p_j[(i - N/2) mod M] = y_j[i]."""
    y = np.asarray(y, dtype=np.float64)
    N = y.shape[-1]
    p = np.zeros(y.shape[:-1] + (M,), dtype=np.complex128)
    p[..., (np.arange(N) - N // 2) % M] = y
    return p


def ray_spectrum(y: np.ndarray, M: int, direct: bool = False) -> np.ndarray:
    """P2 + P3: Y_j[k] = dt sum_m p_j[m] exp(-2 pi i k m / M) in natural order."""
    N = y.shape[-1]
    dt = 2.0 / N
    p = pad_center(y, M)
    if direct:
        k = np.arange(M)
        E = np.exp(-2j * np.pi * np.outer(k, k) / M)
        return dt * (p @ E.T)
    return dt * np.fft.fft(p, axis=-1)


# --- P4 --------------------------------------------------------------------

def weight_table(M: int, N: int, mode: str = FILTER, g=None) -> np.ndarray:
    """W[|k|] for |k| = 0..M/2 (P4).  FBP: W = g (g = None: ramp, g = 1).
    Plain B: W[k] = 1/sigma_k = M dt / k, W[0] = 0.  Always W[M/2] = 0."""
    W = np.zeros(M // 2 + 1, dtype=np.float64)
    if mode == FILTER:
        W[: M // 2] = 1.0 if g is None else np.asarray(g, dtype=np.float64)[: M // 2]
    elif mode == BACKPROJECT:
        dt = 2.0 / N
        k = np.arange(1, M // 2, dtype=np.float64)
        W[1 : M // 2] = M * dt / k
    else:
        raise ValueError(mode)
    return W


def apply_weight(Y: np.ndarray, W: np.ndarray) -> np.ndarray:
    M = Y.shape[-1]
    return Y * W[np.abs(signed_index(M))]


def mean_dc(Y: np.ndarray) -> np.ndarray:
    """Every Y_j[0] becomes the mean over angles (the origin is single-valued)."""
    Y = Y.copy()
    Y[..., :, 0] = Y[..., :, 0].mean(axis=-1, keepdims=True)
    return Y


# --- P5 --------------------------------------------------------------------

def polar_taps(M: int, angles, rows=None):
    """P5 geometry.  For the Cartesian frequency points (r', c') (natural order;
    ``rows`` selects a subset of r' indices) return the four taps
    (row j, signed bin k, weight) of their bilinear interpolation in
    (signed radius, angle), each as arrays [4][len(rows)][M], plus a validity mask.

    The point omega = (c', r') dw has radius rho = sqrt(c'^2 + r'^2) in bins.
    It lies on the line through the origin at angle theta in [0, pi) with
    signed radius kappa: kappa = +rho when r' > 0 or (r' = 0, c' >= 0), else
    kappa = -rho and the direction is flipped.  The angle bracket
    theta_J <= theta < theta_{J+1} runs over J = -1..V-1 with
    theta_{-1} = theta_{V-1} - pi and theta_V = theta_0 + pi; a tap on the
    virtual rows -1 or V reads row V-1 or 0 at bin -k (y(-t, theta) =
    y(t, theta + pi)).  Taps at |k| >= M/2 and points with rho >= M/2 are zero.
    """
    th = angles64(angles)
    V = th.size
    ext = np.concatenate(([th[-1] - np.pi], th, [th[0] + np.pi]))
    sg = signed_index(M).astype(np.float64)
    r_idx = np.arange(M) if rows is None else np.asarray(rows)
    R = sg[r_idx][:, None] * np.ones((1, M))
    C = np.ones((r_idx.size, 1)) * sg[None, :]
    rho = np.sqrt(C * C + R * R)
    inside = rho < M / 2
    up = (R > 0) | ((R == 0) & (C >= 0))
    ux = np.where(up, C, -C)
    uy = np.where(up, R, -R)
    theta = np.arctan2(uy, ux)
    kappa = np.where(up, rho, -rho)
    J = np.searchsorted(th, theta, side="right") - 1
    t0 = ext[J + 1]
    t1 = ext[J + 2]
    fth = (theta - t0) / (t1 - t0)
    K0 = np.floor(kappa)
    fk = kappa - K0
    K0 = K0.astype(np.int64)
    rows_out, bins_out, w_out = [], [], []
    for dJ, dK, w in ((0, 0, (1 - fth) * (1 - fk)), (0, 1, (1 - fth) * fk),
                      (1, 0, fth * (1 - fk)), (1, 1, fth * fk)):
        Jv = J + dJ
        K = K0 + dK
        flip = (Jv == -1) | (Jv == V)
        row = np.where(Jv == -1, V - 1, np.where(Jv == V, 0, Jv))
        b = np.where(flip, -K, K)
        ok = inside & (np.abs(b) < M // 2)
        rows_out.append(row)
        bins_out.append(b)
        w_out.append(np.where(ok, w, 0.0))
    return np.stack(rows_out), np.stack(bins_out), np.stack(w_out)


def grid(Z: np.ndarray, angles, block: int = 512) -> np.ndarray:
    """P5: X^[r', c'] = sum of the four weighted taps of Z (gather form)."""
    V, M = Z.shape
    X = np.zeros((M, M), dtype=np.complex128)
    for r0 in range(0, M, block):
        rows = np.arange(r0, min(M, r0 + block))
        jr, kb, w = polar_taps(M, angles, rows)
        X[rows] = np.sum(w * Z[jr, kb % M], axis=0)
    return X


# --- P6 + P7 + P8 ------------------------------------------------------------

def image_from_grid(X: np.ndarray, N: int, direct: bool = False):
    """P6-P8: x_pad = dw^2 sum X^ e^{+2 pi i (r' r_p + c' c_p)/M}, dw = 1/(M d);
    the volume is Re x_pad at r_p = r - N/2, c_p = c - N/2 (fftshift folded
    into the indices).  Returns (volume [N][N], x_pad [M][M] complex)."""
    M = X.shape[0]
    dw = N / (2.0 * M)
    if direct:
        k = np.arange(M)
        E = np.exp(2j * np.pi * np.outer(k, k) / M)
        xp = dw * dw * (E @ X @ E.T)
    else:
        xp = dw * dw * (M * M) * np.fft.ifft2(X)
    idx = (np.arange(N) - N // 2) % M
    return np.real(xp[np.ix_(idx, idx)]), xp


# --- the whole operator -----------------------------------------------------

def bst(y: np.ndarray, angles, pad_factor: int = 2, mode: str = FILTER, g=None,
        direct: bool = False, return_pad: bool = False):
    """BST FBP (mode FILTER, filter taps g, None = ramp) or plain BST
    backprojection (mode BACKPROJECT) of one sinogram y[V][N] -> [N][N]."""
    y = np.asarray(y, dtype=np.float64)
    V, N = y.shape
    M = pad_factor * N
    angles64(angles)
    Y = ray_spectrum(y, M, direct)                                 # P2, P3
    return bst_from_spectrum(Y, angles, N, mode, g, direct, return_pad)


def bst_from_spectrum(Y: np.ndarray, angles, N: int, mode: str = FILTER, g=None,
                      direct: bool = False, return_pad: bool = False):
    """Stages P4-P8 applied to the ray spectrum Y[V][M] of P3."""
    M = Y.shape[-1]
    Z = mean_dc(apply_weight(Y, weight_table(M, N, mode, g)))      # P4
    X = grid(Z, angles)                                            # P0, P5
    vol, xp = image_from_grid(X, N, direct)                        # P6-P8
    return (vol, xp) if return_pad else vol


def fbp(y, angles, pad_factor: int = 2, g=None, direct: bool = False):
    return bst(y, angles, pad_factor, FILTER, g, direct)


def backproject(y, angles, pad_factor: int = 2, direct: bool = False):
    return bst(y, angles, pad_factor, BACKPROJECT, None, direct)
