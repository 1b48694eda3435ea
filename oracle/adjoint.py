"""Adjoint of the discrete BST operator and the filter-tap gradient (FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The BST operator A (oracle.bst.bst, stages P2..P8) is a real matrix from
sinograms [V][N] to images [N][N].  Its transpose is the composition of the
adjoints of the stages in reverse order:

    crop          -> zero extension into the M x M grid
    2D IFFT * dw^2 -> dw^2 * 2D DFT with the opposite exponent
    gridding      -> scatter of each Cartesian value onto its four polar taps
                     with the same bilinear weights
    DC mean map   -> itself (a symmetric averaging matrix)
    weight W      -> itself (a real diagonal)
    dt * 1D DFT   -> dt * 1D DFT with the opposite exponent
    zero padding  -> crop to the N detector samples

and the real part is taken at the end.  Read in the other direction this is
a Fourier-slice projector (the "FST" dual of the BST, Sec. 2): image ->
2D spectrum -> polar samples -> 1D inverse transforms along t.

For L(g) = ||A_g p - f||^2 with residual gradient R = dL/dx = 2 (A_g p - f):
dL/dg[m] = sum over j and |k| = m of Re(conj(lam_j[k]) * Y0_j[k]), where
Y0 = dt DFT of the padded rays (before weight and mean) and lam is R pulled
back through the crop, the 2D transform, the gridding and the mean map.
dL/dp = A_g^T R.
"""
from __future__ import annotations

import numpy as np

from .bst import FILTER, angles64, polar_taps, ray_spectrum, signed_index, weight_table


def grid_transpose(X: np.ndarray, angles, block: int = 512) -> np.ndarray:
    """Adjoint of oracle.bst.grid: lam[j, k] += w * X[r', c'] over the four taps."""
    M = X.shape[0]
    V = angles64(angles).size
    lam_re = np.zeros(V * M, dtype=np.float64)
    lam_im = np.zeros(V * M, dtype=np.float64)
    for r0 in range(0, M, block):
        rows = np.arange(r0, min(M, r0 + block))
        jr, kb, w = polar_taps(M, angles, rows)
        flat = (jr * M + (kb % M)).reshape(-1)
        xv = np.broadcast_to(X[rows][None], w.shape)
        lam_re += np.bincount(flat, weights=(w * xv.real).reshape(-1), minlength=V * M)
        lam_im += np.bincount(flat, weights=(w * xv.imag).reshape(-1), minlength=V * M)
    return (lam_re + 1j * lam_im).reshape(V, M)


def polar_pullback(f: np.ndarray, angles, pad_factor: int = 2) -> np.ndarray:
    """lam = Mean^T Grid^T (2D IFFT * dw^2)^H Crop^T f for one image f[N][N]."""
    f = np.asarray(f, dtype=np.float64)
    N = f.shape[-1]
    M = pad_factor * N
    dw = N / (2.0 * M)
    idx = (np.arange(N) - N // 2) % M
    xp = np.zeros((M, M), dtype=np.complex128)
    xp[np.ix_(idx, idx)] = f
    Xh = dw * dw * np.fft.fft2(xp)
    lam = grid_transpose(Xh, angles)
    lam[:, 0] = lam[:, 0].mean()
    return lam


def bst_adjoint(f: np.ndarray, angles, pad_factor: int = 2, mode: str = FILTER, g=None) -> np.ndarray:
    """A^T f for one image f[N][N] -> sinogram [V][N] (the radon_adjoint operator)."""
    f = np.asarray(f, dtype=np.float64)
    N = f.shape[-1]
    M = pad_factor * N
    dt = 2.0 / N
    lam = polar_pullback(f, angles, pad_factor)
    lam = lam * weight_table(M, N, mode, g)[np.abs(signed_index(M))]
    q = dt * M * np.fft.ifft(lam, axis=1)
    return np.real(q[:, (np.arange(N) - N // 2) % M])


def filter_grad(p: np.ndarray, R: np.ndarray, angles, pad_factor: int = 2) -> np.ndarray:
    """d/dg[m] of sum(R * A_g p) for m = 0..M/2-1 (R = dL/dx)."""
    p = np.asarray(p, dtype=np.float64)
    N = p.shape[-1]
    M = pad_factor * N
    Y0 = ray_spectrum(p, M)
    lam = polar_pullback(R, angles, pad_factor)
    prod = np.real(np.conj(lam) * Y0).sum(axis=0)
    ak = np.abs(signed_index(M))
    out = np.bincount(ak, weights=prod, minlength=M // 2 + 1)
    return out[: M // 2]
