"""Helpers of the GPU parity tests (host side only)."""
import numpy as np


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def assert_parity(got, ref, rtol_l2=1e-5, atol_frac=1e-4, what=""):
    """The floating-point bar of the path: relative L2 <= 1e-5 and
    max-abs <= 1e-4 * max|ref| against the FP64 oracle."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    r = rel_l2(got, ref)
    m = float(np.abs(got - ref).max())
    lim = atol_frac * float(np.abs(ref).max())
    assert r <= rtol_l2 and m <= lim, f"{what}: rel L2 {r:.3e} (<= {rtol_l2}), max abs {m:.3e} (<= {lim:.3e})"
    return r
