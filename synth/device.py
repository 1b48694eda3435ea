"""ctypes binding of libbstsynth.so, the device-side generator of the large
ellipse-phantom workloads (input generation only)."""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from .phantom import ellipse_table, random_ellipses, slice_seed, uniform_angles

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libbstsynth.so")
_lib = None


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built")
        lib = ctypes.CDLL(LIB_PATH)
        lib.synth_ellipse_sinogram.restype = ctypes.c_int
        lib.synth_ellipse_sinogram.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                               ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                               ctypes.c_void_p]
        lib.synth_add_gaussian_noise.restype = ctypes.c_int
        lib.synth_add_gaussian_noise.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_float, ctypes.c_ulonglong, ctypes.c_longlong,
                                                 ctypes.c_void_p, ctypes.c_void_p]
        _lib = lib
    return _lib


def ellipse_volume(config_index: int, slices: int, angles: int, rays: int, noise_frac: float = 0.0,
                   device="cuda", out=None, kmax: int = 20, first_slice: int = 0) -> torch.Tensor:
    """[slices][angles][rays] float32 sinograms of seeded random ellipse phantoms
    (same per-slice seeds as the host generator), generated on the device.
    ``first_slice``: the index of the first slice in the whole volume; the
    slices and their noise equal those slices of the whole volume generated
    at once (first_slice * angles * rays must be even)."""
    lib = _load()
    lists = [random_ellipses(np.random.default_rng(slice_seed(config_index, first_slice + s)))
             for s in range(slices)]
    tab, cnt = ellipse_table(lists, kmax)
    d_tab = torch.from_numpy(tab).to(device)
    d_cnt = torch.from_numpy(cnt).to(device)
    d_th = torch.from_numpy(uniform_angles(angles)).to(device)
    if out is None:
        out = torch.empty((slices, angles, rays), dtype=torch.float32, device=device)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.synth_ellipse_sinogram(d_tab.data_ptr(), d_cnt.data_ptr(), kmax, d_th.data_ptr(), slices, angles, rays,
                                    out.data_ptr(), st)
    if rc:
        raise RuntimeError(f"synth_ellipse_sinogram failed ({rc})")
    if noise_frac > 0:
        smax = torch.empty((slices,), dtype=torch.float32, device=device)
        rc = lib.synth_add_gaussian_noise(out.data_ptr(), slices, angles, rays, float(noise_frac),
                                          slice_seed(config_index, 0), first_slice, smax.data_ptr(), st)
        if rc:
            raise RuntimeError(f"synth_add_gaussian_noise failed ({rc})")
    return out
