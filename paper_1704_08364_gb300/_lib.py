"""ctypes loader of libbst.so: argument marshalling only, no computation.

The library is built in-tree by ``paper_1704_08364_gb300.build``; loading
fails loudly when it is missing (there is no fallback implementation)."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbst.so")

class FwdConfig(ctypes.Structure):
    """bst_fwd_config_t: the launch shape of the forward path."""
    _fields_ = [("max_radix", ctypes.c_int), ("layout", ctypes.c_int), ("chunk_pairs", ctypes.c_int),
                ("pair_fast", ctypes.c_int), ("max_lanes", ctypes.c_int), ("grid_xchg", ctypes.c_int)]


c_plan = ctypes.c_void_p
c_ptr = ctypes.c_void_p
c_int = ctypes.c_int
c_size = ctypes.c_size_t

# name -> (restype, argtypes); mirrors include/bst.h
SIGNATURES = {
    "bst_plan_create": (c_int, [ctypes.POINTER(c_plan), c_int, c_int, ctypes.POINTER(ctypes.c_float), c_int]),
    "bst_plan_destroy": (c_int, [c_plan]),
    "bst_workspace_bytes": (c_size, [c_plan, c_int]),
    "bst_fbp": (c_int, [c_plan, c_ptr, c_int, c_ptr, c_ptr, c_ptr, c_size, c_ptr]),
    "bst_backproject": (c_int, [c_plan, c_ptr, c_int, c_ptr, c_ptr, c_size, c_ptr]),
    "bst_fbp_prep": (c_int, [c_plan, c_ptr, c_int, c_ptr, c_ptr, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                             c_ptr, c_ptr, c_ptr, c_size, c_ptr]),
    "bst_adjoint_workspace_bytes": (c_size, [c_plan, c_int]),
    "radon_adjoint": (c_int, [c_plan, c_int, c_ptr, c_ptr, c_int, c_ptr, c_ptr, c_size, c_ptr]),
    "bst_fbp_filter_grad": (c_int, [c_plan, c_ptr, c_ptr, c_int, c_ptr, c_ptr, c_size, c_ptr]),
    "brute_workspace_bytes": (c_size, [c_plan, c_int, c_int]),
    "brute_backproject": (c_int, [c_plan, c_ptr, c_int, c_ptr, c_ptr, c_ptr, c_size, c_ptr]),
    "bst_plan_status": (c_int, [c_plan, c_ptr]),
    "bst_status_string": (ctypes.c_char_p, [c_int]),
    "bst_plan_fft_length": (c_int, [c_plan]),
    "bst_fbp_noalloc": (c_int, [c_plan, c_ptr, c_int, c_ptr, c_ptr, c_ptr]),
    "bst_host_workspace_bytes": (c_size, [c_plan, c_int]),
    "bst_fbp_host": (c_int, [c_plan, c_ptr, c_int, c_ptr, c_ptr, c_ptr, c_size, c_ptr]),
    "bst_noalloc_scratch_bytes": (c_size, []),
    "bst_plan_set_schedule": (c_int, [c_plan, c_int]),
    "bst_plan_get_schedule": (c_int, [c_plan]),
    "bst_fbp_backward": (c_int, [c_plan, c_ptr, c_ptr, c_int, c_ptr, c_ptr, c_ptr, c_ptr, ctypes.c_size_t, c_ptr]),
    "bst_plan_set_gridding": (c_int, [c_plan, c_int, c_int]),
    "bst_plan_get_gridding": (c_int, [c_plan, ctypes.POINTER(c_int), ctypes.POINTER(c_int)]),
    "bst_plan_autotune": (c_int, [c_plan, c_int, ctypes.POINTER(c_int)]),
    "bst_plan_set_forward_config": (c_int, [c_plan, ctypes.POINTER(FwdConfig)]),
    "bst_plan_get_forward_config": (c_int, [c_plan, ctypes.POINTER(FwdConfig)]),
    "bst_ragged_create": (c_int, [ctypes.POINTER(c_ptr), c_int, ctypes.POINTER(c_plan)]),
    "bst_ragged_workspace_bytes": (c_size, [c_ptr]),
    "bst_ragged_pair_items": (c_int, [c_ptr]),
    "bst_ragged_bind": (c_int, [c_ptr, ctypes.POINTER(c_ptr), ctypes.POINTER(c_ptr), ctypes.POINTER(c_ptr), c_ptr,
                                c_size, c_int]),
    "bst_ragged_set_spin_limit": (c_int, [c_ptr, c_int]),
    "bst_ragged_fbp": (c_int, [c_ptr, c_int, c_ptr]),
    "bst_ragged_status": (c_int, [c_ptr, c_ptr]),
    "bst_ragged_destroy": (c_int, [c_ptr]),
    "bst_plan_set_timing": (c_int, [c_plan, c_int]),
    "bst_plan_timing": (c_int, [c_plan, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong), c_int]),
}

_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
