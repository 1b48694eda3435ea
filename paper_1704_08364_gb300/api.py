"""Python binding of libbst: the C-ABI calls of include/bst.h on torch tensors.

Argument marshalling only: every step of the BST path runs in the library's
CUDA kernels.  Tensors must be contiguous float32 CUDA tensors; work is
enqueued on torch's current stream.  Workspaces are torch allocations owned
by the Plan object and grown on demand.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib

FILTER = 0
BACKPROJECT = 1
GRID_BILINEAR = 0
GRID_KAISER_BESSEL = 1


class BstError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = _lib.load().bst_status_string(code).decode()
        super().__init__(f"{where}: {msg} (status {code})")
        self.code = code


def _check(code: int, where: str):
    if code != 0:
        raise BstError(code, where)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _need(t, name, shape=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")


class Plan:
    """A BST plan for N detector samples (rays), the given float32 angles in
    [0, pi) (strictly increasing) and pad factor alpha (FFT length M = alpha N)."""

    def __init__(self, rays: int, angles, pad_factor: int = 2):
        lib = _lib.load()
        th = np.ascontiguousarray(np.asarray(angles, dtype=np.float32))
        h = ctypes.c_void_p()
        _check(lib.bst_plan_create(ctypes.byref(h), int(rays), int(th.size),
                                   th.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), int(pad_factor)),
               "bst_plan_create")
        self._h = h
        self._lib = lib
        self.rays = int(rays)
        self.angles = th.copy()
        self.V = int(th.size)
        self.pad_factor = int(pad_factor)
        self.M = lib.bst_plan_fft_length(h)
        self._ws = {}

    @property
    def handle(self):
        return self._h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                self._lib.bst_plan_destroy(h)
            except Exception:
                pass
            self._h = None

    def workspace(self, kind: str, nbytes: int, device) -> torch.Tensor:
        key = (kind, str(device))
        buf = self._ws.get(key)
        if buf is None or buf.numel() < nbytes:
            buf = torch.empty(max(nbytes, 16), dtype=torch.uint8, device=device)
            self._ws[key] = buf
        return buf

    def workspace_bytes(self, slices: int) -> int:
        return int(self._lib.bst_workspace_bytes(self._h, int(slices)))

    def adjoint_workspace_bytes(self, slices: int) -> int:
        return int(self._lib.bst_adjoint_workspace_bytes(self._h, int(slices)))

    def brute_workspace_bytes(self, slices: int, filtered: bool) -> int:
        return int(self._lib.brute_workspace_bytes(self._h, int(slices), int(bool(filtered))))

    def status(self):
        _check(self._lib.bst_plan_status(self._h, _stream()), "bst_plan_status")

    @property
    def schedule(self) -> int:
        """Largest FFT radix of the forward path's Stockham passes (16 or 8)."""
        return int(self._lib.bst_plan_get_schedule(self._h))

    @schedule.setter
    def schedule(self, max_radix: int):
        _check(self._lib.bst_plan_set_schedule(self._h, int(max_radix)), "bst_plan_set_schedule")

    @property
    def forward_config(self) -> dict:
        """Launch shape of the forward path (bst_plan_get_forward_config):
        max_radix, layout ("packed" or "paired"), chunk_pairs, pair_fast, max_lanes,
        grid_xchg (1: register-fed paired gridding, 0: through shared memory)."""
        c = _lib.FwdConfig()
        _check(self._lib.bst_plan_get_forward_config(self._h, ctypes.byref(c)), "bst_plan_get_forward_config")
        return {"max_radix": c.max_radix, "layout": "paired" if c.layout == 1 else "packed",
                "chunk_pairs": c.chunk_pairs, "pair_fast": c.pair_fast, "max_lanes": c.max_lanes,
                "grid_xchg": c.grid_xchg}

    def set_forward_config(self, **kw):
        """Change fields of the launch shape (bst_plan_set_forward_config);
        results are identical up to rounding whatever the shape."""
        cur = self.forward_config
        cur.update(kw)
        layout = {"packed": 0, "paired": 1}.get(cur["layout"], cur["layout"])
        c = _lib.FwdConfig(int(cur["max_radix"]), int(layout),
                           int(cur["chunk_pairs"]), int(cur["pair_fast"]), int(cur["max_lanes"]),
                           int(cur["grid_xchg"]))
        _check(self._lib.bst_plan_set_forward_config(self._h, ctypes.byref(c)), "bst_plan_set_forward_config")
        return self

    @property
    def gridding(self) -> tuple[str, int]:
        """Interpolation kernel of stage P5: ("bilinear", 2) or ("kaiser-bessel", W)."""
        kind, width = ctypes.c_int(0), ctypes.c_int(0)
        _check(self._lib.bst_plan_get_gridding(self._h, ctypes.byref(kind), ctypes.byref(width)),
               "bst_plan_get_gridding")
        return ("kaiser-bessel" if kind.value == GRID_KAISER_BESSEL else "bilinear", int(width.value))

    def set_gridding(self, kind: str = "bilinear", width: int = 6):
        """Select bilinear interpolation or Kaiser-Bessel gridding of width W bins
        (bst_plan_set_gridding; builds the KB tables, synchronises the device)."""
        k = {"bilinear": GRID_BILINEAR, "kaiser-bessel": GRID_KAISER_BESSEL, "kb": GRID_KAISER_BESSEL}[kind]
        _check(self._lib.bst_plan_set_gridding(self._h, k, int(width)), "bst_plan_set_gridding")
        return self

    def autotune(self, slices: int = 0, cache: str | None = None) -> dict:
        """Pick the fastest launch shape of the forward path by timing the
        candidates (bst_plan_autotune: radix schedule, spectrum layout, chunk
        and block order) and return it (forward_config).  With a cache path
        (default: $BST_AUTOTUNE_CACHE if set) the choice is stored per (GPU
        name, N, V, pad factor, gridding) and reused without timing."""
        import json
        import os
        cache = cache or os.environ.get("BST_AUTOTUNE_CACHE")
        key = f"{torch.cuda.get_device_name()}|N={self.rays}|V={self.V}|pad={self.pad_factor}|grid={self.gridding}"
        table = {}
        if cache and os.path.exists(cache):
            try:
                with open(cache) as f:
                    table = json.load(f)
            except (OSError, ValueError):
                table = {}
        entry = table.get(key)
        if isinstance(entry, dict):
            self.set_forward_config(**entry)
            return self.forward_config
        chosen = ctypes.c_int(0)
        _check(self._lib.bst_plan_autotune(self._h, int(slices), ctypes.byref(chosen)), "bst_plan_autotune")
        cfg = self.forward_config
        if cache:
            table[key] = cfg
            os.makedirs(os.path.dirname(os.path.abspath(cache)), exist_ok=True)
            with open(cache, "w") as f:
                json.dump(table, f, indent=1, sort_keys=True)
        return cfg

    # -- forward -------------------------------------------------------------

    def _forward(self, sino, g, out, mode):
        _need(sino, "sino")
        if sino.dim() == 2:
            sino = sino.unsqueeze(0)
        S = sino.shape[0]
        _need(sino, "sino", (S, self.V, self.rays))
        if g is not None:
            _need(g, "g", (self.M // 2,))
        if out is None:
            out = torch.empty((S, self.rays, self.rays), dtype=torch.float32, device=sino.device)
        _need(out, "out", (S, self.rays, self.rays))
        nb = self.workspace_bytes(S)
        ws = self.workspace("fwd", nb, sino.device)
        if mode == FILTER:
            code = self._lib.bst_fbp(self._h, _ptr(sino), S, _ptr(g), _ptr(out), _ptr(ws), ws.numel(), _stream())
            _check(code, "bst_fbp")
        else:
            code = self._lib.bst_backproject(self._h, _ptr(sino), S, _ptr(out), _ptr(ws), ws.numel(), _stream())
            _check(code, "bst_backproject")
        return out

    def fbp(self, sino, g=None, out=None):
        """BST filtered backprojection of sino [S][V][N] -> [S][N][N]."""
        return self._forward(sino, g, out, FILTER)

    def fbp_prep(self, sino, flat=None, dark=None, shift: float = 0.0, kb_beta: float = 0.0,
                 kb_halfwidth: float = 1.0, g=None, out=None):
        """bst_fbp_prep: normalization from counts (flat/dark rows [S][N]),
        centering by `shift` detector samples and the Kaiser-Bessel window P1,
        fused into the ray stage of the filtered backprojection."""
        _need(sino, "sino")
        S = sino.shape[0]
        _need(sino, "sino", (S, self.V, self.rays))
        for t, name in ((flat, "flat"), (dark, "dark")):
            if t is not None:
                _need(t, name, (S, self.rays))
        if g is not None:
            _need(g, "g", (self.M // 2,))
        if out is None:
            out = torch.empty((S, self.rays, self.rays), dtype=torch.float32, device=sino.device)
        _need(out, "out", (S, self.rays, self.rays))
        ws = self.workspace("fwd", self.workspace_bytes(S), sino.device)
        _check(self._lib.bst_fbp_prep(self._h, _ptr(sino), S, _ptr(dark), _ptr(flat), float(shift), float(kb_beta),
                                      float(kb_halfwidth), _ptr(g), _ptr(out), _ptr(ws), ws.numel(), _stream()),
               "bst_fbp_prep")
        return out

    def fbp_noalloc(self, sino, g=None, out=None):
        """As fbp, through bst_fbp_noalloc: the library's fixed scratch array
        instead of a workspace (the output tensor is still the caller's)."""
        _need(sino, "sino")
        if sino.dim() == 2:
            sino = sino.unsqueeze(0)
        S = sino.shape[0]
        _need(sino, "sino", (S, self.V, self.rays))
        if g is not None:
            _need(g, "g", (self.M // 2,))
        if out is None:
            out = torch.empty((S, self.rays, self.rays), dtype=torch.float32, device=sino.device)
        _need(out, "out", (S, self.rays, self.rays))
        _check(self._lib.bst_fbp_noalloc(self._h, _ptr(sino), S, _ptr(g), _ptr(out), _stream()), "bst_fbp_noalloc")
        return out

    def fbp_host(self, sino, g=None, out=None, device=None):
        """BST FBP of a host-resident volume (CPU float32 tensors, ideally pinned)
        through bst_fbp_host: uploads, kernels and downloads overlap in chunks.
        Returns `out` once the work is complete."""
        if not isinstance(sino, torch.Tensor) or sino.is_cuda or sino.dtype != torch.float32 \
                or not sino.is_contiguous():
            raise ValueError("sino must be a contiguous float32 CPU tensor")
        S = sino.shape[0]
        if tuple(sino.shape) != (S, self.V, self.rays):
            raise ValueError("sino has the wrong shape")
        if out is None:
            out = torch.empty((S, self.rays, self.rays), dtype=torch.float32, pin_memory=sino.is_pinned())
        if out.is_cuda or out.dtype != torch.float32 or not out.is_contiguous() or \
                tuple(out.shape) != (S, self.rays, self.rays):
            raise ValueError("out must be a contiguous float32 CPU tensor of shape [S][N][N]")
        if g is not None:
            _need(g, "g", (self.M // 2,))
        dev = device or torch.device("cuda", torch.cuda.current_device())
        nb = int(self._lib.bst_host_workspace_bytes(self._h, S))
        ws = self.workspace("host", nb, dev)
        _check(self._lib.bst_fbp_host(self._h, _ptr(sino), S, _ptr(g), _ptr(out), _ptr(ws), ws.numel(), _stream()),
               "bst_fbp_host")
        torch.cuda.current_stream().synchronize()
        return out

    def backproject(self, sino, out=None):
        """Plain BST backprojection (1/sigma weight, zero DC)."""
        return self._forward(sino, None, out, BACKPROJECT)

    def radon_adjoint(self, vol, mode: int = FILTER, g=None, out=None):
        """Transpose of fbp (mode FILTER, taps g) or backproject (mode BACKPROJECT)."""
        _need(vol, "vol")
        if vol.dim() == 2:
            vol = vol.unsqueeze(0)
        S = vol.shape[0]
        _need(vol, "vol", (S, self.rays, self.rays))
        if g is not None:
            _need(g, "g", (self.M // 2,))
        if out is None:
            out = torch.empty((S, self.V, self.rays), dtype=torch.float32, device=vol.device)
        _need(out, "out", (S, self.V, self.rays))
        nb = self.adjoint_workspace_bytes(S)
        ws = self.workspace("adj", nb, vol.device)
        _check(self._lib.radon_adjoint(self._h, int(mode), _ptr(g), _ptr(vol), S, _ptr(out), _ptr(ws), ws.numel(),
                                       _stream()), "radon_adjoint")
        return out

    def filter_grad(self, sino, grad_vol, out=None):
        """d/dg of sum(grad_vol * fbp(sino, g)) -> [M/2]."""
        _need(sino, "sino")
        _need(grad_vol, "grad_vol")
        S = sino.shape[0]
        _need(sino, "sino", (S, self.V, self.rays))
        _need(grad_vol, "grad_vol", (S, self.rays, self.rays))
        if out is None:
            out = torch.empty((self.M // 2,), dtype=torch.float32, device=sino.device)
        nb = self.adjoint_workspace_bytes(S)
        ws = self.workspace("adj", nb, sino.device)
        _check(self._lib.bst_fbp_filter_grad(self._h, _ptr(sino), _ptr(grad_vol), S, _ptr(out), _ptr(ws),
                                             ws.numel(), _stream()), "bst_fbp_filter_grad")
        return out

    def fbp_backward(self, sino, grad_vol, g=None, want_sino: bool = True, want_g: bool = True):
        """Both gradients of sum(grad_vol * fbp(sino, g)) from one polar pull-back
        (bst_fbp_backward): (grad_sino [S][V][N] or None, grad_g [M/2] or None)."""
        _need(grad_vol, "grad_vol")
        S = grad_vol.shape[0]
        _need(grad_vol, "grad_vol", (S, self.rays, self.rays))
        if want_g:
            _need(sino, "sino", (S, self.V, self.rays))
        if g is not None:
            _need(g, "g", (self.M // 2,))
        dev = grad_vol.device
        gs = torch.empty((S, self.V, self.rays), dtype=torch.float32, device=dev) if want_sino else None
        gg = torch.empty((self.M // 2,), dtype=torch.float32, device=dev) if want_g else None
        nb = self.adjoint_workspace_bytes(S)
        ws = self.workspace("adj", nb, dev)
        _check(self._lib.bst_fbp_backward(self._h, _ptr(sino if want_g else None), _ptr(grad_vol), S, _ptr(g),
                                          _ptr(gs), _ptr(gg), _ptr(ws), ws.numel(), _stream()), "bst_fbp_backward")
        return gs, gg

    def brute_backproject(self, sino, g=None, out=None):
        """Slant-stack backprojection (Eq. 2); with taps g, SS filtered backprojection."""
        _need(sino, "sino")
        if sino.dim() == 2:
            sino = sino.unsqueeze(0)
        S = sino.shape[0]
        _need(sino, "sino", (S, self.V, self.rays))
        if g is not None:
            _need(g, "g", (self.M // 2,))
        if out is None:
            out = torch.empty((S, self.rays, self.rays), dtype=torch.float32, device=sino.device)
        nb = self.brute_workspace_bytes(S, g is not None)
        ws = self.workspace("brute", nb, sino.device) if nb > 0 else None
        _check(self._lib.brute_backproject(self._h, _ptr(sino), S, _ptr(g), _ptr(out), _ptr(ws),
                                           0 if ws is None else ws.numel(), _stream()), "brute_backproject")
        return out


class BstFbpFn(torch.autograd.Function):
    """x = FBP(p; g) with gradients for the sinogram p and the filter taps g.
    Backward (bst_fbp_backward): grad_p = radon_adjoint(grad_x) (the Fourier-slice
    transpose) and grad_g = filter_grad(p, grad_x) from one polar pull-back of
    grad_x; the FFT intermediates are recomputed, not stored."""

    @staticmethod
    def forward(ctx, sino, g, plan: Plan):
        ctx.plan = plan
        ctx.save_for_backward(sino, g)
        return plan.fbp(sino.contiguous(), g.contiguous())

    @staticmethod
    def backward(ctx, grad_x):
        sino, g = ctx.saved_tensors
        plan = ctx.plan
        gx = grad_x.contiguous()
        want_p, want_g = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if not (want_p or want_g):
            return None, None, None
        gp, gg = plan.fbp_backward(sino.contiguous(), gx, g.contiguous(), want_p, want_g)
        return gp, gg, None


def fbp_autograd(sino, g, plan: Plan):
    return BstFbpFn.apply(sino, g, plan)


class RaggedBatch:
    """Sinograms of mixed sizes reconstructed by one persistent launch
    (bst_ragged_*).  plans[i] is the plan of item i; items sharing a plan are
    paired.  bind() fixes the device buffers; run() launches (optionally from a
    captured CUDA graph)."""

    def __init__(self, plans):
        self._lib = _lib.load()
        self.plans = list(plans)
        arr = (ctypes.c_void_p * len(self.plans))(*[p.handle.value for p in self.plans])
        h = ctypes.c_void_p()
        _check(self._lib.bst_ragged_create(ctypes.byref(h), len(self.plans), arr), "bst_ragged_create")
        self._h = h
        self._ws = None
        self._bound = None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                self._lib.bst_ragged_destroy(h)
            except Exception:
                pass
            self._h = None

    @property
    def pair_items(self) -> int:
        return int(self._lib.bst_ragged_pair_items(self._h))

    def bind(self, sinos, volumes, gs=None, flags: int = 0):
        n = len(self.plans)
        if len(sinos) != n or len(volumes) != n:
            raise ValueError("one sinogram and one volume per item")
        for p, sg, v in zip(self.plans, sinos, volumes):
            _need(sg, "sino", (p.V, p.rays))
            _need(v, "volume", (p.rays, p.rays))
        nb = int(self._lib.bst_ragged_workspace_bytes(self._h))
        dev = sinos[0].device
        if self._ws is None or self._ws.numel() < nb:
            self._ws = torch.empty(nb, dtype=torch.uint8, device=dev)
        s_arr = (ctypes.c_void_p * n)(*[t.data_ptr() for t in sinos])
        v_arr = (ctypes.c_void_p * n)(*[t.data_ptr() for t in volumes])
        g_arr = None if gs is None else (ctypes.c_void_p * n)(*[0 if g is None else g.data_ptr() for g in gs])
        _check(self._lib.bst_ragged_bind(self._h, s_arr, g_arr, v_arr, _ptr(self._ws), self._ws.numel(), int(flags)),
               "bst_ragged_bind")
        self._bound = (list(sinos), list(volumes), gs)   # keep the buffers alive
        return self

    def set_spin_limit(self, iterations: int):
        _check(self._lib.bst_ragged_set_spin_limit(self._h, int(iterations)), "bst_ragged_set_spin_limit")

    def run(self, use_graph: bool = False):
        _check(self._lib.bst_ragged_fbp(self._h, int(bool(use_graph)), _stream()), "bst_ragged_fbp")

    def status(self) -> int:
        """Synchronise; return (and clear) the device status code (0 = ok)."""
        return int(self._lib.bst_ragged_status(self._h, _stream()))


# ---------------------------------------------------------------------------
# Module-level calls: each takes the geometry with the data, builds the plan on
# first use (one per device, ray count, angle list and pad factor, kept until
# clear_plans()) and calls that plan's method.

_PLANS: dict = {}


def _device_index() -> int:
    return torch.cuda.current_device()


def plan_for(rays: int, angles, pad_factor: int = 2) -> Plan:
    """The cached plan of this geometry on the current device."""
    th = np.ascontiguousarray(np.asarray(angles, dtype=np.float32))
    key = (_device_index(), int(rays), int(pad_factor), th.tobytes())
    plan = _PLANS.get(key)
    if plan is None:
        plan = _PLANS[key] = Plan(rays, th, pad_factor)
    return plan


def clear_plans():
    """Drop the cached plans (and their device tables)."""
    _PLANS.clear()


def fbp(sino, angles, pad_factor: int = 2, g=None, out=None):
    """BST filtered backprojection of sino [S][V][N] (or [V][N]) at the angles
    theta_j (radians, [0, pi), increasing) -> volume [S][N][N]."""
    return plan_for(sino.shape[-1], angles, pad_factor).fbp(sino, g=g, out=out)


def backproject(sino, angles, pad_factor: int = 2, out=None):
    """Plain BST backprojection b = B y (Eq. 2 through Eq. 3), defined up to a
    constant (zero DC)."""
    return plan_for(sino.shape[-1], angles, pad_factor).backproject(sino, out=out)


def radon_adjoint(vol, angles, mode: int = FILTER, g=None, pad_factor: int = 2, out=None):
    """Transpose of fbp (mode FILTER, taps g) or of backproject (mode
    BACKPROJECT): volume [S][N][N] -> sinogram [S][V][N]."""
    return plan_for(vol.shape[-1], angles, pad_factor).radon_adjoint(vol, mode=mode, g=g, out=out)


def brute_backproject(sino, angles, g=None, pad_factor: int = 2, out=None):
    """Slant-stack backprojection (Eq. 2), the O(N^3) comparator; with taps g
    the slant-stack filtered backprojection."""
    return plan_for(sino.shape[-1], angles, pad_factor).brute_backproject(sino, g=g, out=out)


def fbp_ragged(sinos, angles=None, pad_factor: int = 2, gs=None, use_graph: bool = False):
    """BST FBP of sinograms of mixed sizes (sinos[i]: [V_i][N_i]) in one
    persistent launch.  angles[i] are item i's angles (default j pi / V_i);
    items with the same geometry share a plan and are paired.  Blocks until
    the launch is done and returns the volumes [N_i][N_i]."""
    n = len(sinos)
    if angles is None:
        angles = [np.arange(s.shape[0], dtype=np.float64) * np.pi / s.shape[0] for s in sinos]
    if len(angles) != n:
        raise ValueError("one angle list per sinogram")
    plans = [plan_for(s.shape[-1], a, pad_factor) for s, a in zip(sinos, angles)]
    vols = [torch.empty((p.rays, p.rays), dtype=torch.float32, device=s.device) for p, s in zip(plans, sinos)]
    batch = RaggedBatch(plans).bind(list(sinos), vols, gs)
    batch.run(use_graph)
    code = batch.status()
    if code != 0:
        raise BstError(code, "bst_ragged_fbp")
    return vols
