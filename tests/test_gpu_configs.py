"""GPU parity on the exact shapes of the ragged and autograd workloads, and the
edge cases of the path: the largest FFT length, the fewest angles, an empty
batch."""
import ctypes

import numpy as np
import pytest

import synth
from oracle import adjoint as oa
from oracle import bst as ob
from gpu_util import assert_parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bst():
    import paper_1704_08364_gb300 as m
    return m


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_ragged_64_workload(bst):
    """The 64-item ragged batch (rays from {256 ... 2048}, angles = rays): every
    item of the persistent launch against the same item through its own plan,
    two small items against the oracle."""
    sizes = synth.ragged_sizes()
    plans = {N: bst.Plan(N, synth.uniform_angles(N), 2) for N in sorted(set(sizes))}
    rng = np.random.default_rng(64)
    host = []
    for N in sizes:
        th = synth.uniform_angles(N)
        host.append(synth.gaussian_noise(synth.ellipse_sinogram(synth.random_ellipses(rng), th, N), rng))
    sinos = [_cuda(h) for h in host]
    vols = [torch.full((N, N), float("nan"), device="cuda") for N in sizes]
    rb = bst.RaggedBatch([plans[N] for N in sizes]).bind(sinos, vols)
    rb.run(True)
    assert rb.status() == 0
    for i, (N, s, v) in enumerate(zip(sizes, sinos, vols)):
        ref = plans[N].fbp(s.unsqueeze(0))[0].cpu().numpy()
        assert_parity(v.cpu().numpy(), ref, what=f"ragged-64 item {i} (N={N})")
    small = [i for i, N in enumerate(sizes) if N == min(sizes)][:2]
    for i in small:
        th = synth.uniform_angles(sizes[i])
        assert_parity(vols[i].cpu().numpy(), ob.fbp(host[i].astype(np.float32).astype(np.float64), th),
                      what=f"ragged-64 item {i} vs oracle")


def test_autograd_1024_geometry(bst):
    """The autograd workload's full geometry (1024 angles x 1024 rays, 1024
    taps), two of its sixteen slices: both gradients against the oracle."""
    N = V = 1024
    theta, p, imgs = synth.workload_slices("autograd-1024", [0, 1], with_images=True, supersample=1)
    plan = bst.Plan(N, theta, 2)
    dp = _cuda(p).requires_grad_(True)
    g = torch.ones(N, device="cuda", requires_grad=True)
    x = bst.fbp_autograd(dp, g, plan)
    ((x - _cuda(imgs)) ** 2).sum().backward()
    xr = np.stack([ob.fbp(s.astype(np.float64), theta) for s in p])
    R = 2.0 * (xr - imgs.astype(np.float32).astype(np.float64))
    gp_ref = np.stack([oa.bst_adjoint(R[s], theta) for s in range(2)])
    gg_ref = sum(oa.filter_grad(p[s].astype(np.float64), R[s], theta) for s in range(2))
    assert_parity(dp.grad.cpu().numpy(), gp_ref, what="grad p (1024)")
    assert_parity(g.grad.cpu().numpy(), gg_ref, what="grad g (1024)")


def test_largest_fft_length_at_pad_one(bst):
    """M = 4096 with pad factor 1 (N = 4096 rays), few angles."""
    rng = np.random.default_rng(4096)
    N, V = 4096, 24
    theta = synth.uniform_angles(V)
    sino = rng.standard_normal((1, V, N)).astype(np.float32)
    plan = bst.Plan(N, theta, 1)
    got = plan.fbp(_cuda(sino)).cpu().numpy()
    assert_parity(got[0], ob.fbp(sino[0].astype(np.float64), theta, 1), what="N=4096 pad 1")


def test_two_angles(bst):
    """The fewest angles a plan accepts: the seam brackets span half the circle."""
    rng = np.random.default_rng(2)
    N = 32
    theta = np.array([0.3, 1.9], dtype=np.float32)
    sino = rng.standard_normal((3, 2, N)).astype(np.float32)
    plan = bst.Plan(N, theta, 2)
    got = plan.fbp(_cuda(sino)).cpu().numpy()
    ref = np.stack([ob.fbp(s.astype(np.float64), theta) for s in sino])
    assert_parity(got, ref, what="two angles")
    plan.set_gridding("kaiser-bessel", 6)
    from oracle import kb
    got = plan.fbp(_cuda(sino)).cpu().numpy()
    ref = np.stack([kb.kb_fbp(s.astype(np.float64), theta) for s in sino])
    assert_parity(got, ref, what="two angles, KB")


def test_empty_batch_is_rejected(bst):
    from paper_1704_08364_gb300 import _lib
    L = _lib.load()
    plan = bst.Plan(64, synth.uniform_angles(64), 2)
    buf = torch.zeros(64 * 64, device="cuda")
    ws = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = ctypes.c_void_p(buf.data_ptr())
    assert L.bst_fbp(plan.handle, p, 0, None, ctypes.c_void_p(ws.data_ptr()), ctypes.c_void_p(ws.data_ptr()),
                     ws.numel(), st) == 1
    assert L.bst_workspace_bytes(plan.handle, 0) == 0
