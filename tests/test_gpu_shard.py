"""Slice sharding on one GPU with virtual ranks: each rank runs the path on its
own contiguous range of whole slice pairs, one after another on the device.
Slices are independent (Sec. 1) and a range never splits a pair, so the
concatenated volume equals the unsharded one bit for bit; the filter-tap
gradient, summed over the ranks as the all-reduce would, equals the one of the
whole batch up to FP32 summation order."""
import numpy as np
import pytest

import synth
from paper_1704_08364_gb300.shard import slice_range

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bst():
    import paper_1704_08364_gb300 as m
    return m


def _sinos(S, V, N, seed):
    rng = np.random.default_rng(seed)
    th = synth.uniform_angles(V)
    host = np.stack([synth.gaussian_noise(synth.ellipse_sinogram(synth.random_ellipses(rng), th, N), rng)
                     for _ in range(S)])
    return th, torch.from_numpy(host.astype(np.float32)).cuda()


@pytest.mark.parametrize("world,S", [(2, 8), (3, 11), (4, 6)])
def test_virtual_ranks_forward_equals_unsharded(bst, world, S):
    N = V = 128
    th, sino = _sinos(S, V, N, 100 + world)
    plan = bst.Plan(N, th, 2)
    full = plan.fbp(sino)
    parts = []
    for r in range(world):
        a, b = slice_range(r, world, S)
        if b > a:
            parts.append(plan.fbp(sino[a:b].contiguous()))
    got = torch.cat(parts)
    assert got.shape == full.shape
    assert torch.equal(got, full)


def test_virtual_ranks_filter_gradient_sums_to_full_batch(bst):
    N = V = 64
    S, world = 6, 3
    th, sino = _sinos(S, V, N, 7)
    target = torch.randn(S, N, N, device="cuda", generator=torch.Generator("cuda").manual_seed(7))
    plan = bst.Plan(N, th, 2)

    def grad_g(p, f):
        g = torch.ones(N, device="cuda", requires_grad=True)
        ((bst.fbp_autograd(p, g, plan) - f) ** 2).sum().backward()
        return g.grad

    full = grad_g(sino, target)
    total = torch.zeros_like(full)
    for r in range(world):
        a, b = slice_range(r, world, S)
        total += grad_g(sino[a:b].contiguous(), target[a:b].contiguous())
    scale = full.abs().max().item()
    assert scale > 0
    np.testing.assert_allclose(total.cpu().numpy(), full.cpu().numpy(), rtol=0, atol=2e-5 * scale)


def test_device_generator_slices_equal_those_of_the_whole_volume():
    """bench.py --scaling strong generates each rank's slice range on its own
    device (first_slice): ellipses and noise must equal those slices of the
    whole volume generated at once, so every rank reconstructs its share of
    one workload."""
    from synth import device as sdev
    whole = sdev.ellipse_volume(2, 8, 64, 96, noise_frac=0.01, device="cuda")
    for s0, s1 in ((0, 4), (4, 8), (2, 6)):
        part = sdev.ellipse_volume(2, s1 - s0, 64, 96, noise_frac=0.01, device="cuda", first_slice=s0)
        assert torch.equal(part, whole[s0:s1]), (s0, s1)
