"""GPU parity of radon_adjoint (the transpose of the BST operator) and of the
filter-tap gradient against the FP64 oracle; FP32 adjoint identities on the
GPU; the autograd function against the oracle gradients."""
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


@pytest.mark.parametrize("N,V,alpha", [(16, 12, 2), (32, 40, 2), (64, 48, 1), (96, 64, 2), (128, 128, 2)])
@pytest.mark.parametrize("mode", ["ramp", "taps", "bp"])
def test_adjoint_matches_oracle(bst, N, V, alpha, mode):
    rng = np.random.default_rng(N + V + alpha)
    theta = synth.uniform_angles(V) if N != 96 else np.sort(rng.uniform(0.05, 3.1, V)).astype(np.float32)
    f = rng.standard_normal((3, N, N)).astype(np.float32)
    g = None if mode != "taps" else rng.uniform(0.3, 1.5, alpha * N // 2).astype(np.float32)
    plan = bst.Plan(N, theta, alpha)
    m = bst.BACKPROJECT if mode == "bp" else bst.FILTER
    got = plan.radon_adjoint(_cuda(f), m, None if g is None else _cuda(g)).cpu().numpy()
    plan.status()
    om = ob.BACKPROJECT if mode == "bp" else ob.FILTER
    gg = None if g is None else g.astype(np.float64)
    ref = np.stack([oa.bst_adjoint(x.astype(np.float64), theta, alpha, om, gg) for x in f])
    assert_parity(got, ref, what=f"adjoint N={N} V={V} {mode}")


def test_adjoint_identity_in_fp32(bst):
    """<A p, f> = <p, A^T f> with both sides computed on the GPU."""
    rng = np.random.default_rng(7)
    N, V = 256, 200
    theta = synth.uniform_angles(V)
    plan = bst.Plan(N, theta, 2)
    p = _cuda(rng.standard_normal((2, V, N)))
    f = _cuda(rng.standard_normal((2, N, N)))
    lhs = float((plan.fbp(p).double() * f.double()).sum())
    rhs = float((p.double() * plan.radon_adjoint(f).double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * float(p.double().norm() * f.double().norm()) ** 0.5 * abs(lhs) ** 0.5 + 1e-5 * abs(lhs)


def test_filter_gradient_matches_oracle(bst):
    rng = np.random.default_rng(8)
    N, V = 64, 64
    theta = synth.uniform_angles(V)
    p = rng.standard_normal((3, V, N)).astype(np.float32)
    R = rng.standard_normal((3, N, N)).astype(np.float32)
    plan = bst.Plan(N, theta, 2)
    got = plan.filter_grad(_cuda(p), _cuda(R)).cpu().numpy()
    ref = sum(oa.filter_grad(p[s].astype(np.float64), R[s].astype(np.float64), theta) for s in range(3))
    assert_parity(got, ref, what="filter grad")


def test_autograd_function(bst):
    """Loss ||FBP(p; g) - f||^2 on the autograd workload's geometry (reduced
    to 128 rays): gradients for p and g against the FP64 oracle."""
    N = V = 128
    theta, p, imgs = synth.workload_slices("autograd-1024", [0, 1], rays=N, angles=V, with_images=True)
    plan = bst.Plan(N, theta, 2)
    dp = _cuda(p).requires_grad_(True)
    g = torch.ones(N, device="cuda", requires_grad=True)
    f = _cuda(imgs)
    x = bst.fbp_autograd(dp, g, plan)
    loss = ((x - f) ** 2).sum()
    loss.backward()
    xr = np.stack([ob.fbp(s.astype(np.float64), theta) for s in p])
    R = 2.0 * (xr - imgs)
    gp_ref = np.stack([oa.bst_adjoint(R[s], theta) for s in range(2)])
    gg_ref = sum(oa.filter_grad(p[s].astype(np.float64), R[s], theta) for s in range(2))
    assert_parity(dp.grad.cpu().numpy(), gp_ref, what="grad p")
    assert_parity(g.grad.cpu().numpy(), gg_ref, what="grad g")


def test_backward_equals_the_two_separate_calls(bst):
    """bst_fbp_backward (one pull-back for both gradients) gives what
    radon_adjoint and bst_fbp_filter_grad give separately, with either output
    alone too; odd slice count, random taps."""
    rng = np.random.default_rng(12)
    N, V, S = 128, 96, 3
    theta = synth.uniform_angles(V)
    plan = bst.Plan(N, theta, 2)
    p = _cuda(rng.standard_normal((S, V, N)))
    R = _cuda(rng.standard_normal((S, N, N)))
    g = _cuda(rng.uniform(0.5, 1.5, N))
    gp, gg = plan.fbp_backward(p, R, g)
    ref_p = plan.radon_adjoint(R, bst.FILTER, g)
    ref_g = plan.filter_grad(p, R)
    assert_parity(gp.cpu().numpy(), ref_p.cpu().numpy(), rtol_l2=1e-7, atol_frac=1e-6, what="backward grad p")
    assert_parity(gg.cpu().numpy(), ref_g.cpu().numpy(), rtol_l2=1e-7, atol_frac=1e-6, what="backward grad g")
    only_p, none_g = plan.fbp_backward(p, R, g, want_g=False)
    none_p, only_g = plan.fbp_backward(p, R, g, want_sino=False)
    assert none_g is None and none_p is None
    assert_parity(only_p.cpu().numpy(), ref_p.cpu().numpy(), rtol_l2=1e-7, atol_frac=1e-6, what="grad p alone")
    assert_parity(only_g.cpu().numpy(), ref_g.cpu().numpy(), rtol_l2=1e-7, atol_frac=1e-6, what="grad g alone")
