"""GPU parity of brute_backproject (slant stack, Eq. 2) and of the filtered
slant stack against the FP64 oracle."""
import numpy as np
import pytest

import synth
from oracle import brute
from gpu_util import assert_parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bst():
    import paper_1704_08364_gb300 as m
    return m


@pytest.mark.parametrize("N,V,S", [(16, 12, 1), (64, 50, 3), (96, 64, 9), (256, 256, 2)])
def test_plain_slant_stack(bst, N, V, S):
    rng = np.random.default_rng(N + V)
    theta = synth.uniform_angles(V)
    sino = rng.standard_normal((S, V, N)).astype(np.float32)
    plan = bst.Plan(N, theta, 2)
    got = plan.brute_backproject(torch.from_numpy(sino).cuda()).cpu().numpy()
    plan.status()
    ref = np.stack([brute.backproject(s.astype(np.float64), theta) for s in sino])
    assert_parity(got, ref, what=f"brute N={N}")


def test_nonuniform_angles(bst):
    rng = np.random.default_rng(3)
    theta = np.sort(rng.uniform(0.0, np.pi - 0.01, 33)).astype(np.float32)
    sino = rng.standard_normal((2, 33, 48)).astype(np.float32)
    plan = bst.Plan(48, theta, 2)
    got = plan.brute_backproject(torch.from_numpy(sino).cuda()).cpu().numpy()
    ref = np.stack([brute.backproject(s.astype(np.float64), theta) for s in sino])
    assert_parity(got, ref, what="brute nonuniform")


@pytest.mark.parametrize("alpha", [1, 2])
def test_filtered_slant_stack(bst, alpha):
    theta, sino, _ = synth.workload_slices("single-256", [0], rays=128, angles=96)
    g = np.random.default_rng(1).uniform(0.5, 1.5, alpha * 64).astype(np.float32)
    plan = bst.Plan(128, theta, alpha)
    got = plan.brute_backproject(torch.from_numpy(sino).cuda(), torch.from_numpy(g).cuda()).cpu().numpy()
    ref = brute.ss_fbp(sino[0].astype(np.float64), theta, alpha, g.astype(np.float64))
    assert_parity(got[0], ref, what="ss-fbp")


def test_sampled_pixels_at_2048(bst):
    """Full-size geometry (N = V = 2048), a few slices: sampled pixels against
    the oracle evaluated one by one."""
    theta, sino, _ = synth.workload_slices("volume-2048", [5, 6])
    plan = bst.Plan(2048, theta, 2)
    got = plan.brute_backproject(torch.from_numpy(sino).cuda()).cpu().numpy()
    rng = np.random.default_rng(0)
    rows = rng.integers(0, 2048, 64)
    cols = rng.integers(0, 2048, 64)
    for n in range(2):
        ref = brute.backproject_pixels(sino[n].astype(np.float64), theta, rows, cols)
        assert_parity(got[n][rows, cols], ref, what="brute 2048 sampled")
