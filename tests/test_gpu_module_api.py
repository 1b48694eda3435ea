"""The module-level calls on the GPU: the same volumes as the plan methods
(bit for bit, one path) and, for the ragged call, the oracle's."""
import numpy as np
import pytest

import synth
from oracle import bst as ob
from gpu_util import assert_parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bst():
    import paper_1704_08364_gb300 as m
    yield m
    m.clear_plans()


def _sino(S, V, N, seed):
    rng = np.random.default_rng(seed)
    th = synth.uniform_angles(V)
    host = np.stack([synth.ellipse_sinogram(synth.random_ellipses(rng), th, N) for _ in range(S)])
    return th, host.astype(np.float32)


def test_module_calls_equal_the_plan_methods(bst):
    th, host = _sino(3, 48, 64, 11)
    sino = torch.from_numpy(host).cuda()
    plan = bst.Plan(64, th, 2)
    assert torch.equal(bst.fbp(sino, th), plan.fbp(sino))
    assert torch.equal(bst.backproject(sino, th), plan.backproject(sino))
    vol = plan.fbp(sino)
    assert torch.equal(bst.radon_adjoint(vol, th), plan.radon_adjoint(vol))
    assert torch.equal(bst.brute_backproject(sino, th), plan.brute_backproject(sino))
    assert bst.plan_for(64, th, 2) is bst.plan_for(64, th, 2)


def test_fbp_ragged_matches_the_oracle(bst):
    items = [(128, 96, 1), (256, 128, 2), (128, 96, 3)]   # M = 256 and 512: ragged lengths
    host = []
    for N, V, seed in items:
        th, h = _sino(1, V, N, seed)
        host.append((th, h[0]))
    vols = bst.fbp_ragged([torch.from_numpy(h).cuda() for _, h in host], angles=[th for th, _ in host])
    for (th, h), v in zip(host, vols):
        assert_parity(v.cpu().numpy(), ob.fbp(h.astype(np.float64), th), what=f"ragged item N={h.shape[1]}")
