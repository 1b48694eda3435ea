"""The ragged batch (one persistent launch over sinograms of mixed sizes, with
and without CUDA-graph replay), its bounded dependency waits, and the radix
schedules the autotuner chooses between."""
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
    return m


def _batch(sizes, seed=0):
    rng = np.random.default_rng(seed)
    sinos = []
    for N in sizes:
        th = synth.uniform_angles(N)
        y = synth.ellipse_sinogram(synth.random_ellipses(rng), th, N)
        sinos.append(synth.poisson_log_noise(y, rng).astype(np.float32))
    return sinos


SIZES = [256, 128, 512, 384, 256, 768, 128, 1024, 512, 256, 384, 2048]


@pytest.mark.parametrize("order", [0, 2])
def test_ragged_matches_per_item_path(bst, order):
    """Both queue orders: phases (0) and neighbouring pair-items overlapping (2)."""
    plans = {N: bst.Plan(N, synth.uniform_angles(N), 2) for N in sorted(set(SIZES))}
    host = _batch(SIZES)
    sinos = [torch.from_numpy(h).cuda() for h in host]
    vols = [torch.full((N, N), float("nan"), device="cuda") for N in SIZES]
    rb = bst.RaggedBatch([plans[N] for N in SIZES]).bind(sinos, vols, flags=order)
    assert rb.pair_items == 8   # 256 x3 -> 2, 128 x2 -> 1, 512 x2, 384 x2, 768, 1024, 2048
    refs = [plans[N].fbp(s.unsqueeze(0))[0].cpu().numpy() for N, s in zip(SIZES, sinos)]
    for use_graph in (False, True, True):
        for v in vols:
            v.fill_(float("nan"))
        rb.run(use_graph)
        assert rb.status() == 0
        for i, (v, r) in enumerate(zip(vols, refs)):
            assert_parity(v.cpu().numpy(), r, what=f"ragged item {i} (N={SIZES[i]}, graph={use_graph})")
    for i in (1, 3):   # small items also against the oracle directly
        th = synth.uniform_angles(SIZES[i])
        assert_parity(vols[i].cpu().numpy(), ob.fbp(host[i].astype(np.float64), th), what=f"ragged oracle {i}")


def test_dependency_wait_times_out_and_context_survives(bst):
    """A unit whose dependency is never produced (the diagnostic flag leaves the
    first pair-item's ray stage unqueued) waits at most the spin limit, the
    launch ends with BST_ERR_TIMEOUT, and the next launch works."""
    sizes = [256, 256, 512]
    plans = {N: bst.Plan(N, synth.uniform_angles(N), 2) for N in set(sizes)}
    sinos = [torch.from_numpy(h).cuda() for h in _batch(sizes, 3)]
    vols = [torch.zeros((N, N), device="cuda") for N in sizes]
    rb = bst.RaggedBatch([plans[N] for N in sizes])
    rb.set_spin_limit(2000)
    rb.bind(sinos, vols, flags=1)
    rb.run()
    assert rb.status() == 5   # BST_ERR_TIMEOUT
    rb.bind(sinos, vols, flags=0)
    rb.run()
    assert rb.status() == 0
    for N, s, v in zip(sizes, sinos, vols):
        assert_parity(v.cpu().numpy(), plans[N].fbp(s.unsqueeze(0))[0].cpu().numpy(), what="after timeout")


@pytest.mark.parametrize("N", [192, 512, 1536])
def test_both_radix_schedules_match_the_oracle(bst, N):
    theta, sino, _ = synth.workload_slices("volume-512", [0, 1], rays=N, angles=N)
    plan = bst.Plan(N, theta, 2)
    ref = np.stack([ob.fbp(s.astype(np.float64), theta) for s in sino])
    for sched in (16, 8):
        plan.schedule = sched
        got = plan.fbp(torch.from_numpy(sino).cuda()).cpu().numpy()
        assert_parity(got, ref, what=f"schedule {sched} N={N}")
    chosen = plan.autotune(slices=8)
    assert chosen["max_radix"] in (8, 16) and plan.schedule == chosen["max_radix"]
    assert chosen == plan.forward_config
