"""Every launch shape of the forward path gives the oracle's result: radix
schedule 16 or 8, packed or paired spectrum layout (the paired gather through
shared memory or into registers), chunks of one to three
slice pairs in column- or pair-fastest block order, one or two lanes
(bst_plan_set_forward_config), and the shape the autotuner picks.  The
shapes change how the stages of Sec. 2 are tiled, never what they compute."""
import itertools

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


SHAPES = [dict(max_radix=r, layout=l, chunk_pairs=c, pair_fast=f, max_lanes=n, grid_xchg=x)
          for r, (l, x), (c, f), n in itertools.product((16, 8), (("packed", 0), ("paired", 0), ("paired", 1)),
                                                         ((1, 0), (2, 0), (2, 1), (3, 1)), (2, 1))]


def _oracle(sino, theta, alpha, mode):
    m = ob.FILTER if mode == "fbp" else ob.BACKPROJECT
    return np.stack([ob.bst(s.astype(np.float64), theta, alpha, m) for s in sino])


@pytest.mark.parametrize("N,V,alpha", [(8, 8, 2), (24, 21, 2), (32, 32, 1), (48, 40, 2), (64, 37, 1), (96, 70, 1),
                                       (128, 100, 2), (192, 127, 2), (256, 256, 1), (384, 300, 2),
                                       (512, 96, 2)])
def test_every_launch_shape_matches_the_oracle(bst, N, V, alpha):
    """Both FFT-length families (2^a, 3 * 2^a), both pad factors, odd and even
    angle counts (the paired layout stores rows two by two; an odd last row
    whole), 7 slices (an odd count: the last pair is padded; chunks that do not
    divide the pairs)."""
    rng = np.random.default_rng(7 * N + V)
    theta = synth.uniform_angles(V)
    S = 7
    sino = np.stack([synth.ellipse_sinogram(synth.random_ellipses(rng), theta, N) for _ in range(S)])
    sino = synth.poisson_log_noise(sino, rng).astype(np.float32)
    d = torch.from_numpy(sino).cuda()
    plan = bst.Plan(N, theta, alpha)
    refs = {m: _oracle(sino, theta, alpha, m) for m in ("fbp", "bp")}
    for shape in SHAPES:
        plan.set_forward_config(**shape)
        assert plan.forward_config == shape
        for mode in ("fbp", "bp"):
            got = (plan.fbp(d) if mode == "fbp" else plan.backproject(d)).cpu().numpy()
            plan.status()
            assert_parity(got, refs[mode], what=f"N={N} V={V} a={alpha} {mode} {shape}")


@pytest.mark.parametrize("grid_xchg", [0, 1])
def test_paired_layout_at_2048_with_nonuniform_angles(bst, grid_xchg):
    """The paired layout's seam rows and radial taps at M = 4096: sorted random
    angles (first angle above 0, so the bracket below theta_0 is used), one
    slice pair, the gather through shared memory or into registers."""
    rng = np.random.default_rng(4096)
    N = V = 2048
    theta = np.sort(np.unique(rng.uniform(0.01, np.pi - 0.003, V + 16).astype(np.float32))[:V])
    sino = np.stack([synth.gaussian_noise(synth.ellipse_sinogram(synth.random_ellipses(rng), theta, N), rng)
                     for _ in range(2)]).astype(np.float32)
    plan = bst.Plan(N, theta, 2)
    plan.set_forward_config(layout="paired", chunk_pairs=2, pair_fast=1, grid_xchg=grid_xchg)
    d = torch.from_numpy(sino).cuda()
    got = plan.fbp(d).cpu().numpy()
    for s in range(2):
        assert_parity(got[s], ob.fbp(sino[s].astype(np.float64), theta),
                      what=f"paired 2048 slice {s} grid_xchg {grid_xchg}")


@pytest.mark.parametrize("grid_xchg", [0, 1])
def test_paired_layout_with_prep_stages_and_filter_taps(bst, grid_xchg):
    """bst_fbp_prep (normalization, centering, window) and learnable taps on
    the paired layout, the gather through shared memory or into registers."""
    from oracle import prep
    N, V, S = 128, 96, 3
    rng = np.random.default_rng(19)
    theta = synth.uniform_angles(V)
    y = np.stack([synth.ellipse_sinogram(synth.random_ellipses(rng, fov_safe=True), theta, N) for _ in range(S)])
    flat = rng.uniform(9000, 11000, (S, N))
    counts = flat[:, None, :] * np.exp(-y)
    g = rng.uniform(0.3, 1.4, 2 * N // 2).astype(np.float32)
    plan = bst.Plan(N, theta, 2)
    plan.set_forward_config(layout="paired", chunk_pairs=2, pair_fast=1, grid_xchg=grid_xchg)
    f = lambda a: torch.from_numpy(np.asarray(a, dtype=np.float32)).cuda()
    got = plan.fbp_prep(f(counts), flat=f(flat), shift=-2.3, kb_beta=3.0, kb_halfwidth=0.95, g=f(g)).cpu().numpy()
    for s in range(S):
        ref = prep.prepared_fbp(counts[s].astype(np.float32).astype(np.float64), theta,
                                flat=np.asarray(flat[s], dtype=np.float32).astype(np.float64), shift=-2.3,
                                kb_beta=3.0, kb_half=0.95, g=g.astype(np.float64))
        assert_parity(got[s], ref, what=f"paired prep slice {s}")


def test_autotuned_shape_matches_the_oracle_and_is_kept(bst, tmp_path):
    N = V = 256
    rng = np.random.default_rng(3)
    theta = synth.uniform_angles(V)
    sino = rng.standard_normal((4, V, N)).astype(np.float32)
    plan = bst.Plan(N, theta, 2)
    cache = str(tmp_path / "tune.json")
    cfg = plan.autotune(cache=cache)
    assert cfg == plan.forward_config and cfg["max_radix"] in (8, 16)
    got = plan.fbp(torch.from_numpy(sino).cuda()).cpu().numpy()
    assert_parity(got, _oracle(sino, theta, 2, "fbp"), what=f"autotuned {cfg}")
    other = bst.Plan(N, theta, 2)
    assert other.autotune(cache=cache) == cfg      # read back from the cache, not re-timed


def test_invalid_shapes_are_rejected_and_change_nothing(bst):
    plan = bst.Plan(64, synth.uniform_angles(64), 2)
    before = plan.forward_config
    for bad in (dict(max_radix=4), dict(layout=7), dict(chunk_pairs=0), dict(chunk_pairs=257),
                dict(pair_fast=2), dict(max_lanes=0), dict(max_lanes=3), dict(grid_xchg=2)):
        with pytest.raises(bst.BstError):
            plan.set_forward_config(**bad)
        assert plan.forward_config == before


def test_kb_plan_ignores_the_paired_layout(bst):
    """Kaiser-Bessel gridding reads the packed spectrum whatever the layout field says."""
    from oracle import kb
    rng = np.random.default_rng(23)
    N = V = 64
    theta = synth.uniform_angles(V)
    sino = rng.standard_normal((3, V, N)).astype(np.float32)
    plan = bst.Plan(N, theta, 2).set_gridding("kaiser-bessel", 6)
    plan.set_forward_config(layout="paired")
    got = plan.fbp(torch.from_numpy(sino).cuda()).cpu().numpy()
    assert_parity(got, np.stack([kb.kb_fbp(s.astype(np.float64), theta) for s in sino]), what="KB + paired field")
