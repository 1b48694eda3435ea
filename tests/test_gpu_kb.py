"""GPU parity of Kaiser-Bessel gridding in P5 (bst_plan_set_gridding) against
the FP64 oracle (relative L2 <= 1e-5, max-abs <= 1e-4 max|ref|), through the
C-ABI; at 2048 sampled pixels against the direct polar sum."""
import numpy as np
import pytest

import synth
from oracle import bst as ob
from oracle import kb
from gpu_util import assert_parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bst():
    import paper_1704_08364_gb300 as m
    return m


def _run(bst, sino, theta, alpha=2, mode="fbp", g=None, width=6):
    plan = bst.Plan(sino.shape[-1], theta, alpha)
    plan.set_gridding("kaiser-bessel", width)
    assert plan.gridding == ("kaiser-bessel", width)
    d = torch.from_numpy(np.ascontiguousarray(sino, dtype=np.float32)).cuda()
    dg = None if g is None else torch.from_numpy(np.asarray(g, dtype=np.float32)).cuda()
    out = plan.fbp(d, dg) if mode == "fbp" else plan.backproject(d)
    plan.status()
    return out.cpu().numpy()


def _oracle(sino, theta, alpha=2, mode="fbp", g=None, width=6):
    m = ob.FILTER if mode == "fbp" else ob.BACKPROJECT
    gg = None if g is None else np.asarray(g, dtype=np.float32).astype(np.float64)
    return np.stack([kb.kb_fbp(s.astype(np.float64), theta, alpha, m, gg, width) for s in sino])


def _fov_mask(N, alpha):
    """Pixels compared.  At pad factor 1 the grid has no guard band and the
    deapodization multiplies the field-of-view edge by up to (C(0)/C(1/2))^2
    (~1.5e7 at W = 6), where float rounding of the gridded spectrum becomes an
    order-one error (the FP64 result there is dominated by aliasing anyway):
    there the comparison is on the inscribed disk |u| <= 0.8."""
    if alpha == 2:
        return np.ones((N, N), dtype=bool)
    b = np.arange(N) - N // 2
    return np.hypot(b[None, :], b[:, None]) <= 0.8 * N / 2


@pytest.mark.parametrize("N,V,alpha", [
    (8, 8, 2), (16, 12, 2), (32, 32, 1), (48, 40, 2), (64, 64, 2), (96, 70, 1), (128, 100, 2),
    (192, 128, 2), (256, 256, 1), (384, 300, 2), (512, 96, 2)])
def test_sizes_modes_and_odd_slices(bst, N, V, alpha):
    """Every FFT length family (2^a and 3 * 2^a, one to many strips per
    transform), both pad factors, odd slice counts, both modes."""
    rng = np.random.default_rng(N * 1000 + V + 7)
    theta = synth.uniform_angles(V)
    S = 3
    sino = np.stack([synth.ellipse_sinogram(synth.random_ellipses(rng), theta, N) for _ in range(S)])
    sino = synth.poisson_log_noise(sino, rng).astype(np.float32)
    m = _fov_mask(N, alpha)
    for mode in ("fbp", "bp"):
        got = _run(bst, sino, theta, alpha, mode)
        ref = _oracle(sino, theta, alpha, mode)
        assert_parity(got[:, m], ref[:, m], what=f"KB N={N} V={V} a={alpha} {mode}")


@pytest.mark.parametrize("width", [2, 4, 8])
def test_kernel_widths(bst, width):
    rng = np.random.default_rng(width)
    N, V = 128, 128
    theta = synth.uniform_angles(V)
    sino = np.stack([synth.ellipse_sinogram(synth.random_ellipses(rng), theta, N) for _ in range(2)])
    got = _run(bst, sino.astype(np.float32), theta, 2, "fbp", None, width)
    assert_parity(got, _oracle(sino.astype(np.float32), theta, 2, "fbp", None, width), what=f"KB W={width}")


def test_nonuniform_angles_and_filter_taps(bst):
    rng = np.random.default_rng(5)
    N, V = 256, 180
    theta = np.sort(rng.uniform(0.0, np.pi, V)).astype(np.float32)
    theta[0] = 0.0
    g = rng.uniform(0.3, 1.4, N).astype(np.float32)
    sino = rng.standard_normal((2, V, N)).astype(np.float32)
    got = _run(bst, sino, theta, 2, "fbp", g)
    assert_parity(got, _oracle(sino, theta, 2, "fbp", g), what="KB nonuniform + taps")


def test_prep_stages_with_kb(bst):
    """bst_fbp_prep on a KB plan: normalization, centering and window in the ray
    stage, KB gridding in P5."""
    from oracle import prep
    N, V, S = 128, 96, 2
    rng = np.random.default_rng(23)
    theta = synth.uniform_angles(V)
    y = np.stack([synth.ellipse_sinogram(synth.random_ellipses(rng, fov_safe=True), theta, N) for _ in range(S)])
    flat = rng.uniform(9000, 11000, (S, N))
    dark = rng.uniform(50, 150, (S, N))
    counts = (flat[:, None, :] - dark[:, None, :]) * np.exp(-y) + dark[:, None, :]
    plan = bst.Plan(N, theta, 2)
    plan.set_gridding("kaiser-bessel", 6)
    f32 = lambda a: torch.from_numpy(np.asarray(a, dtype=np.float32)).cuda()
    got = plan.fbp_prep(f32(counts), flat=f32(flat), dark=f32(dark), shift=2.37, kb_beta=3.0,
                        kb_halfwidth=0.95).cpu().numpy()
    for s in range(S):
        ref = prep.prepared_fbp(counts[s].astype(np.float32).astype(np.float64), theta,
                                flat=flat[s].astype(np.float32).astype(np.float64),
                                dark=dark[s].astype(np.float32).astype(np.float64), shift=2.37, kb_beta=3.0,
                                kb_half=0.95, grid_width=6)
        assert_parity(got[s], ref, what=f"KB prep slice {s}")


def test_switching_back_to_bilinear(bst):
    rng = np.random.default_rng(9)
    N = V = 64
    theta = synth.uniform_angles(V)
    sino = torch.from_numpy(rng.standard_normal((2, V, N)).astype(np.float32)).cuda()
    plan = bst.Plan(N, theta, 2)
    plan.set_gridding("kaiser-bessel", 6)
    a = plan.fbp(sino).cpu().numpy()
    plan.set_gridding("bilinear")
    assert plan.gridding == ("bilinear", 2)
    b = plan.fbp(sino).cpu().numpy()
    assert_parity(b, np.stack([ob.fbp(s.astype(np.float64), theta) for s in sino.cpu().numpy()]), what="bilinear")
    assert not np.allclose(a, b)


def test_kb_plan_rejected_by_the_adjoint(bst):
    plan = bst.Plan(32, synth.uniform_angles(32), 2)
    plan.set_gridding("kaiser-bessel", 6)
    with pytest.raises(bst.BstError):
        plan.radon_adjoint(torch.zeros((2, 32, 32), device="cuda"))


def test_volume_2048_sampled_pixels_against_the_direct_sum(bst):
    """The 2048^3 workload with KB gridding in the benchmark's launch
    configuration: sampled slices regenerated on the host, sampled pixels
    against the direct polar sum that the gridding approximates (its error at
    W = 6 and pad factor 2 is ~2e-6 of the image scale), and one whole slice
    against the KB oracle at the parity bar."""
    free, _ = torch.cuda.mem_get_info()
    if free < 72 * 2**30:
        pytest.skip("needs ~70 GiB of free device memory")
    idx = [0, 2047]
    theta, sub, _ = synth.workload_slices("volume-2048", idx)
    plan = bst.Plan(2048, theta, 2)
    plan.set_gridding("kaiser-bessel", 6)
    d = torch.zeros((2048, 2048, 2048), dtype=torch.float32, device="cuda")
    d[idx] = torch.from_numpy(sub).cuda()
    out = plan.fbp(d)
    plan.status()
    got = out[idx].cpu().numpy()
    del d, out
    rng = np.random.default_rng(0)
    rows = np.concatenate(([1024, 0, 2047, 1024, 3], rng.integers(0, 2048, 11)))
    cols = np.concatenate(([1024, 0, 2047, 5, 1024], rng.integers(0, 2048, 11)))
    for n, s in enumerate(idx):
        ref = kb.direct_sum(sub[n].astype(np.float64), theta, 2, pixels=(rows, cols))
        scale = float(np.abs(got[n]).max())
        err = np.abs(got[n][rows, cols] - ref).max()
        assert err <= 2e-5 * scale, f"slice {s}: max err {err:.3e} vs scale {scale:.3e}"
    # the oracle the kernel implements, on one whole slice, at the path's parity bar
    assert_parity(got[0], kb.kb_fbp(sub[0].astype(np.float64), theta), what="KB 2048 slice 0 vs kb_fbp")


def test_host_pipeline_and_noalloc_on_a_kb_plan(bst):
    """bst_fbp_host and bst_fbp_noalloc run the plan's KB gridding too."""
    rng = np.random.default_rng(31)
    N = V = 512
    theta = synth.uniform_angles(V)
    sino = np.stack([synth.ellipse_sinogram(synth.random_ellipses(rng), theta, N) for _ in range(3)]).astype(np.float32)
    plan = bst.Plan(N, theta, 2)
    plan.set_gridding("kaiser-bessel", 6)
    ref = _oracle(sino, theta)
    h = torch.from_numpy(sino).pin_memory()
    assert_parity(plan.fbp_host(h).numpy(), ref, what="KB host pipeline")
    assert_parity(plan.fbp_noalloc(torch.from_numpy(sino).cuda()).cpu().numpy(), ref, what="KB noalloc")
