"""bst_fbp_noalloc: the filtered backprojection for callers that cannot
allocate device memory where they reconstruct (an external memory manager
owns the device's memory, or a cudaMalloc/cudaFree, which may synchronise
the device, is not acceptable in their loop).  Its scratch is a fixed device
array inside the library, so its results must equal those of bst_fbp (which
takes a caller workspace) call after call, with nothing left over from the
previous call.

This file is collected last on purpose: a run that stops at the first
failure has then already run every other test."""
import ctypes

import numpy as np
import pytest

import synth
from gpu_util import assert_parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _noalloc(lib, plan, sino, out):
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.bst_fbp_noalloc(plan.handle, ctypes.c_void_p(sino.data_ptr()), sino.shape[0], None,
                               ctypes.c_void_p(out.data_ptr()), st)


@pytest.mark.parametrize("N,S", [(256, 5), (512, 4)])
def test_noalloc_matches_fbp_on_two_calls_in_a_row(N, S):
    import paper_1704_08364_gb300 as bst
    from paper_1704_08364_gb300 import _lib
    lib = _lib.load()
    assert lib.bst_noalloc_scratch_bytes() == 8 << 20
    theta = synth.uniform_angles(N)
    plan = bst.Plan(N, theta, 2)
    for call in range(2):   # different inputs each call: no state may carry over
        rng = np.random.default_rng(100 * N + call)
        sino = np.stack([synth.ellipse_sinogram(synth.random_ellipses(rng), theta, N) for _ in range(S)])
        sino = torch.from_numpy(synth.poisson_log_noise(sino, rng).astype(np.float32)).cuda()
        ref = plan.fbp(sino)
        out = torch.full((S, N, N), float("nan"), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        free_before, _ = torch.cuda.mem_get_info()
        assert _noalloc(lib, plan, sino, out) == 0
        plan.status()
        free_after, _ = torch.cuda.mem_get_info()
        # the call itself takes no device memory (its scratch was placed when
        # the plan was created); the driver's free count is exact on a device
        # this process uses alone
        assert free_after == free_before, f"free device memory fell by {free_before - free_after} bytes"
        assert_parity(out.cpu().numpy(), ref.cpu().numpy(), what=f"noalloc N={N} call {call}")


def test_noalloc_rejects_plans_beyond_the_scratch():
    import paper_1704_08364_gb300 as bst
    from paper_1704_08364_gb300 import _lib
    lib = _lib.load()
    N = 1024   # one pair needs (1024 * 2048 + 1024 * 2048) * 8 bytes = 32 MiB > 8 MiB
    plan = bst.Plan(N, synth.uniform_angles(N), 2)
    sino = torch.zeros((2, N, N), dtype=torch.float32, device="cuda")
    out = torch.zeros((2, N, N), dtype=torch.float32, device="cuda")
    assert _noalloc(lib, plan, sino, out) == 3   # BST_ERR_WORKSPACE_TOO_SMALL
    assert float(out.abs().max()) == 0.0
