"""Register and spill budget of the 2048^3 forward kernels, read from ptxas
(-Xptxas -v) at compile time; no GPU needed.  A regression guard: the packed
gridding kernel runs four 256-thread blocks per SM and the paired and
register-fed paired ones two 512-thread blocks (64 registers a thread in each
case), spilling at most a few
bytes; the FFT kernels spill nothing."""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NVCC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")


@pytest.fixture(scope="module")
def report(tmp_path_factory):
    nvcc = NVCC if os.path.exists(NVCC) else shutil.which("nvcc")
    if not nvcc:
        pytest.skip("nvcc not available")
    out = tmp_path_factory.mktemp("ptxas") / "k.o"
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-Xptxas", "-v",
                        "-I", os.path.join(ROOT, "paper_1704_08364_gb300", "csrc"),
                        "-I", os.path.join(ROOT, "include"),
                        "-c", os.path.join(ROOT, "tests", "kernel_resources.cu"), "-o", str(out)],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    txt = r.stdout + r.stderr
    res = {}
    # one block per kernel, from its "Compiling entry function" line to the next
    for block in txt.split("Compiling entry function")[1:]:
        for name in ("k_ray_fft", "k_grid_col", "k_grid_col_paired", "k_grid_col_xchg", "k_row_ifft"):
            if re.match(r"\s*'[^']*\d" + name + r"ILi4096", block):
                regs = re.search(r"Used (\d+) registers", block)
                spill = re.search(r"(\d+) bytes spill stores", block)
                assert regs and spill, block
                res[name] = (int(regs.group(1)), int(spill.group(1)))
    assert sorted(res) == ["k_grid_col", "k_grid_col_paired", "k_grid_col_xchg", "k_ray_fft", "k_row_ifft"], txt
    return res


def test_fft_kernels_do_not_spill(report):
    for name in ("k_ray_fft", "k_row_ifft"):
        regs, spill = report[name]
        assert spill == 0, f"{name} spills {spill} bytes"


def test_gridding_kernels_keep_their_blocks_per_sm(report):
    for name in ("k_grid_col", "k_grid_col_paired", "k_grid_col_xchg"):
        regs, spill = report[name]
        assert regs <= 64, f"{name} uses {regs} registers"
        assert spill <= 32, f"{name} spills {spill} bytes"


def test_paired_layout_slot_map_is_a_bijection(tmp_path):
    """The paired spectrum layout's slot map (paired_slot in bst_stages.cuh)
    covers the pair's workspace exactly once, with odd and even row counts."""
    nvcc = NVCC if os.path.exists(NVCC) else shutil.which("nvcc")
    if not nvcc:
        pytest.skip("nvcc not available")
    exe = tmp_path / "layout_check"
    r = subprocess.run([nvcc, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "paper_1704_08364_gb300", "csrc"),
                        "-I", os.path.join(ROOT, "include"), "-x", "cu", os.path.join(ROOT, "tests", "layout_check.cu"),
                        "-o", str(exe)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "OK", out.stdout + out.stderr


def test_twiddle_tables_tile_the_allocation_with_exact_values(tmp_path):
    """The per-pass twiddle tables that the ray kernel reads (bst_twiddle.h,
    pass_tab_base in bst_fft.cuh) cover the plan's twiddle allocation exactly
    once for every FFT length and both radix schedules, and hold
    exp(-2 pi i k s / (NS R)) to float rounding."""
    nvcc = NVCC if os.path.exists(NVCC) else shutil.which("nvcc")
    if not nvcc:
        pytest.skip("nvcc not available")
    exe = tmp_path / "twiddle_check"
    r = subprocess.run([nvcc, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "paper_1704_08364_gb300", "csrc"),
                        "-I", os.path.join(ROOT, "include"), "-x", "cu", os.path.join(ROOT, "tests", "twiddle_check.cu"),
                        "-o", str(exe)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "OK", out.stdout + out.stderr
