"""The multi-rank path on CPU: slice sharding (whole pairs, full cover) and the
filter-gradient sum over world_size-2 gloo ranks, against one process."""
import os
import socket

import numpy as np
import pytest

from paper_1704_08364_gb300.shard import slice_range


@pytest.mark.parametrize("world,slices", [(1, 7), (2, 8), (2, 7), (3, 10), (4, 3), (8, 2048)])
def test_slice_ranges_cover_all_slices_in_pairs(world, slices):
    got = [slice_range(r, world, slices) for r in range(world)]
    assert got[0][0] == 0 and got[-1][1] == slices
    for (a0, a1), (b0, b1) in zip(got, got[1:]):
        assert a1 == b0
    for a0, a1 in got:
        assert (a0 % 2 == 0 or a0 == a1 == slices) and (a1 % 2 == 0 or a1 == slices)
    sizes = [a1 - a0 for a0, a1 in got]
    assert max(sizes) - min(sizes) <= 2


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist

    import synth
    from oracle import adjoint as oa
    from paper_1704_08364_gb300.shard import allreduce_filter_grad, slice_range

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    N = V = 16
    S = 6
    theta = synth.uniform_angles(V)
    rng = np.random.default_rng(0)
    p = rng.standard_normal((S, V, N))
    R = rng.standard_normal((S, N, N))
    a, b = slice_range(rank, world, S)
    g = sum((oa.filter_grad(p[s], R[s], theta) for s in range(a, b)), np.zeros(N))
    t = torch.from_numpy(g)
    allreduce_filter_grad(t)
    np.save(os.path.join(out_dir, f"g{rank}.npy"), t.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_filter_gradient_allreduce_over_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp

    import synth
    from oracle import adjoint as oa

    mp.spawn(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    N = V = 16
    theta = synth.uniform_angles(V)
    rng = np.random.default_rng(0)
    p = rng.standard_normal((6, V, N))
    R = rng.standard_normal((6, N, N))
    ref = sum(oa.filter_grad(p[s], R[s], theta) for s in range(6))
    for r in range(2):
        np.testing.assert_allclose(np.load(tmp_path / f"g{r}.npy"), ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_bench_strong_scaling_ranges_cover_one_volume_in_whole_pairs(world):
    """bench.py --scaling strong: the ranks' slice ranges of one 2048-slice
    volume tile it exactly, each starting on a pair boundary; weak scaling
    gives every rank the whole volume."""
    import argparse
    import bench
    args = argparse.Namespace(scaling="strong", slices=2048)
    got = [bench.rank_slices(args, r, world) for r in range(world)]
    assert got[0][0] == 0 and got[-1][1] == 2048
    assert all(a1 == b0 for (_, a1), (b0, _) in zip(got, got[1:]))
    assert all(a0 % 2 == 0 and (a1 - a0) % 2 == 0 for a0, a1 in got)
    assert sum(a1 - a0 for a0, a1 in got) == 2048
    weak = argparse.Namespace(scaling="weak", slices=2048)
    assert all(bench.rank_slices(weak, r, world) == (0, 2048) for r in range(world))
