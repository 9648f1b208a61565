"""Slice sharding on CPU: the split of P slices over ranks, and two gloo ranks (127.0.0.1) whose
per-rank sliced sums over their own slices (the oracle standing in for each rank's GPU) combine,
through one all-reduce, into the sliced sum over all P slices (Algorithm 1: s is the average of
independent per-slice sums, so the weighted average of the ranks' averages is exact)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle  # noqa: E402
from paper_2401_08260_gb300 import workloads  # noqa: E402
from paper_2401_08260_gb300.shard import SliceShard, slice_range  # noqa: E402

# (kernel, param, d, N, M, P): an uneven split, and P < world (rank 1 owns no slice)
CASES = [("gaussian", 2.0, 5, 300, 200, 7), ("negdist", 0.0, 4, 250, 150, 1), ("laplacian", 0.5, 3, 200, 120, 6)]


def _inputs(d, N, M, P, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.standard_normal((N, d))
    y = rng.standard_normal((M, d)) * 0.8
    w = rng.uniform(0.0, 1.0, N)
    return x, y, w, workloads.directions(P, d, seed=seed + 1)


def test_slice_range_partitions():
    for P in range(1, 41):
        for parts in range(1, 10):
            ranges = [slice_range(P, parts, i) for i in range(parts)]
            assert ranges[0][0] == 0 and ranges[-1][1] == P
            for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
                assert a1 == b0
            sizes = [p1 - p0 for p0, p1 in ranges]
            assert min(sizes) >= 0 and max(sizes) - min(sizes) <= 1
            assert sum(sizes) == P
    with pytest.raises(ValueError):
        slice_range(0, 2, 0)
    with pytest.raises(ValueError):
        slice_range(4, 2, 2)


def test_single_rank_owns_every_slice():
    sh = SliceShard(9, rank=0, world=1)
    assert (sh.p0, sh.p1, sh.weight) == (0, 9, 1.0)
    t = torch.arange(4, dtype=torch.float64)
    assert torch.equal(sh.combine(t), t)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        for i, (kernel, param, d, N, M, P) in enumerate(CASES):
            x, y, w, xi = _inputs(d, N, M, P, seed=70 + i)
            sh = SliceShard(P)  # rank and world from the process group
            if sh.count:
                s_loc, g_loc, _ = oracle.sliced_sum(kernel, param, x, y, w, xi[sh.p0:sh.p1], grad=True)
            else:
                s_loc, g_loc = np.zeros(M), np.zeros((M, d))
            s = sh.combine(torch.from_numpy(s_loc)).numpy()
            g = sh.combine(torch.from_numpy(g_loc)).numpy()
            out[(rank, i)] = (sh.p0, sh.p1, s, g)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_combine_to_the_full_sliced_sum():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    for i, (kernel, param, d, N, M, P) in enumerate(CASES):
        x, y, w, xi = _inputs(d, N, M, P, seed=70 + i)
        s_ref, g_ref, _ = oracle.sliced_sum(kernel, param, x, y, w, xi, grad=True)
        ranges = [out[(r, i)][:2] for r in range(world)]
        assert ranges == [slice_range(P, world, r) for r in range(world)]
        scale = max(np.abs(s_ref).max(), 1e-300)
        gscale = max(np.abs(g_ref).max(), 1e-300)
        for r in range(world):
            _, _, s, g = out[(r, i)]
            # every rank holds the same combined values, equal to the all-slice average
            assert np.max(np.abs(s - s_ref)) <= 1e-13 * scale
            assert np.max(np.abs(g - g_ref)) <= 1e-13 * gscale
