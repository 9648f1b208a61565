"""The N > 1 host logic of bench.py on CPU: two gloo ranks (127.0.0.1) agree on the
slowest rank's step time, and the whole-job rate counts every replica's work."""
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench = _bench()
        local_ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
        ms = bench.max_over_ranks(local_ms)
        rate = bench.job_rate(1000.0, world, ms)
        out[rank] = (ms, rate)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    assert set(out.keys()) == {0, 1}
    for rank in range(world):
        ms, rate = out[rank]
        assert ms == 15.0
        assert rate == pytest.approx(1000.0 * world / 15e-3)


def test_single_process_is_unchanged():
    bench = _bench()
    assert bench.max_over_ranks(7.5) == 7.5
    assert bench.job_rate(2.0e9, 1, 10.0) == pytest.approx(2.0e11)


def test_roofline_amount_covers_every_launch_of_a_step():
    """The per-launch amount is one step's work over the step's launches: three centring
    launches (sources, targets, the 4096-row radius sample) share N + M + 4096 rows."""
    from types import SimpleNamespace
    bench = _bench()
    wl = SimpleNamespace(name="gauss_d784", N=10 ** 6, M=10 ** 6, d=784, P=512)
    kernels = {"center_cast": (3, 1.0), "gather_rows": (1, 0.01), "umma_cheb_moments": (1, 1.0)}
    amount, unit, bound = bench.algorithmic(wl, {}, "bf16", "center_cast", 3, kernels)
    assert (unit, bound) == ("byte", "hbm")
    assert amount * 3 == pytest.approx((2 * 10 ** 6 + 4096) * (4 * 784 + 2 * 784))
    amount, unit, bound = bench.algorithmic(wl, {}, "bf16", "umma_cheb_moments", 1, kernels)
    assert (unit, bound) == ("flop", "tensor") and amount == pytest.approx(2.0 * 10 ** 6 * 784 * 512)
    # a rank of a slice-sharded sum projects onto its own slices only
    amount, _, _ = bench.algorithmic(wl, {}, "bf16", "umma_cheb_moments", 1, kernels, P=256)
    assert amount == pytest.approx(2.0 * 10 ** 6 * 784 * 256)
    traffic = bench.measured_traffic(wl, "center_cast", 3, kernels)
    assert traffic * 3 == pytest.approx(bench.NCU_TRAFFIC_PER_POINT[("gauss_d784", "center_cast")] * (2 * 10 ** 6 + 4096))
