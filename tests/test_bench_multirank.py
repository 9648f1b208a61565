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
    """The per-launch amount is one step's work over the step's launches.  On the fused
    Chebyshev path with d a multiple of four the target kernel reads the FP32 rows itself, so
    two centring launches (sources, the 4096-row radius sample) share N + 4096 rows;
    otherwise three (targets too) share N + M + 4096."""
    from types import SimpleNamespace
    bench = _bench()
    peaks = {"hbm_gbs": 6689.8, "bf16_tflops_sustained": 1772.1}
    kernels = {"center_cast": (2, 1.0), "gather_rows": (1, 0.01), "umma_cheb_moments": (1, 1.0),
               "umma_cheb_target": (1, 1.0)}
    wl = SimpleNamespace(name="gauss_d784", N=10 ** 6, M=10 ** 6, d=784, P=512)
    amount, unit, bound = bench.algorithmic(wl, {}, "bf16", "center_cast", 2, kernels)
    assert (unit, bound) == ("byte", "hbm")
    assert amount * 2 == pytest.approx((10 ** 6 + 4096) * (4 * 784 + 2 * 784))
    # the sources' projection: 2 d P flop per source on the tensor cores
    amount, unit, bound = bench.algorithmic(wl, {}, "bf16", "umma_cheb_moments", 1, kernels, peaks=peaks)
    assert (unit, bound) == ("flop", "tensor") and amount == pytest.approx(2.0 * 10 ** 6 * 784 * 512)
    # 3136 + 32 bytes per target at 6.69 TB/s outlast 2 d P flop at 1.77 PFLOP/s: HBM-bound
    amount, unit, bound = bench.algorithmic(wl, {}, "bf16", "umma_cheb_target", 1, kernels, peaks=peaks)
    assert (unit, bound) == ("byte", "hbm") and amount == pytest.approx(10 ** 6 * (4 * 784 + 32))
    # a rank of a slice-sharded sum projects onto its own slices only
    amount, _, _ = bench.algorithmic(wl, {}, "bf16", "umma_cheb_moments", 1, kernels, P=256)
    assert amount == pytest.approx(2.0 * 10 ** 6 * 784 * 256)
    amount, unit, bound = bench.algorithmic(wl, {}, "bf16", "umma_cheb_target", 1, kernels, P=256, peaks=peaks)
    assert (unit, bound) == ("byte", "hbm") and amount == pytest.approx(10 ** 6 * (4 * 784 + 16))
    # d not a multiple of four: the cast route for the targets too, three centring launches
    wl3 = SimpleNamespace(name="gauss_d786", N=10 ** 6, M=10 ** 6, d=786, P=512)
    kernels3 = dict(kernels, center_cast=(3, 1.0))
    amount, unit, bound = bench.algorithmic(wl3, {}, "bf16", "center_cast", 3, kernels3)
    ld16 = (786 + 7) // 8 * 8
    assert amount * 3 == pytest.approx((2 * 10 ** 6 + 4096) * (4 * 786 + 2 * ld16))
    amount, unit, bound = bench.algorithmic(wl3, {}, "bf16", "umma_cheb_target", 1, kernels3, peaks=peaks)
    assert (unit, bound) == ("flop", "tensor") and amount == pytest.approx(2.0 * 10 ** 6 * 786 * 512)
    # the CTA-pair kernels: 4 d bytes per point, plus two FP64 partial sums per 256-slice half
    # per target or the 4-byte weight per source
    pair_kernels = {"gather_rows": (1, 0.01), "pair_cheb_moments": (1, 1.0), "pair_cheb_target": (1, 1.0)}
    amount, unit, bound = bench.algorithmic(wl, {}, "bf16", "pair_cheb_target", 1, pair_kernels, peaks=peaks)
    assert (unit, bound) == ("byte", "hbm") and amount == pytest.approx(10 ** 6 * (4 * 784 + 32))
    amount, unit, bound = bench.algorithmic(wl, {}, "bf16", "pair_cheb_moments", 1, pair_kernels, peaks=peaks)
    assert (unit, bound) == ("byte", "hbm") and amount == pytest.approx(10 ** 6 * (4 * 784 + 4))
    # traffic is reported only from a capture of the kernel as it is
    for name in ("center_cast", "pair_cheb_target"):
        if (wl.name, name) not in bench.NCU_TRAFFIC_PER_POINT:
            assert bench.measured_traffic(wl, name, 1, pair_kernels) is None


def test_default_steps_per_arm(monkeypatch):
    """Without --steps the library's arm times 200 steps (several clock samples at about 4 ms a
    step) and the oracle's reference arm 10 (its steps are oracle samples of seconds each, and
    the whole run must stay within minutes); an explicit --steps applies to either arm."""
    import sys
    bench = _bench()
    seen = {}
    monkeypatch.setattr(bench, "run_ours", lambda a: seen.update(ours=a.steps))
    monkeypatch.setattr(bench, "run_reference", lambda a: seen.update(reference=a.steps))
    for argv in (["bench.py"], ["bench.py", "--impl", "reference"], ["bench.py", "--impl", "reference", "--steps", "4"]):
        monkeypatch.setattr(sys, "argv", argv)
        bench.main()
    assert seen == {"ours": 200, "reference": 4}
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference"])
    bench.main()
    assert seen["reference"] == 10
