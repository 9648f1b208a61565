"""The roofline bookkeeping of bench.py on CPU: the algorithmic amount it divides by each
kernel's measured time.  A miscounted kernel shows up in the bench line as a fraction far
from its real one (a centring cast once read 68 x its peak because it was charged for all N
sources on the CTA-pair route, where it only centres the radius sample), so the per-kernel
models are pinned here against the counts they state."""
import importlib.util
import os
from types import SimpleNamespace

import pytest

pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_accounting", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _wl(name, N, M, d, P):
    # the fields the bookkeeping reads, without generating the inputs
    return SimpleNamespace(name=name, N=N, M=M, d=d, P=P)


# the kernels one step of the Gaussian d = 784 benchmark launches on the CTA-pair route
PAIR_ROUTE = {"pair_cheb_moments": None, "pair_cheb_target": None, "gather_rows": None, "center_cast": None,
              "umma_project_bf16": None, "cheb_reduce": None, "sample_mean_partial": None}
PEAKS = {"hbm_gbs": 6789.3, "bf16_tflops_sustained": 1721.0}


def test_pair_route_centring_cast_sees_only_the_radius_sample(bench):
    wl = _wl("gauss_d784", 10 ** 6, 10 ** 6, 784, 512)
    assert bench.step_points(wl, "center_cast", PAIR_ROUTE) == 4096
    amount, unit, bound = bench.algorithmic(wl, {}, "bf16", "center_cast", 1, PAIR_ROUTE, peaks=PEAKS)
    assert (unit, bound) == ("byte", "hbm")
    assert amount == 4096 * (4.0 * 784 + 2.0 * 784)
    # the projection of that sample is counted on the sample too
    assert bench.step_points(wl, "umma_project_bf16", PAIR_ROUTE) == 4096


def test_pair_kernels_count_the_fp32_rows_and_the_contraction(bench):
    wl = _wl("gauss_d784", 10 ** 6, 10 ** 6, 784, 512)
    src, unit, bound = bench.algorithmic(wl, {}, "bf16", "pair_cheb_moments", 1, PAIR_ROUTE, peaks=PEAKS)
    flops = 2.0 * 10 ** 6 * 784 * 512
    nbytes = 10 ** 6 * (4.0 * 784 + 4.0)
    # the bound is the one with the longer minimum time under the peaks
    t_hbm, t_tc = nbytes / (PEAKS["hbm_gbs"] * 1e9), flops / (PEAKS["bf16_tflops_sustained"] * 1e12)
    assert (src, unit, bound) == ((flops, "flop", "tensor") if t_tc > t_hbm else (nbytes, "byte", "hbm"))
    tgt, unit, bound = bench.algorithmic(wl, {}, "bf16", "pair_cheb_target", 1, PAIR_ROUTE, peaks=PEAKS)
    nbytes_t = 10 ** 6 * (4.0 * 784 + 8.0 * 4)  # FP32 rows in, four FP64 partial sums out
    assert tgt == (flops if t_tc > nbytes_t / (PEAKS["hbm_gbs"] * 1e9) else nbytes_t)


@pytest.mark.parametrize("kernel", ["pair_cheb_moments", "pair_cheb_target", "center_cast", "umma_project_bf16",
                                    "spread_sorted", "nfft_target"])
def test_per_launch_amount_splits_the_step(bench, kernel):
    """Launches of one step share its work: per-launch amount x launches does not depend on
    how many launches the step took."""
    wl = _wl("gauss_d784", 10 ** 6, 10 ** 6, 784, 512)
    one = bench.algorithmic(wl, {}, "bf16", kernel, 1, PAIR_ROUTE, peaks=PEAKS)[0]
    four = bench.algorithmic(wl, {}, "bf16", kernel, 4, PAIR_ROUTE, peaks=PEAKS)[0]
    assert four * 4 == pytest.approx(one, rel=1e-12)


def test_sorting_route_counts_each_pass(bench):
    """Grouping 1e7 sources of 128 slices by key bucket (2^21 buckets): each histogram launch
    reads the 4-byte keys of all slices, each scatter launch reads and writes the 8-byte
    (key, w) pairs; the lookups read the target projections and, once per slice, the pairs
    and the 32-byte bucket records."""
    N = M = 10 ** 7
    P, nb = 128, 1 << 21
    wl = _wl("laplace_d50", N, M, 50, P)
    info = {"sort_buckets": nb}
    kernels = {"radix_hist": None, "radix_scatter": None, "negdist_target": None}
    assert bench.algorithmic(wl, info, "f32", "radix_hist", 3, kernels)[0] == 4.0 * N * P
    assert bench.algorithmic(wl, info, "f32", "radix_scatter", 3, kernels)[0] == 16.0 * N * P
    look, unit, bound = bench.algorithmic(wl, info, "f32", "negdist_target", 1, kernels)
    assert (unit, bound) == ("byte", "hbm")
    assert look == (4.0 * M + 8.0 * N + 32.0 * (nb + 1)) * P
    both = bench.algorithmic(wl, info, "f32", "negdist_target_both", 1, kernels)[0]
    assert both == look + 4.0 * M * P  # plus the per-slice derivatives written


def test_no_stale_ncu_traffic(bench):
    """Traffic figures exist only for kernels as they were captured; a workload without an
    entry reports none."""
    wl = _wl("laplace_d50", 10 ** 7, 10 ** 7, 50, 128)
    assert bench.measured_traffic(wl, "negdist_target", 1, {}) is None
    for (name, kernel), per_point in bench.NCU_TRAFFIC_PER_POINT.items():
        assert per_point > 0 and isinstance(name, str) and isinstance(kernel, str)
