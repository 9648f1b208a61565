"""Benchmark of the sliced fast kernel summation on GB300.

One step = one pass of the whole path over one batch: directions, centring,
projection of sources and targets, the 1-D fast summation on every slice
(source side then target side) and the slice average, i.e. a plan build plus a
sum through the C ABI.  Default workload: Gaussian kernel, sigma = sqrt(d),
N = M = 1e6 sources and targets in d = 784 (x, y ~ U[0,1]^784, FP32), w = 1/N,
P = 512 directions, 256 Fourier coefficients.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
(exact 1-D sums on the same directions) on a bounded sample of the same
workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "(N+M)*P slice-points/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
            "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
             "clocks_event_reasons.sw_power_cap"

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_inputs(args):
    from paper_2401_08260_gb300 import workloads
    kw = {}
    if args.N:
        kw["N"] = args.N
    if args.M:
        kw["M"] = args.M
    if args.P:
        kw["P"] = args.P
    return workloads.make(args.workload, **kw)


def plan_kwargs(wl, args):
    return dict(kernel=wl.kernel, param=wl.param, P=wl.P, precision=args.precision or wl.precision,
                n_coeff=wl.n_coeff, method=args.method or wl.method, directions=wl.xi)


# DRAM read + write per point of one launch, from the ncu captures (summarised under
# profiles/) of the d = 784, P = 512 BF16 workload at n = 2e5 points; the traffic of these
# kernels grows in proportion to the points.  An entry is valid only for the kernel as
# captured and is removed when that kernel changes.
NCU_TRAFFIC_PER_POINT = {
    # none current: the Chebyshev pair kernels changed (converter loads batched per warp) after
    # their last capture in profiles/pair_cheb_d784_n200k.md (631.9 + 3.2 MB and 631.7 + 8.4 MB
    # of DRAM read + write per 2e5 points, equal to the algorithmic bytes)
}


def f32_direct(wl, kernels):
    """The fused Chebyshev path (the one that gathers a radius sample, `gather_rows`) hands
    contiguous FP32 target rows with d a multiple of four straight to its tensor-core target
    kernel, which centres and rounds them in shared memory; the sources (and otherwise the
    targets too) go through a centring cast first."""
    return "gather_rows" in kernels and wl.d % 4 == 0


def step_points(wl, kernel_name, kernels):
    """Rows that one step's launches of a kernel process together.  The fused Chebyshev path
    also centres, casts and projects a sample of min(4096, N) source rows (on the CTA-pair
    route the only rows the centring cast sees); source-side
    kernels see the N sources, target-side kernels the M targets, the rest both."""
    S = min(4096, wl.N) if "gather_rows" in kernels else 0
    if kernel_name.startswith("center_cast"):
        if "pair_cheb_moments" in kernels:
            return S  # the CTA-pair moments kernel reads the FP32 sources itself
        return wl.N + S if f32_direct(wl, kernels) else wl.N + wl.M + S
    if kernel_name.startswith(("umma_cheb_moments", "pair_cheb_moments", "cheb_moments", "ndft_source", "spread")):
        return wl.N
    if kernel_name.startswith(("umma_cheb_target", "pair_cheb_target", "umma_grad", "cheb_target", "ndft_target",
                               "nfft_target", "negdist_target")):
        return wl.M
    if kernel_name.startswith(("umma_project", "gemm")) and S:
        return S
    return wl.N + wl.M


def measured_traffic(wl, kernel_name, launches_per_step, kernels):
    """DRAM bytes of an average launch, from the per-point ncu figure (None without one)."""
    key = (wl.name, kernel_name)
    if key not in NCU_TRAFFIC_PER_POINT or wl.d != 784 or wl.P != 512 or wl.N != wl.M:
        return None
    return NCU_TRAFFIC_PER_POINT[key] * step_points(wl, kernel_name, kernels) / max(1.0, launches_per_step)


def algorithmic(wl, info, precision, kernel_name, launches_per_step, kernels, P=None, grad=False, peaks=None):
    """(algorithmic amount of an average launch, unit, bound) of a library kernel: the amount
    of one step's launches (their points from `step_points`) over the launches per step.

    Units of work: a point (row of x or y) and a slice-point (one point on one slice).
    Projection: 2 d P flop per point (tensor for BF16 / FP16x3, FP32 ALU otherwise;
    the fused Chebyshev target kernel is counted by its contraction alone).
    NDFT source / target: one complex multiply-add per band coefficient, 8 K flop per
    slice-point (FP32 ALU).  Chebyshev moments / Clenshaw: two FMAs per term, 4 q flop
    per slice-point (FP32 ALU).  Centring cast: 4 d bytes read + 2 ld16 (x2 for the
    hi/lo split) written per point; the gradient's derivative cast: 4 B read and 2 B
    written per target slice-point.  Sorting route: per source key and pass 4 B read
    (histogram) or a (key, w) pair read and written (scatter); the bucket tables read the
    pairs and write one 32-byte record per bucket; the target lookups read the 4-byte target
    projections and, once per slice, the sorted pairs and records they search (gradient:
    plus the derivatives written).  Other kernels: the 4-byte projections they read.
    The fused Chebyshev kernels that read the FP32 rows themselves move 4 d bytes per point
    (plus two FP64 partial sums per 256-slice half per target, or the 4-byte weight per
    source) beside
    their 2 d P flop; at d = 784, P = 512 the two minimum times are within 5% of each other,
    and the bound reported is the one with the longer minimum time under `peaks` (HBM copy
    bandwidth, sustained BF16).
    P: the slices one launch covers (this rank's share when the slices are sharded)."""
    P = wl.P if P is None else P
    pts = step_points(wl, kernel_name, kernels) / max(1.0, launches_per_step)
    per = 1.0 / max(1.0, launches_per_step)
    if kernel_name.startswith(("pair_cheb_target", "pair_cheb_moments")) or \
            (kernel_name.startswith("umma_cheb_target") and f32_direct(wl, kernels)):
        flops = 2.0 * pts * wl.d * P
        if kernel_name.startswith("pair_cheb_target"):
            nbytes = pts * (4.0 * wl.d + 8.0 * (4 if P > 256 else 2))  # FP32 rows in, FP64 partial sums out
        elif kernel_name.startswith("pair_cheb_moments"):
            nbytes = pts * (4.0 * wl.d + 4.0)  # FP32 rows and weights in (moment partials: per CTA pair)
        else:
            nbytes = pts * (4.0 * wl.d + 16.0 * ((P + 255) // 256))
        pk = peaks or {}
        t_hbm = nbytes / (pk.get("hbm_gbs", 6689.8) * 1e9)
        t_tc = flops / (pk.get("bf16_tflops_sustained", pk.get("bf16_tflops", 1772.1)) * 1e12)
        return (nbytes, "byte", "hbm") if t_hbm >= t_tc else (flops, "flop", "tensor")
    if kernel_name.startswith(("umma_project", "pair_project")):
        # 16-bit rows in (hi and lo parts for the FP16x3 split), FP32 projections out; the
        # bound with the longer minimum time (d = 50 is HBM-bound, d >= 784 tensor-bound)
        flops = 2.0 * pts * wl.d * P
        ld16 = (wl.d + 7) // 8 * 8
        nbytes = pts * (2.0 * ld16 * (2 if kernel_name.endswith("project_x3") else 1) + 4.0 * P)
        pk = peaks or {}
        t_hbm = nbytes / (pk.get("hbm_gbs", 6689.8) * 1e9)
        t_tc = flops / (pk.get("bf16_tflops_sustained", pk.get("bf16_tflops", 1772.1)) * 1e12)
        return (nbytes, "byte", "hbm") if t_hbm >= t_tc else (flops, "flop", "tensor")
    if kernel_name.startswith(("gemm", "umma")):
        bound = "tensor" if kernel_name.startswith("umma") else "alu"
        return 2.0 * pts * wl.d * P, "flop", bound
    nb = int(info.get("sort_buckets", 0) or 0)
    if nb > 0 and kernel_name.startswith(("radix_", "slice_minmax", "pair_chunk_sums", "pair_prefix_tab",
                                          "negdist_target")):
        # sorting route (sources of every slice grouped by key bucket): per source key of a
        # pass, 4 B read (histogram) or 8 B read + 8 B written (scatter of the (key, w) pair);
        # the per-slice state the targets look up (sorted pairs and 32-byte bucket records) is
        # counted once per slice, the 4-byte target projection once per slice-point
        kb = 8.0 if precision == "f64" else 4.0
        pairs = 2.0 * kb * wl.N
        records = 32.0 * (nb + 1)
        if kernel_name.startswith("radix_hist"):
            return kb * wl.N * P, "byte", "hbm"
        if kernel_name.startswith("radix_scatter"):
            return 2.0 * pairs * P, "byte", "hbm"
        if kernel_name.startswith("radix_scan"):
            tiles = -(-wl.N // 2048)
            return 2.0 * 4.0 * 256 * tiles * P, "byte", "hbm"
        if kernel_name.startswith("slice_minmax"):
            return per * kb * wl.N * P, "byte", "hbm"
        if kernel_name.startswith("pair_chunk_sums"):
            return per * pairs * P, "byte", "hbm"
        if kernel_name.startswith("pair_prefix_tab"):
            return per * (pairs + records) * P, "byte", "hbm"
        amount = per * (kb * wl.M + pairs + records) * P
        if kernel_name.startswith(("negdist_target_grad", "negdist_target_both")):
            amount += per * kb * wl.M * P  # the per-slice derivatives written
        return amount, "byte", "hbm"
    if kernel_name.startswith("ndft_source") or kernel_name.startswith("ndft_target"):
        K = info["k_hi"] - info["k_lo"] + 1
        return 8.0 * K * pts * P, "flop", "alu"
    if kernel_name.startswith(("cheb_moments", "cheb_target")):
        return 4.0 * info["cheb_terms"] * pts * P, "flop", "alu"
    if kernel_name.startswith("center_cast"):
        k = 2 if precision == "f16x3" else 1
        ld16 = (wl.d + 7) // 8 * 8
        return pts * (4.0 * wl.d + 2.0 * ld16 * k), "byte", "hbm"
    if kernel_name.startswith("spread_sorted"):
        return 8.0 * pts * P, "byte", "hbm"  # the (key, w) pair of every source slice-point
    if kernel_name.startswith("derivs_bf16"):
        # the M x P derivatives of the gradient: FP32 in, BF16 out (row pitch ld16(P))
        return per * wl.M * (4.0 * P + 2.0 * ((P + 7) // 8 * 8)), "byte", "hbm"
    if kernel_name.startswith(("nfft_target", "ndft_reduce", "spread_")):
        return 4.0 * pts * P, "byte", "hbm"
    # bookkeeping kernels (reductions of partial sums, the sample mean, casts of the
    # directions, the FFT of a few thousand grid cells): no roofline model
    return None, None, None


def cpu_sample(wl, budget_s: float):
    """Time the oracle's sliced sum on a bounded sample: k targets against all N
    sources and all P slices.  Returns (slice-points/s extrapolated, seconds, sample text,
    the sampled target indices, the oracle's sliced sums there)."""
    import oracle
    oracle.build()
    idx = oracle.sampled_targets(wl.M, 1)
    t0 = time.perf_counter()
    ref, _ = oracle.sliced_sum(wl.kernel, wl.param, wl.x, wl.y[idx[:1]], wl.w, wl.xi)
    t1 = time.perf_counter() - t0
    k = max(1, min(wl.M, int(budget_s / max(t1, 1e-3))))
    if k > 1:
        idx = oracle.sampled_targets(wl.M, k)
        t0 = time.perf_counter()
        ref, _ = oracle.sliced_sum(wl.kernel, wl.param, wl.x, wl.y[idx], wl.w, wl.xi)
        t1 = time.perf_counter() - t0
        k = len(idx)
    else:
        idx = idx[:1]
    full = t1 * wl.M / k
    rate = (wl.N + wl.M) * wl.P / full
    sample = (f"{k} target(s) x all {wl.N} sources x {wl.P} slices (FP64 exact 1-D sums, projections by numpy); "
              f"{t1:.2f} s measured, full job extrapolated to {full:.3g} s")
    return rate, t1, sample, idx, ref


def sampled_errors(wl, s_dev, idx, ref_sliced, model_error):
    """Errors of the device result at the oracle's sampled targets: l_inf / sum|w| against the
    sliced oracle (same directions, exact 1-D sums: the parity error) and against the direct
    d-dimensional sum (parity plus the slicing error)."""
    import numpy as np
    import oracle
    got = s_dev[idx].double().cpu().numpy()
    wsum = float(np.abs(wl.w.astype(np.float64)).sum())
    direct = oracle.direct_sum(wl.kernel, wl.param, wl.x, wl.y[idx], wl.w)
    return {"linf_over_sum_w_vs_sliced_oracle": float(np.max(np.abs(got - ref_sliced)) / wsum),
            "linf_over_sum_w_vs_direct_sum": float(np.max(np.abs(got - direct)) / wsum),
            "l1_over_sum_w_vs_sliced_oracle": float(np.mean(np.abs(got - ref_sliced)) / wsum),
            "certified_model_error": model_error, "targets": int(len(idx))}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = make_inputs(args)
    steps, warm = args.steps, args.warmup
    budget = max(2.0, 150.0 / (steps + warm))
    rates = []
    sample = ""
    for i in range(warm + steps):
        r, _, sample, _, _ = cpu_sample(wl, budget)
        if i >= warm:
            rates.append(r)
    value = statistics.median(rates)
    cores = len(os.sched_getaffinity(0))
    step_ms = (wl.N + wl.M) * wl.P / value * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "slice-points/s", "n_gpus": args.gpus,
            "steps": steps, "warmup": warm, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "N": wl.N, "M": wl.M, "d": wl.d, "P": wl.P},
            "cpu_baseline": {"value": value, "unit": "slice-points/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "slice-points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def max_over_ranks(x: float, device=None) -> float:
    """Largest x over the ranks of the default process group (x itself when there is
    none): the job's time is its slowest rank's."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, ms_per_step: float) -> float:
    """Whole-job throughput: every rank processes units_per_rank per step (replicas, weak
    scaling; for a slice-sharded sum the caller passes the whole job's units with world = 1),
    the step takes the slowest rank's ms_per_step."""
    return units_per_rank * world / (ms_per_step * 1e-3)


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2401_08260_gb300 import slk

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2401_08260_gb300 import build
    build.build()
    slk.load()

    wl = make_inputs(args)
    kw = plan_kwargs(wl, args)
    precision = kw["precision"]
    x = torch.from_numpy(wl.x).to(dev)
    y = torch.from_numpy(wl.y).to(dev)
    w = torch.from_numpy(wl.w).to(dev)
    s = torch.empty(wl.M, dtype=x.dtype, device=dev)
    # the directions are an input like x, y and w: resident on the device for the timed steps
    # (the end-to-end run below passes the host copy)
    kw_host = kw
    kw = dict(kw, directions=torch.from_numpy(wl.xi).to(dev))
    stream = torch.cuda.current_stream(dev)

    gy = torch.empty_like(y) if args.grad else None
    g_saved = torch.empty(wl.P, wl.M, dtype=y.dtype, device=dev) if args.grad else None
    sharded = args.parallel == "slices"
    if sharded:
        from paper_2401_08260_gb300.shard import ShardedPlan, SliceShard
        P_local = SliceShard(wl.P).count
        if P_local == 0:
            raise SystemExit("--parallel slices needs P >= the number of GPUs")
    else:
        P_local = wl.P

    def step():
        if sharded:
            # this rank's slices of the plan, then one all-reduce of the M sums (and of the gradient)
            sp = ShardedPlan(x, w, **kw)
            s.copy_(sp.sum(y))
            if args.grad:
                gy.copy_(sp.grad(y))
            sp.close()
            return
        plan = slk.Plan(x, w, **kw)
        if args.grad:
            # forward with the per-slice derivatives kept, backward product from them
            plan.sum_derivs(y, out=s, g=g_saved, sync=False)
            plan.grad_derivs(g_saved, out=gy, sync=False)
        else:
            plan.sum(y, out=s, sync=False)
        plan.close()

    for _ in range(args.warmup):
        step()
    if sharded:
        sp = ShardedPlan(x, w, **kw)
        info = sp.plan.info()
        sp.close()
    else:
        plan = slk.Plan(x, w, **kw)
        info = plan.info()
        plan.close()
    torch.cuda.synchronize()

    # ---------------- device-resident timed region
    sampler = ClockSampler(local)
    sampler.start()
    slk.timing_reset()
    slk.timing_enable(True)
    n0 = slk.launch_count()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    t_wall = time.perf_counter()
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    if world > 1:
        dist.barrier()
    launches = slk.launch_count() - n0
    slk.timing_enable(False)
    clocks = sampler.stop()
    kernels = slk.timing_read()
    slk.timing_reset()
    dev_ms = ev0.elapsed_time(ev1)
    # wall time includes the host work of plan creation (parameter selection is cached)
    ms = max_over_ranks(max(dev_ms, t_wall * 1e3) / args.steps, dev)
    # replicas: every rank sums all P slices; sharded: the ranks share one sum's P slices
    job_world = 1 if sharded else world
    value = job_rate((wl.N + wl.M) * wl.P, job_world, ms)

    # ---------------- roofline of every timed kernel, the dominant one on the line itself
    peaks, peak_kind = _peaks()

    def kernel_roofline(name, n_launch, tot_ms):
        per_step = n_launch / args.steps
        amount, unit, bound = algorithmic(wl, info, precision, name, per_step, kernels, P=P_local, grad=args.grad,
                                          peaks=peaks)
        if amount is None:
            return None
        avg_s = tot_ms / n_launch * 1e-3
        if bound == "tensor":
            # a kernel timed inside a long step: the sustained dense BF16 figure (FP16 runs at the same rate)
            peak = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
            achieved = amount / avg_s / 1e12
            runit = "TFLOP/s"
        elif bound == "alu":
            sm_mhz = peaks.get("sm_max_mhz", 2070.0)
            peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12  # FP32 FMA lanes x 2 flops x clock
            achieved = amount / avg_s / 1e12
            runit = "TFLOP/s"
        else:
            peak = peaks["hbm_gbs"]
            achieved = amount / avg_s / 1e9
            runit = "GB/s"
        return {"kernel": name, "bound": bound, "achieved": achieved, "peak": peak, "unit": runit,
                "frac": achieved / peak, "traffic": measured_traffic(wl, name, per_step, kernels),
                "peak_source": peak_kind, "launch_ms": tot_ms / n_launch,
                "share": tot_ms / sum(v[1] for v in kernels.values())}

    top = max(kernels.items(), key=lambda kv: kv[1][1]) if kernels else None
    roofline = kernel_roofline(top[0], *top[1]) if top else None
    # per kernel: ms per step, the fraction of its bound's peak, and that bound
    kernel_fracs = {}
    for kname, (n_launch, tot_ms) in sorted(kernels.items(), key=lambda kv: -kv[1][1]):
        if n_launch <= 0 or tot_ms <= 0.0:
            continue
        r = kernel_roofline(kname, n_launch, tot_ms)
        kernel_fracs[kname] = {"ms_per_step": tot_ms / args.steps, "bound": r["bound"] if r else None,
                               "frac": r["frac"] if r else None}

    # ---------------- end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        xh = torch.from_numpy(wl.x).pin_memory()
        yh = torch.from_numpy(wl.y).pin_memory()
        wh = torch.from_numpy(wl.w).pin_memory()
        sh = torch.empty(wl.M, dtype=xh.dtype).pin_memory()
        e2e_steps = max(1, min(args.steps, 5))

        gh = torch.empty_like(yh).pin_memory() if args.grad else None

        def host_step():
            if sharded:
                sp = ShardedPlan(xh, wh, **kw_host)
                sh.copy_(sp.sum(yh))
                if args.grad:
                    gh.copy_(sp.grad(yh))
                sp.close()
                return
            plan = slk.Plan(xh, wh, **kw_host)
            if args.grad:
                # the derivatives stay on the device between the two calls
                plan.sum_derivs(yh, out=sh, g=g_saved, sync=True)
                plan.grad_derivs(g_saved, out=gh, sync=True)
            else:
                plan.sum(yh, out=sh, sync=True)
            plan.close()

        host_step()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            host_step()
        torch.cuda.synchronize()
        te = max_over_ranks((time.perf_counter() - t0) / e2e_steps, dev)
        bi = xh.numel() * xh.element_size() + yh.numel() * yh.element_size() + wh.numel() * wh.element_size() + \
            P_local * wl.d * 8
        bo = sh.numel() * sh.element_size() + (gh.numel() * gh.element_size() if args.grad else 0)
        if sharded and world > 1:  # the combined results are staged through the GPU for the all-reduce
            bi, bo = bi + bo, bo + bo
        e2e = {"value": job_rate((wl.N + wl.M) * wl.P, job_world, te * 1e3), "unit": "slice-points/s",
               "h2d_bytes_per_step": int(bi),
               "d2h_bytes_per_step": int(bo), "ms_per_step": te * 1e3}

    cpu = None
    errors = None
    if rank == 0 and not args.no_cpu and world == 1:
        r, secs, sample, idx, ref = cpu_sample(wl, args.cpu_budget)
        cpu = {"value": r, "unit": "slice-points/s", "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
               "sample": sample}
        errors = sampled_errors(wl, s, idx, ref, info["model_error"])

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "slice-points/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms,
                "device_ms_per_step": dev_ms / args.steps, "wall_ms_per_step": t_wall * 1e3 / args.steps,
                "higher_is_better": True,
                "scaling": "strong" if sharded else "weak",
                "vs_baseline": None, "dtype": precision, "data": "synthetic",
                "config": {"workload": args.workload, "kernel": wl.kernel, "N": wl.N, "M": wl.M, "d": wl.d,
                           "P": wl.P, "n_coeff": info["n_coeff"], "method": {1: "nfft", 2: "ndft", 3: "cheb"}.get(info["method"]),
                           "parallelism": (f"slices{world}" if sharded else f"replicas{world}") if world > 1
                           else "single",
                           "l2": ("inputs larger than L2 (no flush needed)"
                                  if (wl.x.nbytes + wl.y.nbytes + wl.w.nbytes) > 2 * 129e6
                                  else "inputs smaller than L2, not flushed between steps (warm cache)"),
                           "model_error": info["model_error"], "backward": bool(args.grad)},
                "roofline": roofline, "cpu_baseline": cpu, "errors": errors, "e2e": e2e, "clocks": clocks,
                "gpu_launches": launches,
                "kernels_ms_per_step": {k: v[1] / args.steps for k, v in kernels.items()},
                "kernel_rooflines": kernel_fracs}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------- serving workload

SERVE_D = (50, 784, 3072)
SERVE_P = (64, 256, 1000)
SERVE_KERNELS = ("gaussian", "laplacian", "negdist")
SERVE_PRECISION = {50: "f16x3", 784: "bf16", 3072: "f16x3"}


def serve_requests(n_req: int, seed: int = 11, max_nm: float = 1e6):
    """Request specs of the serving workload: N, M log-uniform in [1e3, max_nm], d in {50, 784,
    3072} (each with the data distribution of its workload), kernels mixed uniformly, P in
    {64, 256, 1000}; 30% of the requests repeat the sources of one of the last 8 distinct
    requests (same kernel, P and sources: a plan-cache hit) with new targets."""
    rng = np.random.Generator(np.random.PCG64(seed))
    specs, distinct = [], []
    for i in range(n_req):
        M = int(round(10 ** rng.uniform(3, math.log10(max_nm))))
        if distinct and rng.random() < 0.3:
            base = distinct[int(rng.integers(max(0, len(distinct) - 8), len(distinct)))]
            specs.append(dict(base, M=M, y_seed=10_000 + i, repeat=True))
            continue
        d = int(rng.choice(SERVE_D))
        kernel = str(rng.choice(SERVE_KERNELS))
        spec = dict(key=len(distinct) + 1, kernel=kernel, d=d, P=int(rng.choice(SERVE_P)),
                    N=int(round(10 ** rng.uniform(3, math.log10(max_nm)))), M=M, x_seed=i, y_seed=10_000 + i,
                    precision=SERVE_PRECISION[d], repeat=False)
        distinct.append(spec)
        specs.append(spec)
    return specs


def serve_inputs(spec, dev, cache):
    """Device tensors (x, w, y, directions) of a request; sources of repeats come from `cache`."""
    import torch
    d = spec["d"]

    def points(n, seed, shift):
        g = torch.Generator(device=dev).manual_seed(seed)
        if d == 784:
            return torch.rand(n, d, device=dev, generator=g)
        if d == 50:
            gm = torch.Generator(device=dev).manual_seed(4)
            means = 2.0 * torch.randn(10, d, device=dev, generator=gm)
            comp = torch.randint(0, 10, (n,), device=dev, generator=g)
            return torch.randn(n, d, device=dev, generator=g) + means[comp]
        return torch.randn(n, d, device=dev, generator=g) + shift

    key = spec["key"]
    if key not in cache:
        g = torch.Generator(device=dev).manual_seed(spec["x_seed"] + 77)
        from paper_2401_08260_gb300 import workloads
        cache[key] = (points(spec["N"], spec["x_seed"], 0.0), torch.rand(spec["N"], device=dev, generator=g),
                      np.ascontiguousarray(workloads.directions(spec["P"], d, seed=spec["x_seed"])))
        while len(cache) > 8:
            cache.pop(next(iter(cache)))
    x, w, xi = cache[key]
    y = points(spec["M"], spec["y_seed"], 0.5 if d == 3072 else 0.0)
    return x, w, y, xi


def serve_desc(spec, xi):
    from paper_2401_08260_gb300 import slk
    d = spec["d"]
    param = {"gaussian": math.sqrt(d), "laplacian": 1.0 / math.sqrt(d), "negdist": 0.0}[spec["kernel"]]
    # certified window half-width per data distribution (projections of the centred data stay inside)
    radius = {50: 16.0, 784: 3.0, 3072: 8.0}[d]
    desc = slk.make_desc(spec["kernel"], param, d, spec["P"], spec["precision"], radius=radius)
    desc.directions = xi.ctypes.data
    return desc


def _serve_stream(srv, specs, arrivals, dev, keyed: bool, max_outstanding: int):
    """Submit the requests at their arrival times (at most max_outstanding in flight), poll
    them as they finish; returns (latencies in ms, plan-cache hits, batched requests, wall s,
    slice-points)."""
    import torch
    from paper_2401_08260_gb300 import slk  # noqa: F401
    cache = {}
    pending, lat, cached, batched = {}, [], 0, 0
    slice_points = 0

    def collect(rid, timeout_us):
        nonlocal cached, batched
        res = srv.poll(rid, timeout_us=timeout_us)
        if res is None:
            return False
        assert res["status"] == 0, res
        lat.append(res["total_ms"])
        cached += res["plan_cached"]
        batched += res["batch_requests"] > 1
        pending.pop(rid)
        return True

    t_start = time.perf_counter()
    for i, spec in enumerate(specs):
        while True:
            now = time.perf_counter() - t_start
            if now >= arrivals[i] and len(pending) < max_outstanding:
                break
            for rid in list(pending):
                collect(rid, 0)
            time.sleep(0.0002)
        x, w, y, xi = serve_inputs(spec, dev, cache)
        out = torch.empty(spec["M"], device=dev)
        torch.cuda.synchronize()
        desc = serve_desc(spec, xi)
        rid = srv.submit(x, w, y, out, desc, source_key=spec["key"] if keyed else 0)
        # the request reads the directions through desc when it starts: keep them until polled
        pending[rid] = (out, y, xi, desc)
        slice_points += (spec["N"] + spec["M"]) * spec["P"]
    for rid in list(pending):
        collect(rid, -1)
    return lat, cached, batched, time.perf_counter() - t_start, slice_points


def run_serve(args):
    """Serving benchmark: one Poisson stream of requests served twice on the same GPU, same
    requests and arrival times, same accuracy: by the plain method (one request at a time,
    plan + sum each, no plan cache: a server with one worker and no source keys) and by the
    concurrent server (memory-budgeted admission, worker streams, plan cache, repeats queued
    behind their plan's build and batched).  The arrival rate is `--serve-load` x the plain
    method's capacity, measured first by running every request alone."""
    import torch
    from paper_2401_08260_gb300 import build, slk
    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    specs = serve_requests(args.serve_requests, max_nm=args.serve_max_nm)
    cache = {}
    # ---- capacity of the plain method: every request alone, in order
    service = []
    for spec in specs:
        x, w, y, xi = serve_inputs(spec, dev, cache)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan = slk.Plan(x, w, spec["kernel"], serve_desc(spec, xi).param, P=spec["P"], precision=spec["precision"],
                        directions=xi, radius=serve_desc(spec, xi).radius)
        plan.sum(y)
        plan.close()
        service.append(time.perf_counter() - t0)
    mean_service = float(np.mean(service))
    rate = args.serve_load / mean_service
    rng = np.random.Generator(np.random.PCG64(12))
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=len(specs)))
    # ---- plain method served at the arrival times: one worker, no cache
    srv = slk.Server(workers=1)
    lat_p, _, _, wall_p, _ = _serve_stream(srv, specs, arrivals, dev, False, args.serve_max_outstanding)
    srv.close()
    # ---- the concurrent server
    srv = slk.Server(workers=args.serve_workers)
    lat, cached, batched, wall, slice_points = _serve_stream(srv, specs, arrivals, dev, True,
                                                             args.serve_max_outstanding)
    srv.close()
    repeats = sum(1 for s_ in specs if s_["repeat"])
    line = {"metric": "serving p50/p99 latency", "unit": "ms", "higher_is_better": False,
            "value": float(np.percentile(lat, 50)), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "throughput_req_s": len(specs) / wall,
            "slice_points_per_s": slice_points / wall, "n_gpus": 1, "requests": len(specs),
            "load": args.serve_load, "arrival_rate_req_s": rate, "workers": args.serve_workers,
            "repeats": repeats, "plan_cache_hits": cached, "batched_requests": batched, "data": "synthetic",
            "plain_one_at_a_time": {"p50_ms": float(np.percentile(lat_p, 50)),
                                    "p99_ms": float(np.percentile(lat_p, 99)),
                                    "throughput_req_s": len(specs) / wall_p,
                                    "mean_service_ms": mean_service * 1e3,
                                    "capacity_req_s": 1.0 / mean_service},
            "config": {"workload": "serving mix", "N_M": f"log-uniform [1e3, {args.serve_max_nm:g}]",
                       "d": list(SERVE_D), "P": list(SERVE_P), "kernels": list(SERVE_KERNELS), "repeats": 0.3}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- slicing vs random Fourier features

def run_rff(args):
    """Section 4.3's comparison on this GPU: the setup of the paper's Table 2 (d = 1000,
    N = M = 1e5, x, y ~ N(0, 0.1^2 I), w ~ U[0,1]; Gaussian sigma^2 = 5 with D = P,
    Laplacian alpha = 0.25 with D = 2P) for slicing and RFF-1 / RFF-2, all FP32: device time of
    one estimate (features / directions drawn by the library) and the per-summand l1 error
    against the direct sum at a seeded sample of targets (FP64 oracle on the host)."""
    import torch
    import oracle
    from paper_2401_08260_gb300 import slk
    dev = torch.device("cuda", 0)
    d, N, M = 1000, args.rff_n, args.rff_n
    rng = np.random.Generator(np.random.PCG64(1))
    X = (0.1 * rng.standard_normal((N, d))).astype(np.float32)
    Y = (0.1 * rng.standard_normal((M, d))).astype(np.float32)
    w = rng.random(N).astype(np.float32)
    idx = oracle.sampled_targets(M, args.rff_targets)
    xs, ws, ys = (torch.from_numpy(a).to(dev) for a in (X, w, Y))
    rows = []

    def timed(fn):
        fn()  # warm-up (and the value)
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        out = fn()
        t1.record()
        torch.cuda.synchronize()
        return out, t0.elapsed_time(t1)

    for kernel, param, dfac in (("gaussian", math.sqrt(5.0), 1), ("laplacian", 0.25, 2)):
        ref = oracle.direct_sum(kernel, param, X, Y[idx], w)
        wsum = float(np.abs(w.astype(np.float64)).sum())

        def l1(s):
            got = s.double().cpu().numpy()[idx]
            return float(np.sum(np.abs(got - ref)) / (len(idx) * wsum))

        for P in args.rff_p:
            s, ms = timed(lambda: slk.kernel_sum(xs, ws, ys, kernel, param, P=P, precision="f32", seed=2))
            row = {"kernel": kernel, "P": P, "slicing_ms": ms, "slicing_l1": l1(s)}
            for v in (1, 2):
                D = dfac * P
                s, ms = timed(lambda: slk.rff_sum(xs, ws, ys, kernel, param, D, variant=v, precision="f32", seed=3))
                row[f"rff{v}_D"] = D
                row[f"rff{v}_ms"] = ms
                row[f"rff{v}_l1"] = l1(s)
            rows.append(row)
    line = {"metric": "slicing vs random Fourier features (per-summand l1 error, device ms)", "unit": "ms",
            "n_gpus": 1, "data": "synthetic", "dtype": "f32",
            "config": {"workload": "Table 2 setup", "d": d, "N": N, "M": M, "x, y": "N(0, 0.1^2 I)", "w": "U[0,1]",
                       "targets_checked": int(len(idx))},
            "rows": rows}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 200 for this library, about 0.8 s at the default workload so that "
                         "the clock sampler sees several samples; 10 for the reference arm, whose steps are oracle "
                         "samples of seconds each)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="gauss_d784")
    ap.add_argument("--precision", default=None)
    ap.add_argument("--method", default=None)
    ap.add_argument("--N", type=int, default=None)
    ap.add_argument("--M", type=int, default=None)
    ap.add_argument("--P", type=int, default=None)
    ap.add_argument("--grad", action="store_true", help="include the y-gradient (backward) in every step")
    ap.add_argument("--parallel", choices=["replicas", "slices"], default="replicas",
                    help="N > 1: independent replicas of the workload (default), or one workload whose "
                         "slices are split over the GPUs with one all-reduce of the sums per step")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--serve", action="store_true", help="run the serving workload instead")
    ap.add_argument("--rff", action="store_true", help="run the slicing vs random Fourier features comparison")
    ap.add_argument("--rff-n", type=int, default=100_000)
    ap.add_argument("--rff-p", type=int, nargs="+", default=[200, 1000, 5000])
    ap.add_argument("--rff-targets", type=int, default=64)
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-load", type=float, default=0.8, help="arrival rate / plain capacity")
    ap.add_argument("--serve-workers", type=int, default=4)
    ap.add_argument("--serve-max-nm", type=float, default=1e6)
    ap.add_argument("--serve-max-outstanding", type=int, default=32)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("at least 3 warm-up steps")
    if args.steps is None:
        args.steps = 10 if args.impl == "reference" else 200
    if args.rff:
        run_rff(args)
    elif args.serve:
        run_serve(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
