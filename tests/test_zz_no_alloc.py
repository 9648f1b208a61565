"""slk_sum_noalloc: kernel sums for callers that must not allocate device memory
while they run (a serving loop that reserved the GPU's memory for its own pool,
or code where the CUDA allocator may not be called).  Called through the C ABI
and compared with slk_sum on two calls in a row (the shared scratch array keeps
the previous call's contents, so the second call checks that it is cleared).

This file is named so that pytest collects it last."""
import ctypes
import math

import numpy as np
import pytest

from paper_2401_08260_gb300 import workloads
from tests._util import cuda_or_skip, rel_inf, to_dev, torch

pytestmark = pytest.mark.gpu


def _noalloc(plan, y, out):
    from paper_2401_08260_gb300 import slk
    lib = slk.load()
    stream = torch.cuda.current_stream(y.device).cuda_stream
    return lib.slk_sum_noalloc(plan.handle, y.data_ptr(), y.shape[0], y.stride(0), out.data_ptr(), stream)


# bf16/cheb is the route where slk_sum and slk_sum_noalloc differ most: slk_sum evaluates
# the Chebyshev form inside the projection kernel, slk_sum_noalloc projects first and then
# evaluates in a separate kernel; the two agree within the BF16 parity tolerance.
@pytest.mark.parametrize("kernel,precision,method", [("gaussian", "f32", "ndft"), ("gaussian", "bf16", "nfft"),
                                                     ("gaussian", "bf16", "cheb"), ("negdist", "f16x3", "auto"),
                                                     ("laplacian", "f32", "auto"), ("gaussian", "f64", "ndft")])
def test_noalloc_matches_slk_sum_twice(kernel, precision, method):
    dev = cuda_or_skip()
    from paper_2401_08260_gb300 import slk
    from paper_2401_08260_gb300.slk import Plan
    d, N, M, P = 64, 5003, 1201, 48
    dt = np.float64 if precision == "f64" else np.float32
    rng = np.random.Generator(np.random.PCG64(77))
    x = rng.standard_normal((N, d)).astype(dt)
    y = rng.standard_normal((M, d)).astype(dt)
    w = rng.random(N).astype(dt)
    xi = workloads.directions(P, d, seed=78)
    param = {"gaussian": math.sqrt(d), "laplacian": 1.0 / math.sqrt(d), "negdist": 0.0}[kernel]
    plan = Plan(to_dev(x, dev), to_dev(w, dev), kernel, param, P=P, precision=precision, method=method, directions=xi,
                radius=0.0)
    yt = to_dev(y, dev)
    ref = plan.sum(yt).cpu().numpy()
    tol = {"f64": 1e-10, "bf16": 2e-3}.get(precision, 1e-5)
    lib = slk.load()
    outs = [torch.full((M,), float("nan"), dtype=yt.dtype, device=dev) for _ in range(2)]
    plan.sync()
    allocs = lib.slk_device_alloc_count()
    for call in range(2):
        assert _noalloc(plan, yt, outs[call]) == 0
        plan.sync()
        assert rel_inf(outs[call], ref, w.sum()) <= tol, (call, rel_inf(outs[call], ref, w.sum()))
    # neither call made a device allocation of the library
    assert lib.slk_device_alloc_count() == allocs


def test_noalloc_rejects_oversize_and_host_pointers():
    dev = cuda_or_skip()
    from paper_2401_08260_gb300 import slk
    from paper_2401_08260_gb300.slk import Plan
    d, P = 8, 64
    rng = np.random.Generator(np.random.PCG64(79))
    x = rng.standard_normal((100, d)).astype(np.float32)
    plan = Plan(to_dev(x, dev), to_dev(np.ones(100, dtype=np.float32), dev), "negdist", 0.0, P=P, precision="f32",
                directions=workloads.directions(P, d, seed=80))
    # P * M * 4 bytes of projections alone exceed the 64 MiB array
    M = (64 << 20) // (4 * P) + 1
    y = torch.zeros((M, d), dtype=torch.float32, device=dev)
    out = torch.empty(M, dtype=torch.float32, device=dev)
    assert _noalloc(plan, y, out) == 1
    assert b"scratch" in slk.load().slk_last_error()
    # host arrays are refused (they would need staging buffers)
    yh = np.zeros((10, d), dtype=np.float32)
    sh = np.zeros(10, dtype=np.float32)
    lib = slk.load()
    assert lib.slk_sum_noalloc(plan.handle, yh.ctypes.data, 10, d, sh.ctypes.data, None) == 1
    # the plan is still usable afterwards
    s = plan.sum(torch.zeros((3, d), dtype=torch.float32, device=dev))
    assert torch.isfinite(s).all()
