"""Sums with per-slice derivatives in one pass (slk_sum_derivs) and the gradient from those
derivatives (slk_grad_derivs), through the C ABI: the sums equal slk_sum's, the derivatives
g[p, m] equal the oracle's derivative of every slice's exact 1-D sum (Section 3.2 with
sign(0) = 0; Sections 3.1 and 3.3 differentiated), and the gradient equals slk_grad's
bit for bit and the oracle's y-gradient."""
import math

import numpy as np
import pytest

import oracle
from paper_2401_08260_gb300 import workloads
from tests._util import cuda_or_skip, rel_inf, to_dev, torch

pytestmark = pytest.mark.gpu

CASES = [("negdist", "f32", "auto"), ("negdist", "f16x3", "auto"), ("negdist", "f64", "auto"),
         ("laplacian", "f32", "auto"), ("laplacian", "f16x3", "auto"), ("gaussian", "f32", "nfft"),
         ("gaussian", "f32", "ndft"), ("gaussian", "f32", "cheb"), ("gaussian", "bf16", "cheb"),
         ("gaussian", "f64", "ndft"), ("matern32", "f32", "auto")]


def _inputs(kernel, precision, N=5003, M=301, d=40, P=29, seed=31):
    rng = np.random.Generator(np.random.PCG64(seed))
    dt = np.float64 if precision == "f64" else np.float32
    x = rng.standard_normal((N, d)).astype(dt)
    y = rng.standard_normal((M, d)).astype(dt)
    w = rng.random(N).astype(dt)
    gs = rng.standard_normal(M).astype(dt)
    xi = workloads.directions(P, d, seed=seed + 1)
    param = math.sqrt(d) if kernel in ("gaussian", "matern32") else (1.0 / math.sqrt(d) if kernel == "laplacian"
                                                                     else 0.0)
    return x, y, w, gs, xi, param


@pytest.mark.parametrize("kernel,precision,method", CASES)
def test_sum_derivs_agrees_with_sum_grad_and_oracle(kernel, precision, method):
    dev = cuda_or_skip()
    from paper_2401_08260_gb300.slk import Plan
    x, y, w, gs, xi, param = _inputs(kernel, precision)
    M, P = y.shape[0], xi.shape[0]
    plan = Plan(to_dev(x, dev), to_dev(w, dev), kernel, param, P=P, precision=precision, directions=xi,
                method=method)
    yd, gsd = to_dev(y, dev), to_dev(gs, dev)
    s_ref = plan.sum(yd)
    s, g = plan.sum_derivs(yd)
    assert tuple(g.shape) == (P, M)
    wsum = float(np.abs(w).sum())
    if precision == "bf16":
        # slk_sum evaluates inside the fused projection kernel; here the projections are
        # stored and evaluated separately: the same BF16 products, other FP32 rounding order
        assert rel_inf(s, s_ref.cpu().numpy(), wsum) <= 1e-6
    else:
        np.testing.assert_array_equal(s.cpu().numpy(), s_ref.cpu().numpy())
    # the gradient from the saved derivatives is slk_grad's (same derivatives, same product)
    gy = plan.grad_derivs(g, gs=gsd)
    gy_ref = plan.grad(yd, gs=gsd)
    np.testing.assert_array_equal(gy.cpu().numpy(), gy_ref.cpu().numpy())
    # the derivatives against the oracle's per-slice derivative sums of the exact 1-D sums
    _, g_oracle, _, G_oracle, _ = oracle.sliced_sum(kernel, param, x, y, w, xi, grad=True, per_slice=True)
    scale = wsum * (oracle.cd(x.shape[1]) if kernel == "negdist" else 1.0)
    # per slice (no averaging over slices) and, for the gradient, averaged over them; the
    # tensor-core precisions (bf16, f16x3) form the backward product from BF16 operands
    # (2^-9 relative per term; 29 slices average little of it away here)
    tol_slice = {"f64": 1e-8, "f32": 1e-4, "f16x3": 1e-4, "bf16": 1e-2}[precision]
    tol_grad = {"f64": 1e-8, "f32": 2e-5, "f16x3": 1e-3, "bf16": 2e-3}[precision]
    err = np.abs(g.cpu().numpy().T.astype(np.float64) - G_oracle) / scale
    if kernel in ("negdist", "laplacian"):
        # the |z - x| part's derivative jumps by 2 c_d w_n (times alpha for the Laplacian)
        # where z crosses a source; a target within rounding of a source projection may
        # land on the other side of that jump than the FP64 oracle's
        jump = 2.0 * float(np.abs(w).max()) * oracle.cd(x.shape[1]) * (param if kernel == "laplacian" else 1.0)
        assert np.mean(err > tol_slice) <= 0.02, np.mean(err > tol_slice)
        assert err.max() <= jump / scale + tol_slice
    else:
        assert err.max() <= tol_slice
    assert rel_inf(gy, g_oracle * gs[:, None], scale) <= tol_grad


def test_host_buffers_and_strided_derivatives():
    """Host arrays in and out give the device results; the C entry point writes the
    derivatives into rows of a wider caller buffer (ldd > M) and reads them back from it."""
    dev = cuda_or_skip()
    import ctypes
    from paper_2401_08260_gb300 import slk
    from paper_2401_08260_gb300.slk import Plan
    x, y, w, gs, xi, param = _inputs("negdist", "f32", N=3001, M=129, P=17, seed=41)
    M, P, d = y.shape[0], xi.shape[0], x.shape[1]
    plan = Plan(to_dev(x, dev), to_dev(w, dev), "negdist", 0.0, P=P, precision="f32", directions=xi)
    s_dev, g_dev = plan.sum_derivs(to_dev(y, dev))
    s_host, g_host = plan.sum_derivs(y)
    np.testing.assert_array_equal(s_host, s_dev.cpu().numpy())
    np.testing.assert_array_equal(g_host, g_dev.cpu().numpy())
    ldd = M + 37
    wide = torch.full((P, ldd), 7.0, dtype=torch.float32, device=dev)
    s2 = torch.empty(M, dtype=torch.float32, device=dev)
    yd = to_dev(y, dev)
    lib = slk.load()
    assert lib.slk_sum_derivs(plan.handle, ctypes.c_void_p(yd.data_ptr()), M, d, ctypes.c_void_p(s2.data_ptr()),
                              ctypes.c_void_p(wide.data_ptr()), ldd, None) == 0
    plan.sync()
    np.testing.assert_array_equal(wide[:, :M].cpu().numpy(), g_dev.cpu().numpy())
    assert bool((wide[:, M:] == 7.0).all())
    gy = torch.empty(M, d, dtype=torch.float32, device=dev)
    gsd = to_dev(gs, dev)
    assert lib.slk_grad_derivs(plan.handle, ctypes.c_void_p(wide.data_ptr()), M, ldd,
                               ctypes.c_void_p(gsd.data_ptr()), ctypes.c_void_p(gy.data_ptr()), d, None) == 0
    plan.sync()
    np.testing.assert_array_equal(gy.cpu().numpy(), plan.grad(yd, gs=gsd).cpu().numpy())


def test_autograd_keeps_the_forward_derivatives():
    """sliced_kernel_sum: forward through slk_sum_derivs, backward through slk_grad_derivs;
    the gradient equals slk_grad's, and without requires_grad the forward is slk_sum."""
    dev = cuda_or_skip()
    from paper_2401_08260_gb300.slk import Plan, sliced_kernel_sum
    x, y, w, gs, xi, param = _inputs("laplacian", "f32", N=4001, M=97, P=23, seed=51)
    plan = Plan(to_dev(x, dev), to_dev(w, dev), "laplacian", param, P=23, precision="f32", directions=xi)
    yd = to_dev(y, dev).requires_grad_(True)
    gsd = to_dev(gs, dev)
    s = sliced_kernel_sum(yd, plan)
    (s * gsd).sum().backward()
    np.testing.assert_array_equal(yd.grad.cpu().numpy(), plan.grad(yd.detach(), gs=gsd).cpu().numpy())
    with torch.no_grad():
        s0 = sliced_kernel_sum(yd.detach(), plan)
    np.testing.assert_array_equal(s0.cpu().numpy(), s.detach().cpu().numpy())
