"""Projection step (Algorithm 1: z = <xi_p, x - mu>) of every precision path
against FP64 inner products, with rounding bounds derived from the input
formats (unit roundoff u = 2^-8 for BF16): BF16 inputs 2u sum|xi_i||x_i|, FP16 hi/lo split 2^-19 sum|xi_i||x_i|,
FP32 accumulation 2^-23 (4 + 2 sqrt(d)) sum|xi_i||x_i|."""
import numpy as np
import pytest

from paper_2401_08260_gb300 import workloads
from tests._util import cuda_or_skip, to_dev, torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["f32", "bf16", "f16x3", "f64"])
@pytest.mark.parametrize("d", [16, 50, 64, 128, 200, 784, 3072])
def test_projection_error_bounds(precision, d):
    dev = cuda_or_skip()
    from paper_2401_08260_gb300.slk import Plan
    rng = np.random.Generator(np.random.PCG64(d))
    n, P = 517, 300
    dt = np.float64 if precision == "f64" else np.float32
    x = rng.standard_normal((n, d)).astype(dt)
    xi = workloads.directions(P, d, seed=d + 1)
    plan = Plan(to_dev(x, dev), to_dev(np.ones(n, dtype=dt), dev), "negdist", 0.0, P=P, precision=precision,
                directions=xi)
    Z = plan.project(to_dev(x, dev)).cpu().numpy().astype(np.float64)
    # FP32 accumulation: a few units of 2^-24 per sqrt(term) on top of the input format
    bound = {"f32": 2.0 ** -23 * (4 + 2 * np.sqrt(d)), "bf16": 2.0 ** -7, "f16x3": 2.0 ** -19,
             "f64": 1e-13}[precision]
    mu = plan.center()
    xc = x.astype(np.float64) - mu
    ref = xi @ xc.T
    scale = np.abs(xi) @ np.abs(xc).T
    ratio = np.abs(Z - ref) / np.maximum(scale, 1e-300)
    worst = float(ratio.max())
    assert worst <= bound, (precision, d, worst, bound, np.unravel_index(ratio.argmax(), ratio.shape))
