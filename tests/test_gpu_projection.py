"""Projection step (Algorithm 1: z = <xi_p, x - mu>) of every precision path
against FP64 inner products, with rounding bounds derived from the input
formats: BF16 inputs 2^-8 sum|xi_i||x_i|, FP16 hi/lo split 2^-19 sum|xi_i||x_i|,
FP32 2^-20 sum|xi_i||x_i| (plus accumulation)."""
import numpy as np
import pytest

from paper_2401_08260_gb300 import workloads
from tests._util import cuda_or_skip, to_dev, torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,bound", [("f32", 2.0 ** -20), ("bf16", 2.0 ** -8), ("f16x3", 2.0 ** -19),
                                             ("f64", 1e-13)])
@pytest.mark.parametrize("d", [16, 50, 64, 128, 200, 784, 3072])
def test_projection_error_bounds(precision, bound, d):
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
    mu = plan.center()
    xc = x.astype(np.float64) - mu
    ref = xi @ xc.T
    scale = np.abs(xi) @ np.abs(xc).T
    ratio = np.abs(Z - ref) / np.maximum(scale, 1e-300)
    worst = float(ratio.max())
    assert worst <= bound, (precision, d, worst, bound, np.unravel_index(ratio.argmax(), ratio.shape))
