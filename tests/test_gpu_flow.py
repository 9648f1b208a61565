"""MMD / energy-distance particle flow (paper_2401_08260_gb300.flow) on the GPU: the velocity
against the oracle's sliced gradients on the same directions, and the flow itself driving the
energy distance to the target sample down."""
import numpy as np
import pytest

import oracle
from tests._util import cuda_or_skip, to_dev, torch

pytestmark = pytest.mark.gpu


def _energy_distance(a, b):
    """Direct energy distance 2E|a-b| - E|a-a'| - E|b-b'| (oracle direct sums of -|.|)."""
    wa = np.full(a.shape[0], 1.0 / a.shape[0])
    wb = np.full(b.shape[0], 1.0 / b.shape[0])
    s_ab = oracle.direct_sum("negdist", 0.0, b, a, wb).mean()
    s_aa = oracle.direct_sum("negdist", 0.0, a, a, wa).mean()
    s_bb = oracle.direct_sum("negdist", 0.0, b, b, wb).mean()
    return -2.0 * s_ab + s_aa + s_bb


def test_energy_flow_velocity_and_descent():
    dev = cuda_or_skip()
    from paper_2401_08260_gb300 import slk
    from paper_2401_08260_gb300.flow import MMDFlow
    d, N, M, P = 8, 3000, 600, 128
    rng = np.random.Generator(np.random.PCG64(51))
    x = rng.standard_normal((N, d)).astype(np.float32)
    y0 = (rng.standard_normal((M, d)) + 1.5).astype(np.float32)
    xd, yd = to_dev(x, dev), to_dev(y0, dev)
    flow = MMDFlow(xd, "negdist", 0.0, P=P, precision="f32", seed=5)

    # one velocity against the oracle: attraction by the plan on x, repulsion by a plan on y
    v = flow.velocity(yd, seed=77).cpu().numpy()
    xi_x = flow.plan_x.directions()
    py = slk.Plan(yd, torch.full((M,), 1.0 / M, device=dev), "negdist", 0.0, P=P, precision="f32", seed=77)
    xi_y = py.directions()
    py.close()
    _, g_att, _ = oracle.sliced_sum("negdist", 0.0, x, y0, np.full(N, 1.0 / N), xi_x, grad=True)
    _, g_rep, _ = oracle.sliced_sum("negdist", 0.0, y0, y0, np.full(M, 1.0 / M), xi_y, grad=True)
    ref = g_att - g_rep
    scale = oracle.cd(d)  # the sliced gradients carry the factor c_d of f = -c_d |x|
    assert np.max(np.abs(v - ref)) / scale <= 2e-5

    # the flow: the energy distance to x falls by an order of magnitude
    ed0 = _energy_distance(y0.astype(np.float64), x.astype(np.float64))
    y = yd
    for _ in range(40):
        y = flow.step(y, tau=0.25)
    yT = y.cpu().numpy().astype(np.float64)
    edT = _energy_distance(yT, x.astype(np.float64))
    assert edT < 0.1 * ed0, (ed0, edT)
    assert np.linalg.norm(yT.mean(axis=0)) < 0.25 * np.linalg.norm(y0.mean(axis=0))
    # the sliced MMD^2 monitor: parity with the oracle's sliced sums on the same directions,
    # and the direct energy distance within the slicing error of its two large terms
    est = flow.mmd2(y, seed=91)
    py = slk.Plan(y, torch.full((M,), 1.0 / M, device=dev), "negdist", 0.0, P=P, precision="f32", seed=91)
    xi_y = py.directions()
    py.close()
    s_yy, _ = oracle.sliced_sum("negdist", 0.0, yT, yT, np.full(M, 1.0 / M), xi_y)
    s_yx, _ = oracle.sliced_sum("negdist", 0.0, x, yT, np.full(N, 1.0 / N), xi_x)
    ref_est = s_yy.mean() - 2.0 * s_yx.mean()
    assert abs(est - ref_est) <= 1e-5 * scale
    xx = oracle.direct_sum("negdist", 0.0, x.astype(np.float64), x.astype(np.float64), np.full(N, 1.0 / N)).mean()
    assert abs((est + xx) - edT) <= 0.15 * ed0
    flow.close()
