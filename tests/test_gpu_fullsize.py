"""Parity at the full workload sizes, in the launch configuration the benchmark
times: every output is computed on the GPU and a seeded sample of targets is
checked against the FP64 oracle (all sources, all slices)."""
import numpy as np
import pytest

import oracle
from paper_2401_08260_gb300 import workloads
from tests._util import cuda_or_skip, rel_inf, to_dev, torch

pytestmark = pytest.mark.gpu


def _run(name, precision, n_sample, grad=False, method=None):
    dev = cuda_or_skip()
    from paper_2401_08260_gb300.slk import Plan
    wl = workloads.make(name)
    plan = Plan(to_dev(wl.x, dev), to_dev(wl.w, dev), wl.kernel, wl.param, P=wl.P, precision=precision,
                n_coeff=wl.n_coeff, method=method or wl.method, directions=wl.xi)
    yt = to_dev(wl.y, dev)
    s = plan.sum(yt)
    idx = oracle.sampled_targets(wl.M, n_sample)
    assert torch.isfinite(s).all()
    g = plan.grad(yt[idx]) if grad else None
    out = oracle.sliced_sum(wl.kernel, wl.param, wl.x, wl.y[idx], wl.w, wl.xi, grad=grad)
    return wl, s.cpu().numpy()[idx], out, g, plan.info()


def test_gauss_d784_bf16_full():
    wl, s, (ref, _), _, info = _run("gauss_d784", "bf16", 4)
    assert rel_inf(s, ref, np.abs(wl.w).sum()) <= 2e-3, info


def test_negdist_d3072_f16x3_full_with_gradient():
    wl, s, (ref, gref, _), g, info = _run("negdist_d3072", "f16x3", 8, grad=True)
    wsum = np.abs(wl.w).sum()
    assert rel_inf(s, ref, wsum) <= 1e-5
    assert rel_inf(g, gref, wsum * oracle.cd(wl.d)) <= 2e-5


def test_laplace_d50_full():
    wl, s, (ref, _), _, info = _run("laplace_d50", "f32", 2)
    assert rel_inf(s, ref, np.abs(wl.w).sum()) <= 1e-5, info
