"""Parity at the full workload sizes, in the launch configuration the benchmark
times: every output is computed on the GPU and a seeded sample of targets is
checked against the FP64 oracle (all sources, all slices)."""
import numpy as np
import pytest

import oracle
from paper_2401_08260_gb300 import workloads
from tests._util import cuda_or_skip, rel_inf, to_dev, torch

pytestmark = pytest.mark.gpu


def _targets(M, n_random, n_tail):
    """Seeded random targets (almost all of them in a later work item of a persistent CTA
    or CTA pair) plus rows of the last partial 128- and 256-row tiles: the first rows of
    the last partial tile and the last rows of the array."""
    idx = set(oracle.sampled_targets(M, n_random).tolist())
    last = M - (M % 128 if M % 128 else 128)
    idx |= set(range(last, min(M, last + n_tail // 2)))
    idx |= set(range(M - (n_tail - n_tail // 2), M))
    return np.array(sorted(idx))


def _run(name, precision, n_sample, grad=False, method=None, n_tail=8):
    dev = cuda_or_skip()
    from paper_2401_08260_gb300.slk import Plan
    wl = workloads.make(name)
    plan = Plan(to_dev(wl.x, dev), to_dev(wl.w, dev), wl.kernel, wl.param, P=wl.P, precision=precision,
                n_coeff=wl.n_coeff, method=method or wl.method, directions=wl.xi)
    yt = to_dev(wl.y, dev)
    s = plan.sum(yt)
    idx = _targets(wl.M, n_sample, n_tail)
    assert torch.isfinite(s).all()
    g = plan.grad(yt[idx]) if grad else None
    out = oracle.sliced_sum(wl.kernel, wl.param, wl.x, wl.y[idx], wl.w, wl.xi, grad=grad)
    return wl, s.cpu().numpy()[idx], out, g, plan.info()


# Sample sizes follow the FP64 oracle's cost per target (all N sources x all P slices of
# exact 1-D sums on the machine's host cores): about 0.3 s at d = 3072 (f linear), 4 s at
# d = 784 (Gaussian series), 20 s at d = 50 (Laplacian series, N = 1e7).


def test_gauss_d784_bf16_full():
    wl, s, (ref, _), _, info = _run("gauss_d784", "bf16", 57)
    assert len(s) >= 64
    assert rel_inf(s, ref, np.abs(wl.w).sum()) <= 2e-3, info


def test_negdist_d3072_f16x3_full_with_gradient():
    wl, s, (ref, gref, _), g, info = _run("negdist_d3072", "f16x3", 57, grad=True)
    assert len(s) >= 64
    wsum = np.abs(wl.w).sum()
    assert rel_inf(s, ref, wsum) <= 1e-5
    assert rel_inf(g, gref, wsum * oracle.cd(wl.d)) <= 2e-5


def test_laplace_d50_full():
    wl, s, (ref, _), _, info = _run("laplace_d50", "f32", 6, n_tail=2)
    assert rel_inf(s, ref, np.abs(wl.w).sum()) <= 1e-5, info
