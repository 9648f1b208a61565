"""Slice ranges on the GPU: a plan over slices [p0, p0 + P) of the library's direction draw,
the per-rank plans of a sharded sum (two ranks emulated in one process: each plan's mean over
its own slices, weighted by its share, with the all-reduce replaced by a host sum), and the
one-shot sum over slice batches (Sec. 5.4, remark on memory and batching), each against the
oracle on the same directions.  Tolerances (max-norm over sum|w|, times c_d for the negative
distance) as in the parity tests: 1e-10 for FP64, 1e-5 for FP32, twice that for gradients."""
import numpy as np
import pytest

import oracle
from paper_2401_08260_gb300 import workloads
from tests._util import cuda_or_skip, rel_inf, to_dev, torch

pytestmark = pytest.mark.gpu


def _inputs(N, M, d, P, seed, dtype=np.float32):
    rng = np.random.Generator(np.random.PCG64(300 + seed))
    x = rng.standard_normal((N, d)).astype(dtype)
    y = (rng.standard_normal((M, d)) * 0.9).astype(dtype)
    w = rng.random(N).astype(dtype)
    return x, y, w, workloads.directions(P, d, seed=400 + seed)


def test_slice_offset_draws_rows_of_the_full_sequence():
    dev = cuda_or_skip()
    from paper_2401_08260_gb300.slk import Plan
    d, P = 33, 10  # odd d: the Box-Muller pair of the last coordinate is half used
    x, _, w, _ = _inputs(500, 10, d, P, seed=0)
    xd, wd = to_dev(x, dev), to_dev(w, dev)
    full = Plan(xd, wd, "negdist", P=P, precision="f32", seed=1234)
    xi = full.directions()
    full.close()
    for p0, k in [(0, 4), (4, 6), (3, 1), (9, 1)]:
        part = Plan(xd, wd, "negdist", P=k, precision="f32", seed=1234, slice_offset=p0)
        assert np.array_equal(part.directions(), xi[p0:p0 + k])
        part.close()
    other = Plan(xd, wd, "negdist", P=4, precision="f32", seed=1235)
    assert not np.array_equal(other.directions(), xi[:4])
    other.close()


@pytest.mark.parametrize("kernel,param,precision,tol", [("gaussian", 3.0, "f32", 1e-5),
                                                        ("negdist", 0.0, "f32", 1e-5),
                                                        ("laplacian", 0.4, "f64", 1e-6)])
@pytest.mark.parametrize("world", [2, 3])
def test_sharded_plans_combine_to_the_full_sum(kernel, param, precision, tol, world):
    dev = cuda_or_skip()
    from paper_2401_08260_gb300.shard import ShardedPlan
    d, N, M, P = 12, 9001, 2049, 23
    dtype = np.float64 if precision == "f64" else np.float32
    x, y, w, _ = _inputs(N, M, d, P, seed=1, dtype=dtype)
    xd, wd, yd = to_dev(x, dev), to_dev(w, dev), to_dev(y, dev)
    s = torch.zeros(M, dtype=torch.float64, device=dev)
    g = torch.zeros(M, d, dtype=torch.float64, device=dev)
    rows = []
    for r in range(world):
        sp = ShardedPlan(xd, wd, kernel, param, P=P, precision=precision, seed=77, rank=r, world=world)
        assert sp.shard.count in (P // world, P // world + 1)
        s += sp.plan.sum(yd).double() * sp.shard.weight
        g += sp.plan.grad(yd).double() * sp.shard.weight
        rows.append(sp.directions())
        sp.close()
    xi = np.concatenate(rows)  # the ranks' rows in order: the draw of one plan over all P slices
    ref, gref, _ = oracle.sliced_sum(kernel, param, x, y, w, xi, grad=True)
    # the negative distance's 1-D counterpart is -c_d |x|: its sums and gradients carry c_d
    scale = w.sum() * (oracle.cd(d) if kernel == "negdist" else 1.0)
    assert rel_inf(s, ref, scale) <= tol
    assert rel_inf(g, gref, scale) <= 2 * tol


@pytest.mark.parametrize("given", [False, True])
@pytest.mark.parametrize("precision,tol", [("f32", 1e-5), ("f64", 1e-10)])
def test_one_shot_sum_over_slice_batches(given, precision, tol):
    dev = cuda_or_skip()
    from paper_2401_08260_gb300 import slk
    d, N, M, P, B = 20, 7001, 1537, 10, 4  # batches of 4, 4 and 2 slices
    dtype = np.float64 if precision == "f64" else np.float32
    x, y, w, xi_given = _inputs(N, M, d, P, seed=2, dtype=dtype)
    xd, wd, yd = to_dev(x, dev), to_dev(w, dev), to_dev(y, dev)
    kw = dict(directions=xi_given) if given else dict(seed=99, slice_offset=5)
    if given:
        xi = xi_given
    else:
        full = slk.Plan(xd, wd, "gaussian", 4.0, P=P, precision=precision, seed=99, slice_offset=5)
        xi = full.directions()
        full.close()
    ref, _ = oracle.sliced_sum("gaussian", 4.0, x, y, w, xi)
    n0 = slk.launch_count()
    s = slk.kernel_sum(xd, wd, yd, "gaussian", 4.0, P=P, precision=precision, slice_batch=B, **kw)
    torch.cuda.synchronize()
    assert slk.launch_count() > n0
    assert rel_inf(s, ref, w.sum()) <= tol
    # host targets and host output: the FP64 accumulator is copied back at the end
    sh = slk.kernel_sum(xd, wd, y, "gaussian", 4.0, P=P, precision=precision, slice_batch=B, **kw)
    assert isinstance(sh, np.ndarray)
    assert rel_inf(sh, ref, w.sum()) <= tol
    # slice_batch >= P: one plan over all slices
    s1 = slk.kernel_sum(xd, wd, yd, "gaussian", 4.0, P=P, precision=precision, slice_batch=P, **kw)
    assert rel_inf(s1, ref, w.sum()) <= tol


def test_invalid_slice_fields():
    dev = cuda_or_skip()
    from paper_2401_08260_gb300 import slk
    x, y, w, _ = _inputs(100, 10, 4, 4, seed=3)
    xd, wd = to_dev(x, dev), to_dev(w, dev)
    with pytest.raises(slk.SlkError):
        slk.Plan(xd, wd, "negdist", P=4, slice_offset=-1)
    with pytest.raises(slk.SlkError):
        slk.Plan(xd, wd, "negdist", P=4, slice_offset=2 ** 31 - 4)
    with pytest.raises(slk.SlkError):
        slk.kernel_sum(xd, wd, to_dev(y, dev), "negdist", P=4, slice_batch=-2)
