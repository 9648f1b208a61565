"""Tensor-core projection (tcgen05 + TMA): BF16 and the FP16 hi/lo split against
the FP64 oracle, over shapes that exercise partial tiles in every dimension
(K tail beyond d, slices beyond P, points beyond n)."""
import math

import numpy as np
import pytest

import oracle
from paper_2401_08260_gb300 import workloads
from tests._util import cuda_or_skip, rel_inf, to_dev, torch

pytestmark = pytest.mark.gpu


def _plan(x, w, kernel, param, xi, precision, **kw):
    from paper_2401_08260_gb300.slk import Plan
    return Plan(x, w, kernel, param, P=xi.shape[0], precision=precision, directions=xi, **kw)


@pytest.mark.parametrize("N,M,P", [(1000, 200, 64), (3001, 257, 512), (2000, 1153, 300)])
def test_bf16_gaussian_d784(N, M, P):
    """BF16 projection, FP32 accumulate: within 2e-3 of the FP64 sliced sum.  The
    Chebyshev method runs the target side fused into the projection's epilogue."""
    dev = cuda_or_skip()
    d = 784
    rng = np.random.Generator(np.random.PCG64(11))
    x = rng.random((N, d), dtype=np.float32)
    y = rng.random((M, d), dtype=np.float32)
    w = np.full(N, 1.0 / N, dtype=np.float32)
    xi = workloads.directions(P, d, seed=12)
    sigma = math.sqrt(d)
    for method in ("ndft", "nfft", "cheb"):
        plan = _plan(to_dev(x, dev), to_dev(w, dev), "gaussian", sigma, xi, "bf16", n_coeff=256, method=method)
        s = plan.sum(to_dev(y, dev))
        ref, _ = oracle.sliced_sum("gaussian", sigma, x, y, w, xi)
        err = rel_inf(s, ref, w.sum())
        assert err <= 2e-3, (method, err)
        # and the BF16 result is close to the FP32 path (rounding of the inputs only)
        p32 = _plan(to_dev(x, dev), to_dev(w, dev), "gaussian", sigma, xi, "f32", n_coeff=256, method=method)
        s32 = p32.sum(to_dev(y, dev))
        assert rel_inf(s, s32.cpu().numpy(), w.sum()) <= 2e-3


def test_bf16_fused_chebyshev_matches_unfused_and_reports_window():
    """The fused route (projection + Clenshaw in one kernel, host or device output)
    agrees with the separate projection and the FP32 Chebyshev path on the same
    coefficients, and a target beyond the radius raises the window error."""
    dev = cuda_or_skip()
    from paper_2401_08260_gb300.slk import Plan, SlkError
    d, N, M, P = 784, 4000, 777, 512
    rng = np.random.Generator(np.random.PCG64(21))
    x = rng.random((N, d), dtype=np.float32)
    y = rng.random((M, d), dtype=np.float32)
    w = rng.random(N).astype(np.float32)
    xi = workloads.directions(P, d, seed=22)
    sigma = math.sqrt(d)
    plan = _plan(to_dev(x, dev), to_dev(w, dev), "gaussian", sigma, xi, "bf16", method="cheb", radius=2.5)
    assert plan.info()["method"] == 3 and plan.info()["cheb_terms"] > 0 and plan.info()["cheb_horner"] == 1
    s_dev = plan.sum(to_dev(y, dev)).cpu().numpy()
    s_host = plan.sum(y)
    np.testing.assert_array_equal(s_dev, s_host)
    ref, _ = oracle.sliced_sum("gaussian", sigma, x, y, w, xi)
    assert rel_inf(s_dev, ref, w.sum()) <= 2e-3
    # same BF16 projections, Clenshaw in the standalone kernel: the gradient path
    # computes t'_p the same way, so compare values through the SIMT FP32 plan instead
    p32 = _plan(to_dev(x, dev), to_dev(w, dev), "gaussian", sigma, xi, "f32", method="cheb", radius=2.5)
    assert rel_inf(s_dev, p32.sum(to_dev(y, dev)).cpu().numpy(), w.sum()) <= 2e-3
    far = y.copy()
    far[M - 1] += 60.0
    with pytest.raises(SlkError) as e:
        plan.sum(to_dev(far, dev))
    assert e.value.status == 4
    plan.sum(to_dev(y, dev))


@pytest.mark.parametrize("d,P,N,M", [(50, 128, 5003, 301), (3072, 1000, 2000, 129), (200, 300, 4097, 64)])
def test_f16x3_negdist(d, P, N, M):
    """FP16 hi/lo split (three products): FP32-level projection accuracy, within 1e-5."""
    dev = cuda_or_skip()
    rng = np.random.Generator(np.random.PCG64(13))
    x = rng.standard_normal((N, d), dtype=np.float32)
    y = (rng.standard_normal((M, d), dtype=np.float32) + 0.5).astype(np.float32)
    w = rng.random(N).astype(np.float32)
    xi = workloads.directions(P, d, seed=14)
    plan = _plan(to_dev(x, dev), to_dev(w, dev), "negdist", 0.0, xi, "f16x3")
    s = plan.sum(to_dev(y, dev))
    ref, _ = oracle.sliced_sum("negdist", 0.0, x, y, w, xi)
    err = rel_inf(s, ref, w.sum())
    assert err <= 1e-5, err


def test_f16x3_laplacian_and_gradient():
    dev = cuda_or_skip()
    wl = workloads.make("laplace_d50", N=8001, M=255, P=40)
    plan = _plan(to_dev(wl.x, dev), to_dev(wl.w, dev), "laplacian", wl.param, wl.xi, "f16x3")
    yt = to_dev(wl.y, dev)
    s = plan.sum(yt)
    g = plan.grad(yt)
    ref, gref, _ = oracle.sliced_sum("laplacian", wl.param, wl.x, wl.y, wl.w, wl.xi, grad=True)
    assert rel_inf(s, ref, wl.w.sum()) <= 1e-5
    assert rel_inf(g, gref, wl.w.sum()) <= 2e-5


@pytest.mark.parametrize("kernel,precision,method,tol", [("gaussian", "bf16", "cheb", 2e-3),
                                                         ("gaussian", "bf16", "ndft", 2e-3),
                                                         ("negdist", "f16x3", "auto", 1e-5)])
def test_large_point_sets_sampled(kernel, precision, method, tol):
    """Point sets of a few hundred thousand rows (many persistent-tile waves, ragged last
    tile): sampled targets, including rows at multiples of 65536, against the oracle."""
    dev = cuda_or_skip()
    d, P = 64, 32
    N, M = 2 * 65536 + 12345, 5 * 65536 + 7
    rng = np.random.Generator(np.random.PCG64(31))
    x = rng.standard_normal((N, d), dtype=np.float32)
    y = (rng.standard_normal((M, d), dtype=np.float32) + 0.25).astype(np.float32)
    w = rng.random(N).astype(np.float32)
    xi = workloads.directions(P, d, seed=32)
    param = math.sqrt(d) if kernel == "gaussian" else 0.0
    plan = _plan(to_dev(x, dev), to_dev(w, dev), kernel, param, xi, precision, method=method)
    s = plan.sum(to_dev(y, dev)).cpu().numpy()
    edges = np.array([0, 65535, 65536, 131071, 131072, 196607, 196608, 262143, 262144, 327679, 327680, M - 1])
    idx = np.unique(np.concatenate([edges, oracle.sampled_targets(M, 12)]))
    ref, _ = oracle.sliced_sum(kernel, param, x, y[idx], w, xi)
    assert rel_inf(s[idx], ref, w.sum()) <= tol


def test_bf16_fused_moments_radius_fallback():
    """The fused source side fixes its radius before projecting (1.5 x the largest projection
    over a sample of sources).  A source outside it (an outlier on an unsampled row) sends the
    plan down the two-pass route, whose radius covers every source; both agree with the oracle."""
    dev = cuda_or_skip()
    from paper_2401_08260_gb300.slk import Plan
    d, N, M, P = 64, 20000, 257, 48
    rng = np.random.Generator(np.random.PCG64(41))
    x = rng.random((N, d), dtype=np.float32)
    y = rng.random((M, d), dtype=np.float32)
    w = rng.random(N).astype(np.float32)
    xi = workloads.directions(P, d, seed=42)
    sigma = math.sqrt(d)
    sigma_ok = _plan(to_dev(x, dev), to_dev(w, dev), "gaussian", sigma, xi, "bf16", method="cheb")
    r_plain = sigma_ok.info()["radius"]
    x_out = x.copy()
    x_out[1] += 6.0  # row 1 is not among the sampled rows s * N / 4096
    plan = _plan(to_dev(x_out, dev), to_dev(w, dev), "gaussian", sigma, xi, "bf16", method="cheb")
    r_out = plan.info()["radius"]
    z_max = np.abs((x_out - x_out[[int(s * N / 4096) for s in range(4096)]].mean(axis=0)) @ xi.T).max()
    assert r_out >= z_max and r_out > 2.0 * r_plain
    for xx, pl in ((x, sigma_ok), (x_out, plan)):
        s = pl.sum(to_dev(y, dev))
        ref, _ = oracle.sliced_sum("gaussian", sigma, xx, y, w, xi)
        assert rel_inf(s, ref, w.sum()) <= 2e-3


@pytest.mark.parametrize("d,N,M,P", [(784, 5000, 1153, 512), (200, 4099, 700, 300)])
def test_bf16_fused_f32_targets_match_cast_route(d, N, M, P):
    """Aligned FP32 rows go straight into the CTA-pair kernels (P <= 512), which centre them
    and round them to BF16 in shared memory; rows whose stride is not a multiple of four
    take the separate centring cast and the single-CTA kernels.  Both routes hand the
    tensor core the same BF16 operands; they differ only in the FP32 order of the slice and
    moment sums, so the results agree to 1e-6 of sum |w|, also for plans built from the two
    layouts of the sources, and with the oracle within the BF16 tolerance."""
    dev = cuda_or_skip()
    from paper_2401_08260_gb300.slk import Plan
    rng = np.random.Generator(np.random.PCG64(51))
    x = rng.random((N, d), dtype=np.float32)
    y = rng.random((M, d), dtype=np.float32)
    w = rng.random(N).astype(np.float32)
    xi = workloads.directions(P, d, seed=52)
    sigma = math.sqrt(d)

    def strided(a):
        # same values, row stride d + 1 (not a multiple of four): the centring-cast route
        buf = torch.zeros((a.shape[0], d + 1), dtype=torch.float32, device=dev)
        buf[:, :d] = torch.from_numpy(a).to(dev)
        v = buf[:, :d]
        assert v.stride(0) == d + 1 and (d + 1) % 4 != 0
        return v

    p_a = Plan(to_dev(x, dev), to_dev(w, dev), "gaussian", sigma, P=P, precision="bf16", directions=xi,
               method="cheb")
    p_b = Plan(strided(x), to_dev(w, dev), "gaussian", sigma, P=P, precision="bf16", directions=xi, method="cheb")
    assert p_a.info()["radius"] == p_b.info()["radius"]
    s_direct = p_a.sum(to_dev(y, dev)).cpu().numpy()
    assert rel_inf(s_direct, p_a.sum(strided(y)).cpu().numpy(), w.sum()) <= 1e-6
    assert rel_inf(s_direct, p_b.sum(to_dev(y, dev)).cpu().numpy(), w.sum()) <= 1e-6
    assert rel_inf(p_b.sum(strided(y)).cpu().numpy(), p_b.sum(to_dev(y, dev)).cpu().numpy(), w.sum()) <= 1e-6
    ref, _ = oracle.sliced_sum("gaussian", sigma, x, y, w, xi)
    assert rel_inf(s_direct, ref, w.sum()) <= 2e-3
    # targets beyond the window are still reported on the direct route
    far = y.copy()
    far[M // 2] += 60.0
    from paper_2401_08260_gb300.slk import SlkError
    with pytest.raises(SlkError) as e:
        p_a.sum(to_dev(far, dev))
    assert e.value.status == 4


@pytest.mark.parametrize("d,N,M,P", [(784, 5000, 1153, 512), (200, 4099, 700, 300), (784, 2000, 100, 256),
                                     (96, 3000, 300, 64), (52, 257, 255, 129), (784, 30001, 513, 512)])
def test_pair_kernels_against_oracle_and_single_cta_route(d, N, M, P):
    """The CTA-pair kernels (one MMA of M = 256 over two CTAs, all P <= 512 slices of a
    256-point tile at once) over one or two 256-slice sub-tiles, ragged point tiles (fewer
    and more tiles than CTA pairs), K tails (d not a multiple of 64) and slices beyond P:
    within the BF16 tolerance of the oracle and within FP32 summation order of the
    single-CTA route, which strided rows (stride d + 1) select."""
    dev = cuda_or_skip()
    from paper_2401_08260_gb300.slk import Plan
    rng = np.random.Generator(np.random.PCG64(61))
    x = rng.random((N, d), dtype=np.float32)
    y = rng.random((M, d), dtype=np.float32)
    w = rng.random(N).astype(np.float32)
    xi = workloads.directions(P, d, seed=62)
    sigma = math.sqrt(d)

    def strided(a):
        buf = torch.zeros((a.shape[0], d + 1), dtype=torch.float32, device=dev)
        buf[:, :d] = torch.from_numpy(a).to(dev)
        return buf[:, :d]

    pair = Plan(to_dev(x, dev), to_dev(w, dev), "gaussian", sigma, P=P, precision="bf16", directions=xi,
                method="cheb")
    single = Plan(strided(x), to_dev(w, dev), "gaussian", sigma, P=P, precision="bf16", directions=xi,
                  method="cheb", radius=pair.info()["radius"])
    assert pair.info()["method"] == 3
    s_pair = pair.sum(to_dev(y, dev)).cpu().numpy()
    s_single = single.sum(strided(y)).cpu().numpy()
    assert rel_inf(s_pair, s_single, w.sum()) <= 1e-6
    idx = np.unique(np.concatenate([np.arange(min(M, 40)), np.arange(max(0, M - 40), M)]))
    ref, _ = oracle.sliced_sum("gaussian", sigma, x, y[idx], w, xi)
    assert rel_inf(s_pair[idx], ref, w.sum()) <= 2e-3
