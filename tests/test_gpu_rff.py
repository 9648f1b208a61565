"""Random Fourier features on the GPU (Section 4.3, the comparison system): RFF-1 and RFF-2
through the C ABI against the oracle's estimators on the same features, the library's own
feature draw against the spectral measures, and the comparison the paper draws (slicing
beats RFF on the Laplacian kernel at equal budget)."""
import math

import numpy as np
import pytest

import oracle
from paper_2401_08260_gb300 import workloads
from tests._util import cuda_or_skip, rel_inf, to_dev, torch

pytestmark = pytest.mark.gpu


def _data(N, M, d, seed, scale=0.1):
    rng = np.random.Generator(np.random.PCG64(seed))
    return scale * rng.standard_normal((N, d)), scale * rng.standard_normal((M, d)), rng.random(N)


@pytest.mark.parametrize("kernel,param", [("gaussian", math.sqrt(5.0)), ("laplacian", 0.25)])
@pytest.mark.parametrize("variant", [1, 2])
def test_rff_fp64_matches_oracle(kernel, param, variant):
    """FP64: the library's RFF estimate equals the oracle's on the same features (ragged
    feature and point counts)."""
    dev = cuda_or_skip()
    from paper_2401_08260_gb300 import slk
    d, N, M, D = 100, 3001, 517, 333
    X, Y, w = _data(N, M, d, 11)
    V, b = oracle.rff_features(kernel, param, d, D, np.random.Generator(np.random.PCG64(12)))
    feat = np.concatenate([V, b[:, None]], axis=1)
    s = slk.rff_sum(to_dev(X, dev), to_dev(w, dev), to_dev(Y, dev), kernel, param, D, variant=variant,
                    precision="f64", features=feat)
    ref = oracle.rff_sum(X, Y, w, V, b, variant)
    assert rel_inf(s, ref, w.sum()) <= 1e-12


@pytest.mark.parametrize("variant", [1, 2])
def test_rff_fp32_gaussian_matches_oracle(variant):
    """FP32 (Gaussian features, arguments of order one): within 1e-5 of sum|w|, with host and
    device inputs giving the same result."""
    dev = cuda_or_skip()
    from paper_2401_08260_gb300 import slk
    d, N, M, D = 784, 4000, 300, 512
    rng = np.random.Generator(np.random.PCG64(13))
    X = rng.random((N, d), dtype=np.float32)
    Y = rng.random((M, d), dtype=np.float32)
    w = np.full(N, 1.0 / N, dtype=np.float32)
    sigma = math.sqrt(d)
    V, b = oracle.rff_features("gaussian", sigma, d, D, np.random.Generator(np.random.PCG64(14)))
    feat = np.concatenate([V, b[:, None]], axis=1)
    s_dev = slk.rff_sum(to_dev(X, dev), to_dev(w, dev), to_dev(Y, dev), "gaussian", sigma, D, variant=variant,
                        precision="f32", features=feat).cpu().numpy()
    s_host = slk.rff_sum(X, w, Y, "gaussian", sigma, D, variant=variant, precision="f32", features=feat)
    np.testing.assert_array_equal(s_dev, s_host)
    ref = oracle.rff_sum(X, Y, w, V, b, variant)
    assert rel_inf(s_dev, ref, w.sum()) <= 1e-5


@pytest.mark.parametrize("kernel,param", [("gaussian", 2.0), ("laplacian", 0.5)])
def test_library_feature_draw(kernel, param):
    """The library's features follow the spectral measure: the sample mean of cos<u, v_p>
    reproduces F(|u|) within 5 / sqrt(D) (d = 3), the phases are uniform on [0, 2 pi), and
    the library's RFF-2 with its own draw equals the oracle on the exported features."""
    dev = cuda_or_skip()
    from paper_2401_08260_gb300 import slk
    d, D = 3, 60000
    feat = slk.rff_features(kernel, param, d, D, seed=21)
    V, b = feat[:, :d], feat[:, d]
    assert b.min() >= 0.0 and b.max() < 2 * math.pi and abs(b.mean() - math.pi) < 0.05
    rng = np.random.Generator(np.random.PCG64(22))
    for r in (0.0, 0.5, 1.5):
        u = rng.standard_normal(d)
        u *= r / max(np.linalg.norm(u), 1e-300)
        ref = math.exp(-r * r / (2 * param * param)) if kernel == "gaussian" else math.exp(-param * r)
        assert abs(np.mean(np.cos(V @ u)) - ref) <= 5.0 / math.sqrt(D)
    X, Y, w = _data(500, 40, d, 23, scale=1.0)
    s = slk.rff_sum(to_dev(X, dev), to_dev(w, dev), to_dev(Y, dev), kernel, param, 256, variant=2, precision="f64",
                    seed=24)
    feat256 = slk.rff_features(kernel, param, d, 256, seed=24)
    ref = oracle.rff_sum(X, Y, w, feat256[:, :d], feat256[:, d], 2)
    assert rel_inf(s, ref, w.sum()) <= 1e-12


def test_slicing_beats_rff_on_the_laplacian():
    """Section 4.3: at the same budget (P = D = 1000... here P = 500, D = 1000 as the paper's
    D = 2P for the Laplacian) slicing's per-summand l1 error against the direct sum is below
    both RFF variants' for the Laplacian kernel (alpha = 0.25, d = 1000, x, y ~ N(0, 0.1^2 I))."""
    dev = cuda_or_skip()
    from paper_2401_08260_gb300 import slk
    from paper_2401_08260_gb300.slk import Plan
    d, N, M, P, D, alpha = 1000, 4000, 200, 500, 1000, 0.25
    X, Y, w = _data(N, M, d, 31)
    ref = oracle.direct_sum("laplacian", alpha, X, Y, w)

    def l1(s):
        s = s.cpu().numpy() if hasattr(s, "cpu") else s
        return np.sum(np.abs(s - ref)) / (M * np.sum(np.abs(w)))

    xs, ws, ys = to_dev(X, dev), to_dev(w, dev), to_dev(Y, dev)
    plan = Plan(xs, ws, "laplacian", alpha, P=P, precision="f64", directions=workloads.directions(P, d, seed=32))
    e_slice = l1(plan.sum(ys))
    e_rff = [l1(slk.rff_sum(xs, ws, ys, "laplacian", alpha, D, variant=v, precision="f64", seed=33)) for v in (1, 2)]
    assert e_slice < min(e_rff), (e_slice, e_rff)
