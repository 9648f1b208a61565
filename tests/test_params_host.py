"""Host-side Fourier parameter selection (no GPU): the period L and coefficient count N_c the
library chooses for a Gaussian plan, put into the truncated periodic Fourier sum with the
coefficients c_k = f^(k / L) / L of the closed-form transform (Lemma 2.6, the oracle's
evaluation), reproduce the oracle's 1-D counterpart f on the window |u| <= 2R that differences
of projections cover, within the model error the library certifies (truncation plus
periodisation plus the NFFT window's aliasing, so the bound holds with room)."""
import math

import numpy as np
import pytest

import oracle
from paper_2401_08260_gb300 import slk


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2401_08260_gb300 import build
    build.build()
    oracle.build()


@pytest.mark.parametrize("sigma,d,R,precision,tol", [
    (28.0, 784, 3.0, "f32", 0.0),     # the d = 784 benchmark's window (default FP32 target)
    (4.0, 16, 5.0, "f64", 1e-9),      # the d = 16 workload's scale, FP64 accuracy
    (math.sqrt(50.0), 50, 4.0, "f32", 1e-6),
])
def test_nfft_parameters_reproduce_f_within_the_certified_error(sigma, d, R, precision, tol):
    info = slk.fourier_params("gaussian", sigma, d, R, precision=precision, method="nfft", tol=tol)
    L, Nc, err = info["period"], info["n_coeff"], info["model_error"]
    assert info["method"] == 1 and Nc > 0 and L >= 2 * R and err > 0
    k = np.arange(1, Nc // 2)
    c0 = oracle.fhat_gauss(d, sigma, 0.0) / L
    ck = oracle.fhat_gauss(d, sigma, k / L) / L
    u = np.linspace(-2 * R, 2 * R, 401)
    phi = c0 + 2.0 * (ck[None, :] * np.cos(2 * np.pi * np.outer(u, k) / L)).sum(axis=1)
    exact = oracle.f("gaussian", d, sigma, np.abs(u))
    dev = np.abs(phi - exact).max()
    assert dev <= err
    # and the certificate is not vacuous: the realised deviation is within 10x of it
    # (0.46 to 0.81 of it at these three settings)
    assert dev >= err / 10


def test_chebyshev_is_chosen_for_the_benchmark_window():
    """At the d = 784 benchmark's window the automatic method is the Chebyshev form with a
    handful of terms (well inside the fused kernels' 8, 10, 12 or 16)."""
    info = slk.fourier_params("gaussian", 28.0, 784, 3.0, precision="bf16")
    assert info["method"] == 3 and 1 <= info["cheb_terms"] <= 16
    assert info["model_error"] <= 1e-5


@pytest.mark.parametrize("sigma,d,R,precision,tol", [
    (4.0, 16, 5.0, "f64", 0.0),       # the d = 16 workload: FP64 default target
    (28.0, 784, 3.0, "f32", 0.0),
])
def test_ndft_band_reproduces_f_within_the_certified_error(sigma, d, R, precision, tol):
    """The NDFT keeps the band k_lo <= |k| <= k_hi (it drops coefficients from both ends while
    the dropped mass stays within a share of the target); for d > 1 the k = 0 coefficient is
    f^(0) / L = 0 (f^ grows like omega^(d-1) at 0).  The band's cosine sum reproduces f on the
    window within the certified error."""
    info = slk.fourier_params("gaussian", sigma, d, R, precision=precision, method="ndft", tol=tol)
    L, k_lo, k_hi, err = info["period"], info["k_lo"], info["k_hi"], info["model_error"]
    assert info["method"] == 2 and 1 <= k_lo <= k_hi
    assert oracle.fhat_gauss(d, sigma, 0.0) == 0.0
    k = np.arange(k_lo, k_hi + 1)
    ck = oracle.fhat_gauss(d, sigma, k / L) / L
    u = np.linspace(-2 * R, 2 * R, 401)
    phi = 2.0 * (ck[None, :] * np.cos(2 * np.pi * np.outer(u, k) / L)).sum(axis=1)
    exact = oracle.f("gaussian", d, sigma, np.abs(u))
    dev = np.abs(phi - exact).max()
    assert dev <= err


@pytest.mark.parametrize("precision", ["bf16", "f32"])
def test_chebyshev_form_reproduces_f_within_the_certified_error(precision):
    """The Chebyshev form of the truncated Fourier sum (Jacobi-Anger expansion on the window
    [-R, R]): with the band and term count the host chooses, the separable approximation
    sum_{l,j<q} M_lj T_l(z/R) T_j(s/R), M_lj = 2 e_l e_j cos(pi (l - j) / 2) sum_k c_k
    J_l(w_k) J_j(w_k) (e_0 = 1, e_j = 2, w_k = 2 pi k R / L, Bessel values from scipy),
    reproduces the oracle's f(|z - s|) over the whole window square within the certified
    model error."""
    jv = pytest.importorskip("scipy.special").jv
    sigma, d = 28.0, 784
    info = slk.fourier_params("gaussian", sigma, d, 3.0, precision=precision)
    assert info["method"] == 3
    L, R, q = info["period"], info["radius"], info["cheb_terms"]
    k = np.arange(info["k_lo"], info["k_hi"] + 1)
    ck = oracle.fhat_gauss(d, sigma, k / L) / L
    om = 2 * np.pi * k * R / L
    ll = np.arange(q)
    e = np.where(ll == 0, 1.0, 2.0)
    J = jv(ll[:, None], om[None, :])
    M = 2 * e[:, None] * e[None, :] * np.cos(np.pi * (ll[:, None] - ll[None, :]) / 2) * ((J * ck) @ J.T)
    u = np.linspace(-1.0, 1.0, 121)
    T = np.cos(np.outer(np.arccos(u), ll))
    approx = T @ M @ T.T
    exact = oracle.f("gaussian", d, sigma, np.abs(R * (u[:, None] - u[None, :])))
    dev = np.abs(approx - exact).max()
    assert dev <= info["model_error"]
    # one term fewer is visibly worse: the certified count is not padded generously
    approx_short = T[:, :-1] @ M[:-1, :-1] @ T[:, :-1].T
    assert np.abs(approx_short - exact).max() > dev
