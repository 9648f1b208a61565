"""FP64 CPU oracle for the sliced fast kernel summation.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library (``paper_2401_08260_gb300``)
and never imports it.

The oracle computes what the paper defines, plainly and slowly:

* ``direct_sum``  -- the d-dimensional kernel sum s_m = sum_n w_n F(|x_n - y_m|)
  (problem statement, Section 3).
* ``sliced_sum``  -- Algorithm 1 with *exact* 1-D sums on given directions:
  (1/P) sum_p sum_n w_n f(|<xi_p, y_m - x_n>|), f the 1-D counterpart of
  Table 1 (Theorem 2.3); optionally the y-gradient
  (1/P) sum_p xi_p sum_n w_n f'(|d|) sign(d), sign(0) = 0.
* ``f``, ``F``, ``cd``, ``fhat_gauss`` -- the kernel functions of Table 1,
  Section 3.2 and Lemma 2.6.
* ``f_gauss_fourier`` -- the Gaussian counterpart by Fourier inversion of
  Lemma 2.6 (an independent second evaluator).
* ``negdist_alg2`` -- Algorithm 2 plus the permutation step of Section 3.2,
  used to check that the sorting route is exact.
* ``rff_features``, ``rff_sum`` -- the random Fourier feature estimators RFF-1 and
  RFF-2 of Section 4.3 (the paper's comparison system), on given features.

Projections <xi_p, x_n> are a matrix product (numpy FP64); everything else is
in ``slk_oracle.c`` (FP64, OpenMP over independent outputs).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

GAUSSIAN, LAPLACIAN, NEGDIST, MATERN32 = 0, 1, 2, 3
KERNELS = {"gaussian": GAUSSIAN, "laplacian": LAPLACIAN, "negdist": NEGDIST, "matern32": MATERN32}

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "slk_oracle.c")
_SO = os.path.join(_HERE, "liboracle_slk.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C part of the oracle with gcc (portable flags only)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-D_GNU_SOURCE",
               "-o", _SO + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_SO + ".tmp", _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            D, I, L, P = ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
            lib.orc_cd.restype, lib.orc_cd.argtypes = D, [I]
            lib.orc_F.restype, lib.orc_F.argtypes = D, [I, D, D]
            lib.orc_f_vec.restype, lib.orc_f_vec.argtypes = D, [I, I, D, P, L, P, P]
            lib.orc_fhat_gauss.restype, lib.orc_fhat_gauss.argtypes = D, [I, D, D]
            lib.orc_direct_sum.restype = None
            lib.orc_direct_sum.argtypes = [I, D, I, P, L, P, L, P, P, P]
            lib.orc_sliced_accumulate.restype = D
            lib.orc_sliced_accumulate.argtypes = [I, I, D, P, L, P, P, L, I, P, P, P, P]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _kid(kernel) -> int:
    return KERNELS[kernel] if isinstance(kernel, str) else int(kernel)


def cd(d: int) -> float:
    """c_d = sqrt(pi) Gamma((d+1)/2) / Gamma(d/2) (Section 3.2)."""
    return _load().orc_cd(int(d))


def F(kernel, param: float, r) -> np.ndarray:
    """Radial basis function F(r) of Table 1 (param = sigma, the paper's alpha, or the
    Matern length scale beta)."""
    r = np.asarray(r, dtype=np.float64)
    lib = _load()
    k = _kid(kernel)
    return np.vectorize(lambda v: lib.orc_F(k, float(param), float(v)))(r)


def f(kernel, d: int, param: float, x, deriv: bool = False, return_err: bool = False):
    """1-D counterpart f(|x|) of Table 1 by its power series (Theorem 2.3).

    With ``deriv`` also returns f'(|x|); with ``return_err`` also the largest
    rounding bound (largest series term x #terms x eps)."""
    x = _c64(x)
    flat = x.reshape(-1)
    out = np.empty_like(flat)
    dout = np.empty_like(flat)
    err = _load().orc_f_vec(_kid(kernel), int(d), float(param), _ptr(flat), flat.size, _ptr(out), _ptr(dout))
    res = [out.reshape(x.shape)]
    if deriv:
        res.append(dout.reshape(x.shape))
    if return_err:
        res.append(err)
    return res[0] if len(res) == 1 else tuple(res)


def fhat_gauss(d: int, sigma: float, omega) -> np.ndarray:
    """Lemma 2.6: Fourier transform of the Gaussian counterpart (log-space)."""
    lib = _load()
    return np.vectorize(lambda w: lib.orc_fhat_gauss(int(d), float(sigma), float(w)))(
        np.asarray(omega, dtype=np.float64))


def f_gauss_fourier(d: int, sigma: float, x, panels: int = 400, order: int = 16) -> np.ndarray:
    """Gaussian counterpart by Fourier inversion of Lemma 2.6:
    f(x) = 2 int_0^inf fhat(w) cos(2 pi w x) dw, composite Gauss-Legendre over the
    band where fhat exceeds e^-45 of its peak."""
    x = _c64(x)
    # fhat ~ exp(-u) u^((d-1)/2), u = 2 pi^2 sigma^2 w^2; peak at u = (d-1)/2
    a = 0.5 * (d - 1)
    umax = a + 45.0 + 12.0 * math.sqrt(a + 1.0) + 10.0
    umin = max(0.0, a - 12.0 * math.sqrt(a + 1.0) - 10.0) if d > 1 else 0.0
    wlo = math.sqrt(umin / (2.0 * math.pi ** 2 * sigma ** 2))
    whi = math.sqrt(umax / (2.0 * math.pi ** 2 * sigma ** 2))
    t, wt = np.polynomial.legendre.leggauss(order)
    edges = np.linspace(wlo, whi, panels + 1)
    mid = 0.5 * (edges[1:] + edges[:-1])
    half = 0.5 * (edges[1:] - edges[:-1])
    nodes = (mid[:, None] + half[:, None] * t[None, :]).reshape(-1)
    weights = (half[:, None] * wt[None, :]).reshape(-1)
    fh = fhat_gauss(d, sigma, nodes)
    out = 2.0 * np.cos(2.0 * math.pi * np.multiply.outer(x, nodes)) @ (weights * fh)
    return out


def direct_sum(kernel, param: float, X, Y, w, grad: bool = False):
    """O-direct: s_m = sum_n w_n F(|x_n - y_m|), FP64, Neumaier-compensated."""
    X, Y, w = _c64(X), _c64(Y), _c64(w)
    N, d = X.shape
    M = Y.shape[0]
    s = np.zeros(M)
    g = np.zeros((M, d)) if grad else None
    _load().orc_direct_sum(_kid(kernel), float(param), int(d), _ptr(X), N, _ptr(Y), M, _ptr(w), _ptr(s),
                           _ptr(g) if grad else None)
    return (s, g) if grad else s


def project(X, Xi) -> np.ndarray:
    """z[n, p] = <xi_p, x_n> in FP64 (a plain matrix product)."""
    return _c64(X) @ _c64(Xi).T


def sliced_sum(kernel, param: float, X, Y, w, Xi, grad: bool = False, chunk: int = 1 << 16,
               per_slice: bool = False):
    """O-sliced: (1/P) sum_p sum_n w_n f(|<xi_p, y_m - x_n>|) with exact 1-D sums.

    Xi is P x d (row p is the direction xi_p).  Returns s (M,), and with ``grad``
    also the y-gradient (M x d); with ``per_slice`` also the per-slice sums
    T (M x P) and gradient sums G (M x P).  ``info['err']`` holds the largest
    rounding bound of the f evaluations."""
    X, Y, w, Xi = _c64(X), _c64(Y), _c64(w), _c64(Xi)
    N, d = X.shape
    M = Y.shape[0]
    P = Xi.shape[0]
    kid = _kid(kernel)
    Zy = np.ascontiguousarray(project(Y, Xi))
    S = np.zeros((M, P))
    SC = np.zeros((M, P))
    G = np.zeros((M, P)) if grad else None
    GC = np.zeros((M, P)) if grad else None
    lib = _load()
    emax = 0.0
    for n0 in range(0, N, chunk):
        n1 = min(N, n0 + chunk)
        Zx = np.ascontiguousarray(project(X[n0:n1], Xi))
        wc = np.ascontiguousarray(w[n0:n1])
        e = lib.orc_sliced_accumulate(kid, int(d), float(param), _ptr(Zx), n1 - n0, _ptr(wc), _ptr(Zy), M, P,
                                      _ptr(S), _ptr(SC), _ptr(G) if grad else None, _ptr(GC) if grad else None)
        emax = max(emax, e)
    T = S + SC
    s = np.array([math.fsum(row) for row in T]) / P
    out = [s]
    if grad:
        Gt = G + GC
        out.append((Gt @ Xi) / P)
    if per_slice:
        out.append(T)
        if grad:
            out.append(Gt)
    out.append({"err": emax})
    return tuple(out)


def negdist_alg2(zx, w, zy, cdv: float) -> np.ndarray:
    """Algorithm 2 of Section 3.2 plus the permutation of the general case.

    z = (y_1..y_M, x_1..x_N), v = (0..0, w_1..w_N); sort z by a permutation
    sigma; a = cumsum(c_d v_sigma); a~_i = a_i (z_{i+1} - z_i) with a~_{N+M} = 0;
    b = cumsum(a~) with b_0 = 0;  t_i = b_{N+M-1} - 2 b_{i-1} - a_{N+M} (z_{N+M} - z_i);
    then t is scattered back through sigma.  Returns t for the M targets."""
    zx, w, zy = _c64(zx), _c64(w), _c64(zy)
    M = zy.size
    z = np.concatenate([zy, zx])
    v = np.concatenate([np.zeros(M), w])
    order = np.argsort(z, kind="stable")
    zs = z[order]
    a = np.cumsum(cdv * v[order])
    L = zs.size
    at = np.zeros(L)
    at[:-1] = a[:-1] * (zs[1:] - zs[:-1])
    b = np.concatenate([[0.0], np.cumsum(at)])  # b[i] = b_i, 1-based, b_0 = 0
    i = np.arange(1, L + 1)
    t_sorted = b[L - 1] - 2.0 * b[i - 1] - a[L - 1] * (zs[L - 1] - zs)
    t = np.empty(L)
    t[order] = t_sorted
    return t[:M]


def rff_features(kernel, param: float, d: int, D: int, rng: np.random.Generator):
    """Random Fourier features of Section 4.3: D samples v_p of the spectral measure mu of
    the kernel (K(x, y) = E_{v ~ mu} cos<x - y, v>, Bochner's theorem) and D phases
    b_p ~ U[0, 2 pi).  Gaussian F(r) = exp(-r^2 / (2 sigma^2)): mu = N(0, sigma^-2 I);
    Laplacian F(r) = exp(-alpha r): mu = the multivariate Cauchy law with scale alpha,
    sampled as alpha g / |h| with g ~ N(0, I_d), h ~ N(0, 1).  Returns (V (D x d), b (D,))."""
    k = _kid(kernel)
    g = rng.standard_normal((D, d))
    if k == GAUSSIAN:
        V = g / float(param)
    elif k == LAPLACIAN:
        h = rng.standard_normal(D)
        V = float(param) * g / np.abs(h)[:, None]
    else:
        raise ValueError("random Fourier features need a positive definite kernel (Gaussian or Laplacian)")
    b = 2.0 * math.pi * rng.random(D)
    return V, b


def rff_sum(X, Y, w, V, b, variant: int) -> np.ndarray:
    """Random Fourier feature estimate of s_m = sum_n w_n K(x_n, y_m) (Section 4.3), in FP64.

    variant 1 (RFF-1):  s_m = (2 / D) sum_p cos(<y_m, v_p> + b_p) sum_n w_n cos(<x_n, v_p> + b_p)
    variant 2 (RFF-2):  s_m = (1 / D) sum_p [cos<y_m, v_p> C_p + sin<y_m, v_p> S_p],
                        C_p = sum_n w_n cos<x_n, v_p>,  S_p = sum_n w_n sin<x_n, v_p>.
    The printed equations omit the 1 / D of the sample average of the expectations they
    subsample; it is restored here."""
    X, Y, w, V, b = _c64(X), _c64(Y), _c64(w), _c64(V), _c64(b)
    D = V.shape[0]
    Zx = X @ V.T  # N x D
    Zy = Y @ V.T  # M x D
    if variant == 1:
        C = np.cos(Zx + b[None, :]).T @ w
        return (2.0 / D) * (np.cos(Zy + b[None, :]) @ C)
    if variant == 2:
        C = np.cos(Zx).T @ w
        S = np.sin(Zx).T @ w
        return (np.cos(Zy) @ C + np.sin(Zy) @ S) / D
    raise ValueError("variant is 1 or 2")


def sampled_targets(M: int, count: int, seed: int = 5) -> np.ndarray:
    """Seeded subsample of `count` target indices (sorted; includes the last index
    when count >= 2, to cover the ragged tail)."""
    if count >= M:
        return np.arange(M)
    rng = np.random.Generator(np.random.PCG64(seed))
    if count < 2:
        return np.sort(rng.choice(M, size=count, replace=False))
    idx = rng.choice(M - 1, size=count - 1, replace=False)
    return np.sort(np.concatenate([idx, [M - 1]]))
