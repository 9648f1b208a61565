"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random numbers (numpy PCG64, FP64 then cast); it holds
none of the summation method's arithmetic.  Both the CUDA path and the CPU
oracle consume its output, so it is the one piece of code they share.

Seeds: directions 0, x 1, y 2, w 3, mixture means 4 (target subsample 5 is in
the oracle's sampler).  Directions are drawn uniformly on S^{d-1} as
normalised standard Gaussian vectors (Algorithm 1, first step) and are passed
to the library as an input.

Named workloads (sizes at full scale):

* ``gauss_d16``      Gaussian, sigma = sqrt(d) = 4, N = M = 1000, d = 16, x, y ~ N(0, I),
                     w ~ U[0,1], P = 64, 64 Fourier coefficients, FP64 NDFT.
* ``gauss_d784``     Gaussian, sigma = 28, N = M = 1e6, d = 784, x, y ~ U[0,1]^d (FP32,
                     image-shaped), w = 1/N, P = 512, 256 Fourier coefficients,
                     BF16 projection.
* ``negdist_d3072``  negative distance, N = M = 2e5, d = 3072, x ~ N(0, I),
                     y ~ N(0.5 * 1, I), w ~ U[0,1], P = 1000, FP32 (tensor-core
                     projection with FP32-level accuracy), exact prefix sums
                     (double-float within chunks, FP64 per chunk and bucket).
* ``laplace_d50``    Laplacian exp(-alpha r) with alpha = 1/sqrt(50) (length scale
                     sqrt(d)), 10-component Gaussian mixture (means ~ N(0, 4I),
                     unit covariance, equal weights) for x and y, d = 50,
                     N = M = 1e7, P = 128, FP32-accurate (FP16 hi/lo tensor-core) projection.
* ``paper_sec4``     the paper's Section 4.1 setup: x, y ~ N(0, 0.1^2 I), w ~ U[0,1].
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_DIRECTIONS, SEED_X, SEED_Y, SEED_W, SEED_MEANS = 0, 1, 2, 3, 4


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


@dataclass
class Workload:
    name: str
    kernel: str          # "gaussian" | "laplacian" | "negdist"
    param: float         # sigma (Gaussian) or the paper's alpha (Laplacian, F = exp(-alpha r))
    d: int
    N: int
    M: int
    P: int
    n_coeff: int         # Fourier coefficients (0 = automatic)
    precision: str       # "f64" | "f32" | "bf16" | "f16x3"
    method: str          # "auto" | "nfft" | "ndft"
    dtype: type          # storage type of x, y, w
    x: np.ndarray = field(repr=False, default=None)
    y: np.ndarray = field(repr=False, default=None)
    w: np.ndarray = field(repr=False, default=None)
    xi: np.ndarray = field(repr=False, default=None)   # P x d, FP64, unit rows

    @property
    def slice_points(self) -> int:
        return (self.N + self.M) * self.P


SPECS = {
    "gauss_d16": dict(kernel="gaussian", d=16, N=1000, M=1000, P=64, n_coeff=64, precision="f64",
                      method="ndft", dtype=np.float64, dist="normal"),
    "gauss_d784": dict(kernel="gaussian", d=784, N=10 ** 6, M=10 ** 6, P=512, n_coeff=256, precision="bf16",
                       method="auto", dtype=np.float32, dist="cube"),
    "negdist_d3072": dict(kernel="negdist", d=3072, N=2 * 10 ** 5, M=2 * 10 ** 5, P=1000, n_coeff=0,
                          precision="f16x3", method="auto", dtype=np.float32, dist="normal_shift"),
    "laplace_d50": dict(kernel="laplacian", d=50, N=10 ** 7, M=10 ** 7, P=128, n_coeff=0, precision="f16x3",
                        method="auto", dtype=np.float32, dist="mixture"),
    "paper_sec4": dict(kernel="gaussian", d=50, N=10 ** 4, M=10 ** 4, P=256, n_coeff=0, precision="f32",
                       method="auto", dtype=np.float32, dist="paper"),
}


def default_param(kernel: str, d: int) -> float:
    """sigma = sqrt(d) for the Gaussian; alpha = 1/sqrt(d) for the Laplacian."""
    if kernel == "gaussian":
        return math.sqrt(d)
    if kernel == "laplacian":
        return 1.0 / math.sqrt(d)
    return 0.0


def directions(P: int, d: int, seed: int = SEED_DIRECTIONS) -> np.ndarray:
    """P directions uniform on S^{d-1}: normalised N(0, I_d) draws, FP64 (P x d)."""
    g = _rng(seed).standard_normal((P, d))
    return g / np.linalg.norm(g, axis=1, keepdims=True)


def _points(dist: str, n: int, d: int, seed: int, dtype, is_y: bool) -> np.ndarray:
    rng = _rng(seed)
    if dist == "normal":
        return rng.standard_normal((n, d), dtype=np.float64).astype(dtype)
    if dist == "normal_shift":
        a = rng.standard_normal((n, d), dtype=np.float32 if dtype == np.float32 else np.float64)
        if is_y:
            a += 0.5
        return a.astype(dtype, copy=False)
    if dist == "cube":
        return rng.random((n, d), dtype=np.float32 if dtype == np.float32 else np.float64).astype(dtype, copy=False)
    if dist == "paper":
        return (0.1 * rng.standard_normal((n, d))).astype(dtype)
    if dist == "mixture":
        means = 2.0 * _rng(SEED_MEANS).standard_normal((10, d))
        comp = rng.integers(0, 10, size=n)
        a = rng.standard_normal((n, d), dtype=np.float32)
        a += means[comp].astype(np.float32)
        return a.astype(dtype, copy=False)
    raise ValueError(dist)


def _weights(name: str, n: int, dtype) -> np.ndarray:
    if name == "gauss_d784":
        return np.full(n, 1.0 / n, dtype=dtype)
    return _rng(SEED_W).random(n).astype(dtype)


def make(name: str, N: int | None = None, M: int | None = None, P: int | None = None, d: int | None = None,
         param: float | None = None, dtype=None, with_data: bool = True) -> Workload:
    """Build a named workload, optionally at a reduced size (same distributions)."""
    s = dict(SPECS[name])
    d = d or s["d"]
    N = N or s["N"]
    M = M or s["M"]
    P = P or s["P"]
    dtype = dtype or s["dtype"]
    if param is None:
        param = 1.0 if (name == "paper_sec4" and s["kernel"] == "gaussian") else default_param(s["kernel"], d)
    wl = Workload(name=name, kernel=s["kernel"], param=param, d=d, N=N, M=M, P=P, n_coeff=s["n_coeff"],
                  precision=s["precision"], method=s["method"], dtype=dtype)
    if with_data:
        wl.x = _points(s["dist"], N, d, SEED_X, dtype, False)
        wl.y = _points(s["dist"], M, d, SEED_Y, dtype, True)
        wl.w = _weights(name, N, dtype)
        wl.xi = directions(P, d)
    return wl
