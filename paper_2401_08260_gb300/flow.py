"""MMD particle flows driven by the sliced kernel sums.

The squared maximum mean discrepancy between particles y_1..y_M (weights 1/M) and a fixed
sample x_1..x_N (weights v_n, sum 1) for a radial kernel K = F(|.|) is

    MMD^2(y) = 1/M^2 sum_{m,m'} K(y_m, y_m') - 2/M sum_{m,n} v_n K(y_m, x_n) + const,

and its gradient flow moves every particle along

    -M/2 grad_{y_m} MMD^2 = sum_n v_n grad K(y_m, x_n) - 1/M sum_{m'} grad K(y_m, y_m')

(attraction to the sample minus repulsion between particles; the m' = m term vanishes for a
radial kernel).  With the negative distance kernel K = -|.|, MMD^2 is the energy distance.
Both sums are y-gradients of kernel sums with the particles as targets: the first against a
plan on x built once, the second against a plan on the current particles, rebuilt every step
with fresh directions (each step's slicing noise is independent).  Every sum runs in the
library (`slk.Plan.grad` / `slk.Plan.sum`); this module only keeps the particles and the plans.
"""
from __future__ import annotations

from . import slk


class MMDFlow:
    """Explicit-Euler MMD flow of particles towards a fixed weighted sample x.

    x, v: the target sample (N x d) and its weights (default 1/N), torch tensors on the GPU
    or host arrays; kernel, param, P, precision, radius: as for `slk.Plan` (a radius is needed
    for the Fourier kernels once the particles leave the sample's projected range)."""

    def __init__(self, x, kernel: str = "negdist", param: float = 0.0, P: int = 256, precision: str = "f32",
                 v=None, seed: int = 0, radius: float = 0.0):
        import torch
        self.kernel, self.param, self.P, self.precision, self.radius = kernel, param, P, precision, radius
        self.seed = seed
        n = x.shape[0]
        if v is None:
            v = torch.full((n,), 1.0 / n, dtype=x.dtype, device=x.device) if hasattr(x, "device") else None
            if v is None:
                import numpy as np
                v = np.full(n, 1.0 / n, dtype=x.dtype)
        self.x, self.v = x, v
        self.plan_x = slk.Plan(x, v, kernel, param, P=P, precision=precision, seed=seed, radius=radius)
        self.steps_done = 0

    def _plan_y(self, y, seed):
        import torch
        m = y.shape[0]
        wy = torch.full((m,), 1.0 / m, dtype=y.dtype, device=y.device)
        return slk.Plan(y, wy, self.kernel, self.param, P=self.P, precision=self.precision, seed=seed,
                        radius=self.radius)

    def velocity(self, y, seed: int | None = None):
        """sum_n v_n grad K(y_m, x_n) - 1/M sum_m' grad K(y_m, y_m') for every particle (M x d)."""
        s = self.seed + 1 + self.steps_done if seed is None else seed
        plan_y = self._plan_y(y, s)
        try:
            attract = self.plan_x.grad(y)
            repel = plan_y.grad(y)
        finally:
            plan_y.close()
        return attract - repel

    def step(self, y, tau: float):
        """One explicit Euler step y <- y + tau * velocity(y); returns the new particles."""
        vel = self.velocity(y)
        self.steps_done += 1
        return y + tau * vel

    def mmd2(self, y, seed: int | None = None) -> float:
        """Sliced estimate of MMD^2(y) (without the constant x-x term)."""
        s = self.seed + 1 + self.steps_done if seed is None else seed
        plan_y = self._plan_y(y, s)
        try:
            yy = plan_y.sum(y)
            yx = self.plan_x.sum(y)
        finally:
            plan_y.close()
        m = y.shape[0]
        return float(yy.sum() / m - 2.0 * yx.sum() / m)

    def close(self):
        self.plan_x.close()
