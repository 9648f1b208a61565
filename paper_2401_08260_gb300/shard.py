"""Slice sharding: one sliced sum split over the ranks of a process group.

The sliced sum of Algorithm 1 is an average over P directions of independent one-dimensional
sums, s_m = (1/P) sum_p t_{p,m}.  Split the slice indices into disjoint ranges [p0_r, p1_r), one
per rank; rank r plans only its P_r = p1_r - p0_r slices (the library draws rows p0_r .. p1_r - 1
of the seed's direction sequence, or takes those rows of given directions), so its plan returns
the mean over its own slices, s_r.  Then

    s = sum_r (P_r / P) s_r,

one all-reduce(sum) of M values (or of the M x d gradient) after each rank has scaled its part.
x, w and y are replicated on every rank; nothing else is exchanged.  The same split serves
slice batching on one GPU (Sec. 5.4, remark on memory and batching), where the parts run one
after another instead of side by side (see `slk.kernel_sum(..., slice_batch=B)`).

Every sum runs in the library (`slk.Plan`); this module holds the split and the collective.
"""
from __future__ import annotations

from typing import Optional, Tuple


def slice_range(P: int, parts: int, index: int) -> Tuple[int, int]:
    """Slices [p0, p1) of part `index` when P slices are split into `parts` contiguous ranges
    whose sizes differ by at most one (parts > P leaves some ranges empty)."""
    if P < 1 or parts < 1 or not 0 <= index < parts:
        raise ValueError("need P >= 1, parts >= 1 and 0 <= index < parts")
    return index * P // parts, (index + 1) * P // parts


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


class SliceShard:
    """This rank's part of a P-slice sum and the combination of the parts.

    rank, world default to the initialised torch.distributed group (else 0 of 1)."""

    def __init__(self, P: int, rank: Optional[int] = None, world: Optional[int] = None, group=None):
        dist = _dist()
        if world is None:
            world = dist.get_world_size(group) if dist else 1
        if rank is None:
            rank = dist.get_rank(group) if dist else 0
        self.P, self.rank, self.world, self.group = int(P), int(rank), int(world), group
        self.p0, self.p1 = slice_range(self.P, self.world, self.rank)

    @property
    def count(self) -> int:
        """P_r: the number of slices this rank owns (0 when P < world for some ranks)."""
        return self.p1 - self.p0

    @property
    def weight(self) -> float:
        """P_r / P: this rank's share of the average over all slices."""
        return self.count / self.P

    def combine(self, local):
        """sum over ranks of (P_r / P) * local_r: `local` is this rank's mean over its own slices
        (a torch tensor; zeros on a rank without slices).  One all-reduce(sum) when world > 1;
        a host tensor is staged through the current GPU when the group's backend is NCCL."""
        t = local * self.weight
        if self.world == 1:
            return t
        dist = _dist()
        if dist is None:
            raise RuntimeError("a sharded sum over several ranks needs an initialised process group")
        stage = not t.is_cuda and dist.get_backend(self.group) == "nccl"
        buf = t.cuda() if stage else t
        dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=self.group)
        return buf.to(local.device) if stage else buf


class ShardedPlan:
    """A `slk.Plan` over this rank's slices of a P-slice sum, with sums combined across ranks.

    Arguments as for `slk.Plan` (directions: all P rows; this rank takes its own), plus rank,
    world and group of the split.  Every rank must call `sum` / `grad` with the same targets."""

    def __init__(self, x, w, kernel: str, param: float = 0.0, P: int = 256, precision: str = "f32",
                 seed: int = 0, directions=None, slice_offset: int = 0, rank: Optional[int] = None,
                 world: Optional[int] = None, group=None, **plan_kw):
        from . import slk
        self.shard = SliceShard(P, rank, world, group)
        self.P, self.d, self.precision = int(P), int(x.shape[1]), precision
        self.plan = None
        if self.shard.count:
            p0, p1 = self.shard.p0, self.shard.p1
            rows = directions[p0:p1] if directions is not None else None
            self.plan = slk.Plan(x, w, kernel, param, P=self.shard.count, precision=precision, seed=seed,
                                 directions=rows, slice_offset=slice_offset + p0, **plan_kw)

    def _zeros(self, y, shape):
        import torch
        dtype = torch.float64 if self.precision == "f64" else torch.float32
        dev = y.device if isinstance(y, torch.Tensor) else "cpu"
        return torch.zeros(shape, dtype=dtype, device=dev)

    @staticmethod
    def _tensor(a):
        import torch
        return a if isinstance(a, torch.Tensor) else torch.from_numpy(a)

    def sum(self, y):
        """s_m over all P slices (every rank receives the same values)."""
        local = self._tensor(self.plan.sum(y)) if self.plan else self._zeros(y, (y.shape[0],))
        return self.shard.combine(local)

    def grad(self, y, gs=None):
        """Gradient of sum_m gs_m s_m with respect to y over all P slices (M x d)."""
        local = self._tensor(self.plan.grad(y, gs)) if self.plan else self._zeros(y, (y.shape[0], self.d))
        return self.shard.combine(local)

    def directions(self):
        """This rank's rows of the directions (P_r x d, FP64), or None on a rank without slices."""
        return self.plan.directions() if self.plan else None

    def close(self):
        if self.plan is not None:
            self.plan.close()
            self.plan = None
