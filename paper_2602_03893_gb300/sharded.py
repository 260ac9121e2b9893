"""The operator with its Gaussians partitioned across the ranks of a torch.distributed process
group (one GPU per rank): rank r owns the z-slab of lattice rows that gpair_shard_range gives
shard r of world_size.

The forward is a sum over Gaussians (Methods, Eq. single_forward summed over the set), so each
rank computes its slab's partial signals with gpair_forward_shard and one all-reduce (sum) of
the N_d x N_t signals completes y on every rank.  The residual is then the same everywhere, and
the amplitude gradient of a Gaussian needs only that residual, so gpair_adjoint_shard fills each
rank's rows of the gradient with no communication; the solver's elementwise update is local too.

The all-reduce runs on the device for a NCCL group; any other backend (gloo) reduces a host copy.
All arithmetic runs in libgpair's kernels; this module only partitions and communicates.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

from . import _lib


class ShardedOperator:
    """Forward and adjoint of a grid-implicit Gaussian set split into z-slabs over the group."""

    def __init__(self, gaussians: _lib.Gaussians, arr: _lib.SensorArray, group=None, local_forward=None):
        if gaussians.grid is None:
            raise ValueError("the partitioned operator needs grid-implicit Gaussians")
        self.g, self.arr, self.group = gaussians, arr, group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.z_begin, self.z_end = _lib.gpair_shard_range(gaussians.grid, self.rank, self.world)
        # the per-rank forward; a test may substitute another implementation of the same slab sum
        self._local_forward = local_forward or (
            lambda y: _lib.gpair_forward_shard(self.g, self.arr, self.rank, self.world, y))

    @property
    def rows(self) -> slice:
        """This rank's slice of the flattened amplitude / gradient arrays (x fastest)."""
        n = self.g.grid.nx * self.g.grid.ny
        return slice(self.z_begin * n, self.z_end * n)

    def _allreduce(self, y: torch.Tensor) -> None:
        if dist.get_backend(self.group) == "nccl" or not y.is_cuda:
            dist.all_reduce(y, op=dist.ReduceOp.SUM, group=self.group)
        else:
            h = y.cpu()
            dist.all_reduce(h, op=dist.ReduceOp.SUM, group=self.group)
            y.copy_(h)

    def forward(self, y: torch.Tensor) -> torch.Tensor:
        """y (N_d x N_t) = the full forward of the set, on every rank."""
        self._local_forward(y)
        self._allreduce(y)
        return y

    def adjoint(self, delta: torch.Tensor, gA: torch.Tensor) -> torch.Tensor:
        """gA[self.rows] = the amplitude gradient of this rank's Gaussians; other entries untouched."""
        return _lib.gpair_adjoint_shard(self.g, self.arr, self.rank, self.world, delta, gA)
