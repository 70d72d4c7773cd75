"""Bookkeeping of runs with one process per GPU.

The solve does not shard across GPUs here: each rank solves an independent
replica of the system (its own source), so the only cross-rank operations are
the bench's barrier and the max / sum of its scalars - none on the data path.
Works with NCCL (tensors on the rank's GPU) and with gloo (tensors on the CPU).
"""
from __future__ import annotations

import os


def dist_env():
    """(world size, rank, local rank) from the launcher's environment."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Replicas:
    """world, rank: this process; device: where the reduction tensors live
    (the rank's GPU for NCCL, "cpu" for gloo)."""

    def __init__(self, world: int, rank: int, device="cpu"):
        self.world, self.rank, self.device = world, rank, device

    def barrier(self):
        if self.world > 1:
            import torch.distributed as dist

            dist.barrier()

    def _reduce(self, v, op):
        if self.world == 1:
            return float(v)
        import torch
        import torch.distributed as dist

        t = torch.tensor([float(v)], dtype=torch.float64, device=self.device)
        dist.all_reduce(t, op=op)
        return float(t.item())

    def max(self, v):
        import torch.distributed as dist

        return self._reduce(v, dist.ReduceOp.MAX)

    def sum(self, v):
        import torch.distributed as dist

        return self._reduce(v, dist.ReduceOp.SUM)

    def source_seed(self) -> int:
        """Each replica solves its own Gaussian source."""
        return self.rank

    def time_per_solve(self, elapsed_max_s: float, steps: int) -> float:
        """Whole-job time per solve: the slowest rank's time over all ranks' solves."""
        return elapsed_max_s / (steps * self.world)
