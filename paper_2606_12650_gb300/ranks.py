"""Replica bookkeeping for runs on several GPUs of one node.

The solve does not shard: every rank solves its own independent problems
(seeds offset by the rank), with no collective on the data path.  The only
collectives are host-side bookkeeping around a timed region: a barrier before
and after it, and the job's figures -- the slowest rank's time and the sum of
the work units over ranks, so that throughput = all units / slowest time.
"""
from __future__ import annotations

import os

SEED_STRIDE = 1000     # distance between the seeds of two ranks' problem draws


def rank_env():
    """(rank, local_rank, world_size) from the torchrun environment."""
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def rank_seed(base: int, rank: int) -> int:
    """Seed of a rank's own draw; ranks never share a problem."""
    return base + SEED_STRIDE * rank


class Job:
    """The ranks of one run.  `dist` is torch.distributed (initialised when
    world > 1); `device` is where the reduction tensors live (the rank's GPU
    under NCCL, the CPU under gloo)."""

    def __init__(self, world: int, dist=None, device="cpu", local: int | None = None):
        self.world = world
        self.dist = dist
        self.device = device
        self.local = local

    def barrier(self):
        if self.world <= 1:
            return
        if self.dist.get_backend() == "nccl":
            self.dist.barrier(device_ids=[self.local])
        else:
            self.dist.barrier()

    def aggregate(self, t: float, units: float):
        """(max of t over ranks, sum of units over ranks)."""
        if self.world <= 1:
            return float(t), float(units)
        import torch
        tt = torch.tensor([float(t)], device=self.device, dtype=torch.float64)
        self.dist.all_reduce(tt, op=self.dist.ReduceOp.MAX)
        uu = torch.tensor([float(units)], device=self.device, dtype=torch.float64)
        self.dist.all_reduce(uu, op=self.dist.ReduceOp.SUM)
        return float(tt.item()), float(uu.item())

    def throughput(self, t_s: float, units: float):
        """Whole-job units per second: all ranks' units over the slowest
        rank's seconds."""
        t_max, u_sum = self.aggregate(t_s, units)
        return u_sum / t_max, t_max, u_sum
