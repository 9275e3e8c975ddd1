"""Host-side coordination of independent replicas (one process per GPU).

The propagator has no data-path exchange between independent runs: each rank
advances its own members.  The only collective is the max-reduce of the
timing (and a barrier around the timed region).  The same code runs with
NCCL on GPUs and with gloo on CPU.
"""
from __future__ import annotations

import os


def dist_env():
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


class Replicas:
    def __init__(self, backend="nccl", device=None):
        import torch
        import torch.distributed as dist
        self.torch = torch
        self.rank, self.world, self.local_rank = dist_env()
        self.device = device
        self.dist = None
        if self.world > 1:
            kw = {}
            if backend == "nccl" and device is not None:
                kw["device_id"] = torch.device(device)
            dist.init_process_group(backend, **kw)
            self.dist = dist

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def max_over_ranks(self, x):
        """Largest value of x over the ranks (x itself on one rank)."""
        if self.dist is None:
            return float(x)
        t = self.torch.tensor([float(x)], dtype=self.torch.float64, device=self.device or "cpu")
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def weak_throughput(self, units_per_rank, seconds):
        """Whole-job units per second: every rank processed units_per_rank in
        at most `seconds` (the max over ranks)."""
        return self.world * units_per_rank / seconds

    def member_seed(self, member, base=2):
        """Seed of a rank's member: distinct across ranks."""
        return 1000 * self.rank + member + base

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()
            self.dist = None
