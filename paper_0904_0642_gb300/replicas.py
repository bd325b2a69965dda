"""Replica runs over ranks: every rank advances its own independent chain.

Independent Markov chains need no exchange, so the multi-GPU form of the
sweep is N replicas, one per GPU (one process per GPU, launched by
torch.distributed.run).  Only the timing is collective: a barrier on both
sides of the timed region and the maximum of the per-rank times, so the
whole-job rate is (units processed by all ranks) / (slowest rank's time).
"""
from __future__ import annotations

import os


class Replicas:
    """Rank bookkeeping and the two timing collectives (barrier, max)."""

    def __init__(self, backend: str | None = None, device=None):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local_rank = int(os.environ.get("LOCAL_RANK", "0"))
        self._dist = None
        self._device = device
        if self.world > 1:
            import torch.distributed as dist
            if not dist.is_initialized():
                kw = {}
                if backend == "nccl" and device is not None:
                    kw["device_id"] = device
                dist.init_process_group(backend or "gloo", **kw)
            self._dist = dist

    def seed(self, base: int) -> int:
        """A distinct chain seed per rank."""
        return base + self.rank

    def barrier(self):
        if self._dist is not None:
            self._dist.barrier()

    def max(self, x: float) -> float:
        if self._dist is None:
            return float(x)
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64, device=self._device or "cpu")
        self._dist.all_reduce(t, op=self._dist.ReduceOp.MAX)
        return float(t.item())

    def rate(self, units_per_rank: float, seconds_this_rank: float) -> float:
        """Whole-job rate: all ranks' units over the slowest rank's time."""
        return self.world * units_per_rank / self.max(seconds_this_rank)

    def close(self):
        if self._dist is not None and self._dist.is_initialized():
            self._dist.destroy_process_group()
