"""Multi-GPU replicas: one process per GPU, each solving its own problems, no collective on the
data path.  The solver itself is one GPU by design; the independent right-hand sides, batches
and systems scale by running one replica per GPU (weak scaling).  The process group serves only
the barrier around the timed region and the reductions of the per-rank counts and times.

Launch as ``torchrun --nproc-per-node N --master-addr 127.0.0.1 ...``; RANK, WORLD_SIZE and
LOCAL_RANK come from the environment.
"""
from __future__ import annotations

import os

__all__ = ["Replicas"]


class Replicas:
    """Rank bookkeeping, barrier and the two reductions a replicated timing needs."""

    def __init__(self, backend: str | None = None):
        self.rank = int(os.environ.get("RANK", "0"))
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.local_rank = int(os.environ.get("LOCAL_RANK", "0"))
        self.dist = None
        if self.world > 1:
            import torch.distributed as dist

            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            if not dist.is_initialized():
                dist.init_process_group(backend or "nccl", rank=self.rank, world_size=self.world)
            self.dist = dist

    def _reduce(self, value: float, op: str, device=None) -> float:
        if self.dist is None:
            return float(value)
        import torch

        t = torch.tensor([float(value)], dtype=torch.float64, device=device)
        self.dist.all_reduce(t, op=getattr(self.dist.ReduceOp, op))
        return float(t.item())

    def barrier(self):
        if self.dist is not None:
            if self.dist.get_backend() == "nccl":  # the rank's own GPU (set by the caller)
                self.dist.barrier(device_ids=[self.local_rank])
            else:
                self.dist.barrier()

    def max(self, value: float, device=None) -> float:
        """The slowest rank's time (the whole job ends when it does)."""
        return self._reduce(value, "MAX", device)

    def sum(self, value: float, device=None) -> float:
        """Units (edge-updates, solves) processed by all ranks."""
        return self._reduce(value, "SUM", device)

    def job_rate(self, units: float, seconds: float, device=None) -> float:
        """Whole-job throughput: the units every rank processed over the slowest rank's time."""
        return self.sum(units, device) / self.max(seconds, device)

    def close(self):
        if self.dist is not None and self.dist.is_initialized():
            self.dist.destroy_process_group()
        self.dist = None
