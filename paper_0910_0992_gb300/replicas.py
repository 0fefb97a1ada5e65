"""Replica runs over ranks: one process per GPU, each solving its own problems.

The temporally preconditioned solve keeps whole time lines on one GPU and its batches of sources
are independent, so a multi-GPU run is N replicas with no collective on the data path: every rank
solves its own sources, and only the timing is combined (a barrier before and after the timed
region, the slowest rank's time, the units of all ranks over it). Rendezvous comes from the
torchrun environment (RANK, WORLD_SIZE, LOCAL_RANK, MASTER_ADDR, MASTER_PORT).
"""

import os


class Replicas:
    """Process-group bookkeeping for a replica run; a no-op with one rank."""

    def __init__(self, backend="nccl", device=None):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.dist = None
        if self.world > 1:
            import torch.distributed as dist

            kwargs = {"device_id": device} if (backend == "nccl" and device is not None) else {}
            dist.init_process_group(backend, **kwargs)
            self.dist = dist
            self.rank = dist.get_rank()

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def max(self, x, device="cpu"):
        """The largest x over the ranks (the slowest rank's time)."""
        if self.dist is None:
            return float(x)
        import torch

        t = torch.tensor([float(x)], dtype=torch.float64, device=device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def whole_job_rate(self, units_per_rank, seconds):
        """Throughput of the whole job: every rank processed units_per_rank in at most seconds."""
        return self.world * units_per_rank / seconds

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()
            self.dist = None
