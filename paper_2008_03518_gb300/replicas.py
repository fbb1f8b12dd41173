"""Replica bookkeeping for runs with one process per GPU.

First-come-first-served planning is sequential per plan table, so N GPUs run N independent
replicas of the workload (each its own table and requests) and exchange nothing on the
data path. What the ranks share is the measurement: a barrier on both sides of the timed
region, the slowest rank's time, and the whole-job rate (all ranks' plans over that time).
This module holds that host-side logic, for the nccl backend on GPUs and gloo on CPU.
"""
import os


def dist_env():
    """(rank, local_rank, world_size) from the launcher's environment (1 process: 0, 0, 1)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


class Replicas:
    """The job's ranks. With world_size 1 nothing is initialised and every reduction is
    the identity; otherwise torch.distributed runs on `backend` (nccl: tensors on the
    current CUDA device; gloo: on the CPU)."""

    def __init__(self, backend="nccl"):
        self.rank, self.local_rank, self.world = dist_env()
        self.backend = backend
        self._dist = None
        if self.world > 1:
            import torch
            import torch.distributed as dist

            if not dist.is_initialized():
                if backend == "nccl":
                    dist.init_process_group("nccl", device_id=torch.device("cuda", 0))
                else:
                    dist.init_process_group(backend)
            self._dist = dist

    def _tensor(self, x):
        import torch

        dev = "cuda" if self.backend == "nccl" else "cpu"
        return torch.tensor([float(x)], dtype=torch.float64, device=dev)

    def barrier(self):
        if self._dist is not None:
            self._dist.barrier()

    def max(self, x):
        """Largest x over the ranks (the slowest rank's time)."""
        if self._dist is None:
            return float(x)
        t = self._tensor(x)
        self._dist.all_reduce(t, op=self._dist.ReduceOp.MAX)
        return float(t.item())

    def sum(self, x):
        if self._dist is None:
            return float(x)
        t = self._tensor(x)
        self._dist.all_reduce(t, op=self._dist.ReduceOp.SUM)
        return float(t.item())

    def whole_job_rate(self, units_this_rank, ms_this_rank):
        """Units all ranks processed per second of the slowest rank's time."""
        total = self.sum(units_this_rank)
        ms = self.max(ms_this_rank)
        return total / (ms / 1e3), ms

    def close(self):
        if self._dist is not None:
            self._dist.destroy_process_group()
            self._dist = None
