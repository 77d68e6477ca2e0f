"""Replicas on several GPUs: one independent build per rank (weak scaling).

The method's instances are independent, so ranks exchange nothing on the data
path; the only collectives are a barrier around the timed region and the
maximum of the ranks' times, which sets the whole job's time.  The backend is
the caller's (NCCL on GPUs; gloo serves the CPU tests of this logic).
"""
import os

import numpy as np

__all__ = ["rank_env", "init", "replica_rows", "barrier", "max_over_ranks", "aggregate", "finish"]


def rank_env():
    """(rank, world, local_rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend):
    """Join the process group when there is more than one rank."""
    _, world, _ = rank_env()
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend)
    return world


def replica_rows(n, rank):
    """Row order of rank `rank`'s replica: a different draw of the same
    workload on every rank (rank 0 keeps the workload's own order)."""
    if rank == 0:
        return np.arange(n)
    return np.random.default_rng(rank).permutation(n)


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(value, device="cpu"):
    """The largest `value` over all ranks (every rank gets it)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(points_per_rank, steps, seconds, world):
    """Whole-job throughput: every rank's points over the slowest rank's time."""
    return world * points_per_rank * steps / seconds


def finish():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.destroy_process_group()
