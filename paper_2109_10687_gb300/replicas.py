"""Host logic for running independent replicas of the solve, one process per
GPU.

The solve needs no exchange between GPUs, so N GPUs run N independent
problems (weak scaling).  The only collective operations are the barrier
around the timed region and the maximum of the per-rank times, from which
the whole-job throughput follows.
"""

import os

import torch
import torch.distributed as dist


def rank_env():
    """(world size, rank, local rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def replica_seeds(gauge_seed, source_seed, rank):
    """Each rank draws its own gauge field and source (independent replicas)."""
    return gauge_seed + rank, source_seed + rank


def barrier(world):
    if world > 1:
        dist.barrier()


def max_over_ranks(value, world, device=None):
    """The largest per-rank value (the slowest rank's time)."""
    if world == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, units_per_rank, elapsed_max):
    """Units all ranks processed divided by the slowest rank's time."""
    return world * units_per_rank / elapsed_max
