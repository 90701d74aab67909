"""Multi-GPU running of the search as independent replicas.

Scan pairs are independent (each pose depends on its own two scans only), so N ranks, one per
GPU, each take their own shard of pairs: there is no data-path collective.  The only
communication is the timing protocol: a barrier on both sides of the timed region and the
maximum of the per-rank step times, from which the whole-job rate is all ranks' pairs divided by
the slowest rank's time (weak scaling: the pairs per rank stay fixed as N grows).
"""
from __future__ import annotations

import os


def world():
    """(world size, rank, local rank) from the launcher's environment (1, 0, 0 without one)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(pairs_per_rank, rank):
    """(first pair index, pair count) of a rank's shard of the synthetic workload."""
    return rank * pairs_per_rank, pairs_per_rank


def init(backend):
    """Joins the process group when launched with more than one rank; returns torch.distributed or
    None."""
    if world()[0] <= 1:
        return None
    import torch.distributed as dist
    dist.init_process_group(backend)
    return dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(value, dist, device="cpu"):
    """The largest of the ranks' values (every rank receives it)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world_size, pairs_per_rank, ms_per_step_max):
    """Whole-job pairs per second: every rank's pairs over the slowest rank's step time."""
    return world_size * pairs_per_rank / (ms_per_step_max * 1e-3)
