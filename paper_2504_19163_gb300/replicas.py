"""Multi-GPU runs of the bound / render step: independent replicas, one process per GPU.

The path shards trivially (every rank runs the whole step on its own GPU: weak scaling), so there
is no collective on the data path; the only cross-rank operations are the barriers around the timed
region and the max over ranks of the step time, which sets the whole-job throughput
(units processed by all ranks / slowest rank's time)."""
from __future__ import annotations

import os
from typing import Optional

import torch


def rank_env():
    """(rank, local_rank, world_size) from the launcher's environment (1 process when unset)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def init(backend: str, device: Optional[torch.device] = None):
    """torch.distributed process group for world_size > 1, else None."""
    rank, local, world = rank_env()
    if world <= 1:
        return None
    import torch.distributed as dist
    if backend == "nccl":
        dist.init_process_group("nccl", device_id=device)
    else:
        dist.init_process_group(backend)
    return dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(x: float, dist, device="cpu") -> float:
    """The largest value of x over all ranks (x itself with one rank)."""
    if dist is None:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job throughput of weak-scaled replicas: every rank processed units_per_rank in at most
    ms_max milliseconds."""
    return units_per_rank * world / (ms_max / 1e3)


def finish(dist):
    if dist is not None:
        dist.destroy_process_group()
