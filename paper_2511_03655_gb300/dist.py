"""Multi-GPU host logic: one process per GPU, independent shards.

The trajectories of an ensemble are independent, so every rank integrates
its own shard (seeded by its rank) with no collective on the data path; the
only communication is a barrier around the timed region and the max / sum
of timings and step counts, done with whatever torch.distributed backend the
process group uses (NCCL between GPUs, gloo on the CPU in tests).
"""
from __future__ import annotations

import os

import torch
import torch.distributed as dist


def world() -> tuple[int, int, int]:
    """(rank, world size, local rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard_seed(base_seed_id: int, rank: int) -> int:
    """Seed id of rank r's shard: rank 0 draws the standard ensemble, the
    others disjoint streams 1000 seeds apart."""
    return base_seed_id + 1000 * rank


def _device_for(backend: str):
    return torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")


def reduce_max(x: float) -> float:
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=_device_for(dist.get_backend()))
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(x: float) -> float:
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=_device_for(dist.get_backend()))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier():
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()
