"""Sharding of the generator workloads over several GPUs (one process each).

The V-family generators of a workload are independent (Sec. 3: every
generator is seeded and jumped on its own), so the path shards by generator
with no collective on the data path: rank r of a world of W ranks owns
generators [r * G, (r + 1) * G) of the workload's global generator sequence,
G per rank (weak scaling: per-GPU work fixed as W grows).  The only
communication is for timing: a barrier around the timed region and the
maximum of the ranks' times.

The collectives work on either backend: NCCL with CUDA tensors on GPU runs,
gloo with CPU tensors (used by the multi-process tests on the host).
"""
from __future__ import annotations

import os

import numpy as np

from . import inputs as I


def rank_slice(per_rank: int, world: int, rank: int) -> tuple[int, int]:
    """(first, count) of the generators rank `rank` owns."""
    if world < 1 or not 0 <= rank < world or per_rank < 0:
        raise ValueError("need world >= 1, 0 <= rank < world and per_rank >= 0")
    return rank * per_rank, per_rank


def rank_seeds(workload: str, world: int, rank: int, per_rank: int | None = None) -> np.ndarray:
    """Seeds of the generators owned by `rank`."""
    n = I.WORKLOADS[workload]["generators"] if per_rank is None else per_rank
    first, count = rank_slice(n, world, rank)
    return I.workload_seeds(workload, first, count)


def env_world() -> tuple[int, int, int]:
    """(world size, rank, local rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def _device():
    dist = _dist()
    if dist is not None and dist.get_backend() == "nccl":
        import torch
        return torch.device("cuda", torch.cuda.current_device())
    return "cpu"


def barrier() -> None:
    dist = _dist()
    if dist is not None and dist.get_world_size() > 1:
        dist.barrier()


def max_over_ranks(x: float) -> float:
    dist = _dist()
    if dist is None or dist.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float) -> float:
    dist = _dist()
    if dist is None or dist.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
