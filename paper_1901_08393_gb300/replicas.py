"""Replica parallelism: independent capacity problems spread over ranks.

A single problem here fits one GPU, so several GPUs run independent problems
(meshes, requests) with no collective on the data path; torch.distributed is used
only to agree on timing and totals at the end.
"""
from __future__ import annotations

import datetime
import os


def world():
    """(world_size, rank, local_rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(items, rank: int, world_size: int):
    """Items of this rank: round-robin, so ranks get equal counts +-1 in input order."""
    return [x for k, x in enumerate(items) if k % world_size == rank]


def init(backend: str, timeout_s: float = 60.0, device=None):
    import torch.distributed as dist

    kw = {"timeout": datetime.timedelta(seconds=timeout_s)}
    if device is not None:
        kw["device_id"] = device
    dist.init_process_group(backend, **kw)


def reduce_max(value: float) -> float:
    """Slowest rank's time: whole-job time of replicas that started together."""
    import torch
    import torch.distributed as dist

    if not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value: float) -> float:
    import torch
    import torch.distributed as dist

    if not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t)
    return float(t.item())


def gather(obj):
    """Every rank's object, in rank order, on every rank."""
    import torch.distributed as dist

    if not dist.is_initialized() or dist.get_world_size() == 1:
        return [obj]
    out = [None] * dist.get_world_size()
    dist.all_gather_object(out, obj)
    return out
