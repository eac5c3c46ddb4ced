"""Replica parallelism across GPUs of one node.

A Laplace solve on one grid does not shard here: every GPU (one process each, launched
by torch.distributed.run) solves its own independent problems. The only collectives are
a barrier around the timed region and a max/sum of host scalars (timings, counts) --
nothing on the data path.
"""
from __future__ import annotations

import os

import torch
import torch.distributed as dist


def world() -> tuple[int, int, int]:
    """(rank, world_size, local_rank) from the launcher's environment (1 process if unset)."""
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def init(backend: str | None = None) -> tuple[int, int, int]:
    rank, size, local = world()
    if size > 1 and not dist.is_initialized():
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return rank, size, local


def barrier():
    if dist.is_initialized():
        dist.barrier()


def reduce_scalar(value: float, op: str = "max") -> float:
    """Max or sum of a host float over all ranks (identity with one process)."""
    if not dist.is_initialized():
        return float(value)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def shard(count: int, rank: int, size: int) -> range:
    """Contiguous block of `count` independent units owned by `rank` (sizes differ by <= 1)."""
    base, extra = divmod(count, size)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def finish():
    if dist.is_initialized():
        dist.barrier()
        dist.destroy_process_group()
