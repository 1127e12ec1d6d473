"""Host-side logic for running independent solves on several GPUs (one process per GPU).

The hot path does not exchange data between GPUs: each rank solves its own LP instances
(weak scaling, no collective on the data path).  The only collectives are on the host
after the timed region: a barrier around it and a MAX over ranks of the elapsed time and a
SUM of the iterations, so that the reported throughput is whole-job work / slowest rank.
"""
from __future__ import annotations

import os


def env_rank_world() -> tuple[int, int, int]:
    """(rank, local_rank, world_size) from the torchrun environment (1 process by default)."""
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    return rank, local, world


def instance_seeds(rank: int, world: int, per_rank: int = 1, base: int = 0) -> list[int]:
    """Seeds of the instances rank `rank` solves: disjoint across ranks, `per_rank` each."""
    if not (0 <= rank < world) or per_rank < 1:
        raise ValueError("bad rank/world/per_rank")
    return [base + rank * per_rank + q for q in range(per_rank)]


def reduce_elapsed_and_work(elapsed_s: float, work: float, group=None) -> tuple[float, float]:
    """(max elapsed over ranks, total work over ranks); identity without torch.distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(elapsed_s), float(work)
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.tensor([float(elapsed_s)], dtype=torch.float64, device=dev)
    w = torch.tensor([float(work)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(w, op=dist.ReduceOp.SUM, group=group)
    return float(t.item()), float(w.item())
