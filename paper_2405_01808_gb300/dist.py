"""Multi-GPU helpers: frames are independent (no interleaving across codewords,
Sec. IV), so N GPUs decode N disjoint frame shards with no collective on the
data path. torch.distributed is used only around the timed region: a barrier
before it, and afterwards the sum of the units processed and the maximum of the
per-rank elapsed times (whole-job throughput = total units / slowest rank)."""
from __future__ import annotations

import os


def rank_info():
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard_stream(rank: int, index: int) -> int:
    """Seed stream of one SNR batch of one rank: disjoint frames per rank."""
    return 100 * rank + index


def aggregate(units: list[float], elapsed_ms: float, dist=None, device=None):
    """Sum `units` over ranks and take the max of `elapsed_ms`.

    Without a process group this is the identity. With one, the tensors live on
    `device` (the rank's GPU for NCCL, the CPU for gloo)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return list(units), elapsed_ms
    import torch

    dev = device if device is not None else "cpu"
    u = torch.tensor([float(x) for x in units], dtype=torch.float64, device=dev)
    t = torch.tensor([float(elapsed_ms)], dtype=torch.float64, device=dev)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return u.cpu().tolist(), float(t.cpu().item())
