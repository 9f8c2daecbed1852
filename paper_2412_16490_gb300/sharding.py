"""Grasp sharding across ranks (one process per GPU).

Grasps are independent -- the energy has no cross-grasp term and no upper
step exchanges data (Sec. IV-A) -- so N GPUs run N replicas of the path on
contiguous grasp ranges with no collective during the run.  The only
communication is an optional final gather of the results.
"""
from __future__ import annotations


def shard_range(B: int, rank: int, world: int) -> tuple[int, int]:
    """[lo, hi) of the grasps rank `rank` of `world` owns: contiguous, sizes
    differing by at most one, lower ranks taking the extra grasps."""
    if world < 1 or not (0 <= rank < world) or B < 0:
        raise ValueError("need world >= 1, 0 <= rank < world, B >= 0")
    base, extra = divmod(B, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def gather_shards(local, B: int, dist=None):
    """Concatenate every rank's [hi - lo, ...] tensor into the full [B, ...]
    batch on every rank (all_gather of padded shards, then trim)."""
    import torch
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return local
    world, rank = dist.get_world_size(), dist.get_rank()
    sizes = [shard_range(B, r, world) for r in range(world)]
    width = max(hi - lo for lo, hi in sizes)
    pad = torch.zeros((width,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    pad[: local.shape[0]] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad)
    return torch.cat([p[: hi - lo] for p, (lo, hi) in zip(parts, sizes)], 0)
