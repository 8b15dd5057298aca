"""Splitting independent ACI products across ranks (replicas only).

One ACI product does not shard: its bonds are visited in sequence through the frames and every
pivot step needs a global argmax over the Pi block (Algorithm 1, Algorithm 2). Independent
products (a batch of pairs, or the time steps of a sequence) are split across ranks by index,
with no collective on the data path; rank 0 gathers only the per-rank counts and timings.
"""

from __future__ import annotations


def shard(n_items: int, rank: int, world: int) -> range:
    """Contiguous block of item indices owned by ``rank`` (sizes differ by at most one)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank/world")
    base, extra = divmod(n_items, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def gather_to_rank0(obj, group=None):
    """Host-side gather of a small Python object (counts, timings) to rank 0."""
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return [obj]
    world = dist.get_world_size(group)
    out = [None] * world if dist.get_rank(group) == 0 else None
    dist.gather_object(obj, out, dst=0, group=group)
    return out
