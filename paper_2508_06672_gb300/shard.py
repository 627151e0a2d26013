"""Row sharding of a candidate grid over ranks, and the max-loc merge.

Candidates are independent (Algorithm 1's inner loop), so a grid is split
into contiguous blocks of latitude rows, one per GPU, with no exchange during
the computation. The only exchange is the final argmax: each rank's best
(value, global linear index), merged with the same rule as the device argmax
(largest value, ties to the lowest index, NaN never wins).
"""
from __future__ import annotations

import math


def shard_rows(nlat: int, world: int, rank: int):
    """(row0, nrows) of rank's block; the first nlat % world ranks get one
    row more."""
    if not (0 <= rank < world) or nlat < world:
        raise ValueError("need 0 <= rank < world <= nlat")
    base, extra = divmod(nlat, world)
    row0 = rank * base + min(rank, extra)
    return row0, base + (1 if rank < extra else 0)


def merge_argmax(entries):
    """entries: iterable of (value, global_index); index < 0 = no candidate.
    Returns the winning (value, index) or (nan, -1)."""
    best = (math.nan, -1)
    for v, i in entries:
        if i < 0 or v != v:
            continue
        if best[1] < 0 or v > best[0] or (v == best[0] and i < best[1]):
            best = (float(v), int(i))
    return best


def allreduce_argmax(value, index, group=None):
    """Max-loc over the ranks of a torch.distributed group (any backend)."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    mine = torch.tensor([float(value), float(index)], dtype=torch.float64)
    if dist.get_backend(group) == "nccl":
        mine = mine.cuda()
    out = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(out, mine, group=group)
    return merge_argmax((float(t[0]), int(t[1])) for t in out)
