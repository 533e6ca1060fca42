"""Orientation sweeps sharded over ranks (one GPU per rank).

Right-hand sides (incident directions x polarizations) are independent, so a
sweep splits into contiguous RHS blocks, one per rank, with no exchange
while solving; only the per-RHS results (a few numbers each) are gathered at
the end.  This replaces the guide's MPI distribution of target orientations
("MPI" section) and is the multi-GPU form of the hot path.
"""
from __future__ import annotations


def shard_rhs(R: int, rank: int, world: int) -> range:
    """Contiguous block of RHS indices owned by `rank` (sizes differ by <= 1)."""
    if world <= 0 or not 0 <= rank < world or R < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(R, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def gather_results(local: list, dist=None) -> list:
    """All ranks' per-RHS result lists, concatenated in rank (= RHS) order."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return list(local)
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, list(local))
    out = []
    for p in parts:
        out.extend(p)
    return out


def solve_sweep(solve_block, khat, ehat, dist=None):
    """Solve the RHS block of this rank with ``solve_block(khat_block, ehat_block)``
    (which returns one result per RHS) and gather every rank's results."""
    R = len(khat)
    if dist is not None and dist.is_initialized():
        rank, world = dist.get_rank(), dist.get_world_size()
    else:
        rank, world = 0, 1
    idx = shard_rhs(R, rank, world)
    local = solve_block(khat[idx.start:idx.stop], ehat[idx.start:idx.stop]) if len(idx) else []
    return gather_results(local, dist)
