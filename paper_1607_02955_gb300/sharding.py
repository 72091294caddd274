"""Splitting one JL farness query (Algorithm 1) over several GPUs.

The k rows of Q are independent solves and f~(v) is a sum over them, so
each rank takes a contiguous, 32-aligned block of rows (cfc_farness_jl_rows),
and the ranks' q partial sums are added by one all-reduce: the only exchange
on the path, q doubles per query.  The graph and its hierarchy are
replicated on every rank.
"""
from __future__ import annotations

import numpy as np


def shard_rows(k_total: int, world: int, rank: int) -> tuple[int, int]:
    """(row_begin, row_count) of this rank: blocks of 32 rows dealt out as
    evenly as possible in rank order (row_begin a multiple of 32, as the row
    generator needs); a rank may get no rows when k_total < 32 * world."""
    if k_total < 1 or world < 1 or not 0 <= rank < world:
        raise ValueError("need k_total >= 1 and 0 <= rank < world")
    blocks = (k_total + 31) // 32
    per, extra = divmod(blocks, world)
    b0 = rank * per + min(rank, extra)
    nb = per + (1 if rank < extra else 0)
    r0 = min(k_total, 32 * b0)
    r1 = min(k_total, 32 * (b0 + nb))
    return r0, r1 - r0


def allreduce_partials(partial_fn, k_total: int, q: int, group=None) -> np.ndarray:
    """Sum over the ranks of `group` of partial_fn(row_begin, row_count) (a
    length-q array of this rank's row terms).  Ranks without rows add zeros."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    r0, c = shard_rows(k_total, world, rank)
    part = np.asarray(partial_fn(r0, c), np.float64) if c > 0 else np.zeros(q, np.float64)
    t = torch.tensor(part, dtype=torch.float64)
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.cpu().numpy()


def cfc_farness_jl_distributed(h, k_total: int, seed: int, nodes, opts=None, group=None) -> np.ndarray:
    """cfc_farness_jl over the ranks of `group` (each holding its own copy of
    the hierarchy on its own GPU): row shards, then one all-reduce."""
    from ._binding import cfc_farness_jl_rows
    nd = np.ascontiguousarray(nodes, np.int32)
    return allreduce_partials(lambda r0, c: cfc_farness_jl_rows(h, k_total, r0, c, seed, nd, opts=opts),
                              k_total, nd.size, group)
