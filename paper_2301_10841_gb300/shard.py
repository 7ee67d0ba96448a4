"""Sharding a join across ranks (one process per GPU): node 0's cover rows
are split into contiguous ranges, every other relation is replicated, and
each rank's COUNT and MINs are merged with one all-reduce at the end -- the
only exchange, since the ranges are independent.  The merge works on any
torch.distributed backend (gloo on CPU, NCCL on GPUs)."""

from __future__ import annotations

INT32_MAX = 2**31 - 1


def row_range(n, rank, world):
    """Rank `rank`'s contiguous range [lo, hi) of n rows."""
    return n * rank // world, n * (rank + 1) // world


def merge(count, mins, group=None, device="cpu"):
    """Sum of the ranks' counts and the minimum of their MINs (None where a
    rank has no result row); every rank gets the merged values."""
    import torch
    import torch.distributed as dist
    c = torch.tensor([int(count)], dtype=torch.int64, device=device)
    m = torch.tensor([INT32_MAX if v is None else int(v) for v in mins] or [INT32_MAX],
                     dtype=torch.int64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(m, op=dist.ReduceOp.MIN, group=group)
    total = int(c.item())
    merged = [None if total == 0 or int(v) == INT32_MAX else int(v) for v in m.tolist()]
    return total, merged[:len(mins)]
