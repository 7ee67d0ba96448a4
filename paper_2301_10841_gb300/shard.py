"""Sharding a join across ranks (one process per GPU): node 0's cover rows
are split into contiguous ranges, every other relation is replicated, and
each rank's COUNT and MINs are merged with one all-reduce at the end -- the
only exchange, since the ranges are independent.  The merge works on any
torch.distributed backend (gloo on CPU, NCCL on GPUs)."""

from __future__ import annotations

NO_ROW = 2**31  # above every int32 value: "this rank has no result row"


def row_range(n, rank, world):
    """Rank `rank`'s contiguous range [lo, hi) of n rows."""
    return n * rank // world, n * (rank + 1) // world


def merge(count, mins, group=None, device="cpu"):
    """Sum of the ranks' counts and the minimum of their MINs (None where a
    rank has no result row); every rank gets the merged values.

    MINs travel as int64 with NO_ROW (2^31, no int32 value) for a rank
    without a row, so a true MIN of 2^31 - 1 is kept.  Counts are uint64:
    they travel as their two 32-bit halves, summed separately in int64 (no
    overflow below 2^31 ranks) and recombined; a total of 2^64 or more
    raises OverflowError, as COUNT(*) overflow does in the library."""
    import torch
    import torch.distributed as dist
    count = int(count)
    if not 0 <= count < 2**64:
        raise ValueError("count must be a uint64")
    c = torch.tensor([count & 0xFFFFFFFF, count >> 32], dtype=torch.int64, device=device)
    m = torch.tensor([NO_ROW if v is None else int(v) for v in mins] or [NO_ROW],
                     dtype=torch.int64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(m, op=dist.ReduceOp.MIN, group=group)
    lo, hi = (int(x) for x in c.tolist())
    total = lo + (hi << 32)
    if total >= 2**64:
        raise OverflowError("merged COUNT(*) exceeds 2^64 - 1")
    merged = [None if total == 0 or int(v) == NO_ROW else int(v) for v in m.tolist()]
    return total, merged[:len(mins)]
