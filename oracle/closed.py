"""Closed forms and library routines that pin the oracle -- TEST INFRASTRUCTURE ONLY.

None of these evaluate a Free Join plan; each reaches a join result through
mathematics that is independent of hash joins and hash tries.
"""

from __future__ import annotations

import numpy as np


def adjacency(src, dst, n):
    """Multiplicity adjacency matrix A[x, y] = #rows (x, y) of the edge table."""
    a = np.zeros((n, n), dtype=np.float64)
    np.add.at(a, (np.asarray(src, dtype=np.int64), np.asarray(dst, dtype=np.int64)), 1.0)
    return a


def trace_power(a, k):
    """trace(A^k) by float64 BLAS matmul.

    For the triangle query E(x,y),E(y,z),E(z,x) the bag count is trace(A^3);
    for the 4-cycle E(w,x),E(x,y),E(y,z),E(z,w) it is trace(A^4).  Every
    partial sum is an integer below 2^53 at the sizes used, so the float64
    result is exact.
    """
    p = np.eye(a.shape[0])
    for _ in range(k):
        p = p @ a
    t = float(np.trace(p))
    assert t < 2.0 ** 53
    return int(round(t))


def complete_digraph_cycles(n, k):
    """trace((J - I)^k) for the complete directed graph on n vertices without
    self-loops: the eigenvalues of J - I are n - 1 (once) and -1 (n - 1 times),
    so the count of closed k-walks -- the bag count of the k-cycle query,
    which has no disequalities -- is (n-1)^k + (n-1)(-1)^k.  For k = 3 this is
    n(n-1)(n-2)."""
    return (n - 1) ** k + (n - 1) * (-1) ** k


def star_join_direct(fact_cols, dims, thresholds):
    """COUNT and MIN of Q(k.., a..) :- F(k1..kd), D1(k1,a1), ..., Dd(kd,ad)
    with the selection a_i < theta_i on each dimension, by direct addressing.

    ``dims[i] = (key, attr)`` with keys in [0, len(key)).  For each dimension
    the passing rows are counted per key (cnt_i) and their least attribute is
    kept (lo_i).  A fact row contributes prod_i cnt_i[k_i] output tuples, and
    its MIN of a_i is lo_i[k_i].  This is the single-scan semi-join
    formulation; it uses no hash table.
    Returns (count, [min a_1, ..., min a_d]) with None for an empty result.
    """
    n = len(fact_cols[0])
    mult = np.ones(n, dtype=np.uint64)
    lows = []
    for (key, attr), theta, fk in zip(dims, thresholds, fact_cols):
        key = np.asarray(key, dtype=np.int64)
        attr = np.asarray(attr, dtype=np.int64)
        size = int(key.max()) + 1 if len(key) else 0
        keep = attr < theta
        cnt = np.zeros(size + 1, dtype=np.uint64)
        np.add.at(cnt, key[keep], np.uint64(1))
        lo = np.full(size + 1, np.iinfo(np.int64).max, dtype=np.int64)
        np.minimum.at(lo, key[keep], attr[keep])
        fk = np.asarray(fk, dtype=np.int64)
        inside = (fk >= 0) & (fk < size)
        idx = np.where(inside, fk, size)  # slot `size` holds count 0
        mult *= cnt[idx]
        lows.append(lo[idx])
    live = mult > 0
    count = int(mult.sum(dtype=np.uint64))
    mins = [int(l[live].min()) if live.any() else None for l in lows]
    return count, mins
