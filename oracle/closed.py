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


def four_cycles_two_paths(src, dst, n, block=16384):
    """Bag count of the 4-cycle query E(w,x),E(x,y),E(y,z),E(z,w) as
    sum over (w, y) of P2[w, y] * P2[y, w], where P2 = A A counts the
    2-paths from w to y (exact int64 sparse products; a 4-cycle is a
    2-path w -> y followed by a 2-path y -> w).  Equal to trace(A^4) but
    needs only the nonzeros of A^2, so it reaches graphs whose dense
    adjacency matrix does not fit.  The w's are taken `block` at a time:
    rows W of P2 are A[W] A, and the entries P2[y, w] for w in W are the
    columns W of P2, A A[:, W]."""
    import scipy.sparse as sp
    a = sp.csr_matrix((np.ones(len(src), dtype=np.int64),
                       (np.asarray(src, dtype=np.int64), np.asarray(dst, dtype=np.int64))),
                      shape=(n, n))
    a.sum_duplicates()
    ac = a.tocsc()
    total = 0
    for w0 in range(0, n, block):
        w1 = min(n, w0 + block)
        rows = (a[w0:w1] @ a).tocsr()           # P2[w, y], w in W
        cols = (a @ ac[:, w0:w1]).T.tocsr()     # P2[y, w] as [w, y], w in W
        total += int(rows.multiply(cols).sum())
    return total


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


def pkfk_direct(atoms, min_vars=()):
    """COUNT and MIN of a full conjunctive query whose atoms form a tree of
    primary-key / foreign-key links, by direct addressing -- the semi-join
    composition "follow each foreign key to its key row" (no hash table).

    The first atom is the root.  Every later atom shares exactly one
    variable with the atoms before it, read from its own first column, and
    that column holds distinct non-negative keys (its primary key); its other
    variables are its own.  An atom's pushed-down selections remove its rows
    before addressing.  For every root row passing its selections, the row
    of each later atom is found by addressing that atom's key array with the
    value of the shared variable in the row reached so far; the root row
    contributes one output tuple iff every atom has such a row (keys are
    unique, so no more than one).  Returns (count, mins) with None for an
    empty result.
    """
    ops = {"<": np.less, "<=": np.less_equal, ">": np.greater, ">=": np.greater_equal,
           "==": np.equal, "!=": np.not_equal}

    def passing(a):
        n = len(a["cols"][0]) if a["cols"] else 0
        ok = np.ones(n, dtype=bool)
        for j, op, v in a.get("preds", []):
            ok &= ops[op](np.asarray(a["cols"][j], dtype=np.int64), v)
        return ok

    root = atoms[0]
    n = len(root["cols"][0])
    alive = passing(root)
    # value of each bound variable for every root row (rows of later atoms
    # gathered through their keys)
    val = {v: np.asarray(c, dtype=np.int64) for v, c in zip(root["vars"], root["cols"])}
    for a in atoms[1:]:
        shared = [v for v in a["vars"] if v in val]
        assert len(shared) == 1 and a["vars"][0] == shared[0], "not a key/foreign-key tree"
        key = np.asarray(a["cols"][0], dtype=np.int64)
        assert len(np.unique(key)) == len(key) and (len(key) == 0 or key.min() >= 0)
        size = int(key.max()) + 1 if len(key) else 0
        ok = passing(a)
        row_of = np.full(size + 1, -1, dtype=np.int64)  # slot `size`: no row
        row_of[key[ok]] = np.nonzero(ok)[0]
        fk = val[shared[0]]
        inside = (fk >= 0) & (fk < size)
        r = row_of[np.where(inside, fk, size)]
        alive &= r >= 0
        rr = np.where(r >= 0, r, 0)
        for v, c in zip(a["vars"][1:], a["cols"][1:]):
            c = np.asarray(c, dtype=np.int64)
            val[v] = c[rr] if len(c) else np.zeros(n, dtype=np.int64)
    count = int(alive.sum())
    mins = [int(val[v][alive].min()) if count else None for v in min_vars]
    return count, mins
