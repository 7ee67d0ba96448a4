"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random relations and writes down query shapes; it
holds no join arithmetic, so both the CUDA library's tests and the CPU oracle
can be fed from it.  Every generator takes an explicit seed and uses numpy's
PCG64.

Relations are dicts ``{"name": str, "cols": [int32 arrays]}``; queries are
lists of atoms ``{"rel": relation, "cols": [int32 arrays], "vars": [...],
"preds": [(j, op, value)]}`` where ``cols`` are the relation's columns in the
atom's variable order (the form the oracle reads) and ``rel_cols`` the
column indices into the relation (the form the CUDA library reads).
"""

from __future__ import annotations

import numpy as np


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def atom(rel, vars_, rel_cols=None, preds=()):
    rel_cols = list(range(len(vars_))) if rel_cols is None else list(rel_cols)
    return {"rel": rel, "cols": [rel["cols"][c] for c in rel_cols], "vars": list(vars_),
            "rel_cols": rel_cols, "preds": list(preds)}


# ---------------------------------------------------------------------------
# Graphs
# ---------------------------------------------------------------------------

def uniform_digraph(n, m, seed):
    """m distinct directed edges drawn uniformly without replacement from the
    n(n-1) ordered pairs without self-loops; int32 endpoints."""
    rng = _rng(seed)
    idx = rng.choice(n * (n - 1), size=m, replace=False)
    src = idx // (n - 1)
    off = idx % (n - 1)
    dst = off + (off >= src)  # skip the diagonal
    return {"name": "E", "cols": [src.astype(np.int32), dst.astype(np.int32)]}


def complete_digraph(n):
    src, dst = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    keep = src != dst
    return {"name": "E", "cols": [src[keep].astype(np.int32), dst[keep].astype(np.int32)]}


def rmat(scale, n_edges, seed, a=0.57, b=0.19, c=0.19):
    """R-MAT graph with 2^scale vertices: edges are drawn quadrant by quadrant
    with probabilities (a, b, c, 1-a-b-c) per bit level (no noise); self-loops
    and duplicates are dropped and drawing continues until exactly n_edges
    distinct edges exist.  Vertex ids are then relabelled by a seeded random
    permutation."""
    rng = _rng(seed)
    n = 1 << scale
    have = np.empty(0, dtype=np.int64)
    while len(have) < n_edges:
        k = int((n_edges - len(have)) * 1.15) + 1024
        u = np.zeros(k, dtype=np.int64)
        v = np.zeros(k, dtype=np.int64)
        for _ in range(scale):
            r = rng.random(k)
            ubit = r >= a + b                  # quadrants c, d
            vbit = ((r >= a) & (r < a + b)) | (r >= a + b + c)  # quadrants b, d
            u = (u << 1) | ubit
            v = (v << 1) | vbit
        code = u * n + v
        code = code[u != v]
        have = np.unique(np.concatenate([have, code]))
    if len(have) > n_edges:
        have = rng.choice(have, size=n_edges, replace=False)
    perm = rng.permutation(n)
    src = perm[have // n].astype(np.int32)
    dst = perm[have % n].astype(np.int32)
    order = rng.permutation(n_edges)
    return {"name": "E", "cols": [src[order], dst[order]]}


def triangle_query(edges):
    """Q(x,y,z) :- E(x,y), E(y,z), E(z,x) with x=0, y=1, z=2 (self-join renamed
    into three atoms over the same columns)."""
    return [atom(edges, [0, 1]), atom(edges, [1, 2]), atom(edges, [2, 0])]


def four_cycle_query(edges):
    """Q(w,x,y,z) :- E(w,x), E(x,y), E(y,z), E(z,w) with w=0, x=1, y=2, z=3."""
    return [atom(edges, [0, 1]), atom(edges, [1, 2]), atom(edges, [2, 3]), atom(edges, [3, 0])]


# ---------------------------------------------------------------------------
# Star join
# ---------------------------------------------------------------------------

ZIPF_EXACT_MAX = 4_000_000  # larger domains use the continuous inverse CDF


def zipf_ranks(n_items, s, size, rng):
    """Ranks in [0, n_items) with P(rank r) proportional to (r+1)^-s, by
    inverse-CDF lookup on the cumulative weights.  Domains above
    ZIPF_EXACT_MAX items (the chooser's 1M-50M-row evaluation relations) use
    the inverse of the continuous power law on [1, n_items + 1) instead,
    floor(x) - 1 with x = (1 + u ((n+1)^(1-s) - 1))^(1/(1-s)) (x = (n+1)^u
    when s = 1): the same tail exponent without an n-element table."""
    if n_items > ZIPF_EXACT_MAX:
        u = rng.random(size)
        if abs(s - 1.0) < 1e-9:
            x = np.power(float(n_items + 1), u)
        else:
            x = np.power(1.0 + u * ((n_items + 1.0) ** (1.0 - s) - 1.0), 1.0 / (1.0 - s))
        return np.clip(np.floor(x).astype(np.int64) - 1, 0, n_items - 1)
    w = np.arange(1, n_items + 1, dtype=np.float64) ** (-s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    u = rng.random(size)
    return np.minimum(np.searchsorted(cdf, u, side="right"), n_items - 1)


STAR_DIMS = (100_000, 250_000, 500_000, 1_000_000)
STAR_THETA = 100_000_000  # attr uniform in [0, 1e9): keeps 10% in expectation


def star_schema(n_fact=10_000_000, dims=STAR_DIMS, s=1.1, seed=2):
    """Fact table F with one int32 foreign key per dimension, each Zipf(s) over
    its dimension's key space with ranks mapped to keys through a seeded random
    permutation; dimension D_i has a dense unique int32 key 0..|D_i|-1 and an
    int32 attribute uniform in [0, 1e9)."""
    rng = _rng(seed)
    fks, dim_rels = [], []
    for i, nd in enumerate(dims):
        perm = rng.permutation(nd)
        fks.append(perm[zipf_ranks(nd, s, n_fact, rng)].astype(np.int32))
        key = np.arange(nd, dtype=np.int32)
        attr = rng.integers(0, 1_000_000_000, size=nd, dtype=np.int64).astype(np.int32)
        dim_rels.append({"name": f"D{i + 1}", "cols": [key, attr]})
    fact = {"name": "F", "cols": fks}
    return fact, dim_rels


def star_query(fact, dim_rels, theta=STAR_THETA):
    """Q(k1..kd, a1..ad) :- F(k1..kd), D1(k1,a1), ..., Dd(kd,ad), with the
    selection a_i < theta pushed into each dimension atom.  Variables: k_i = i,
    a_i = d + i."""
    d = len(dim_rels)
    atoms = [atom(fact, list(range(d)))]
    for i, rel in enumerate(dim_rels):
        atoms.append(atom(rel, [i, d + i], preds=[(1, "<", theta)]))
    return atoms


# ---------------------------------------------------------------------------
# Batches of independent PK-FK queries
# ---------------------------------------------------------------------------

BATCH_THETA = 500_000_000  # payload uniform in [0, 1e9): keeps 50% in expectation


def _pk_relation(name, n, fk_targets, s, rng):
    """n rows: a dense unique key 0..n-1 (when this relation is referenced),
    one Zipf(s) foreign key per target size (ranks through a seeded
    permutation), and two int32 payload columns uniform in [0, 1e9)."""
    cols = [np.arange(n, dtype=np.int32)]
    for nt in fk_targets:
        perm = rng.permutation(nt)
        cols.append(perm[zipf_ranks(nt, s, n, rng)].astype(np.int32))
    for _ in range(2):
        cols.append(rng.integers(0, 1_000_000_000, size=n, dtype=np.int64).astype(np.int32))
    return {"name": name, "cols": cols}


def batch_query(q, min_rows=1_000, max_rows=2_000_000, base_seed=4):
    """Query q of the batched workload (seed base_seed + q): a chain or a star
    (q even: chain) of 2..6 relations with row counts log-uniform in
    [min_rows, max_rows]; every referenced relation has a dense unique key,
    foreign keys are Zipf(s) with s uniform in [0.5, 1.5], and the second
    payload column of every referenced relation carries the selection
    p2 < 5e8.  Returns (atoms, left-deep order, MIN variables): the MIN of
    the first payload column of every relation.

    Chain R1 -> R2 -> ... -> Rk: R1(a1, p), Ri(a_{i-1}, a_i, p, p2),
    Rk(a_{k-1}, p, p2).  Star F -> D1..D(k-1): F(a1..a(k-1), p),
    Di(ai, p, p2).  Key columns not referenced are left out of the atoms."""
    rng = _rng(base_seed + q)
    k = int(rng.integers(2, 7))
    s = float(rng.uniform(0.5, 1.5))
    sizes = [int(round(np.exp(rng.uniform(np.log(min_rows), np.log(max_rows))))) for _ in range(k)]
    atoms, mins = [], []
    nv = 0

    def fresh():
        nonlocal nv
        nv += 1
        return nv - 1

    if q % 2 == 0:  # chain
        link = [fresh() for _ in range(k - 1)]
        for i in range(k):
            targets = [sizes[i + 1]] if i + 1 < k else []
            rel = _pk_relation(f"Q{q}R{i + 1}", sizes[i], targets, s, rng)
            p, p2 = fresh(), fresh()
            mins.append(p)
            if i == 0:  # key, fk, p, p2 -> R1(a1, p)
                atoms.append(atom(rel, [link[0], p], rel_cols=[1, 2]))
            elif i + 1 < k:  # key, fk, p, p2
                atoms.append(atom(rel, [link[i - 1], link[i], p, p2], rel_cols=[0, 1, 2, 3],
                                  preds=[(3, "<", BATCH_THETA)]))
            else:  # key, p, p2
                atoms.append(atom(rel, [link[i - 1], p, p2], rel_cols=[0, 1, 2],
                                  preds=[(2, "<", BATCH_THETA)]))
    else:  # star
        link = [fresh() for _ in range(k - 1)]
        fact = _pk_relation(f"Q{q}F", sizes[0], sizes[1:], s, rng)
        p = fresh()
        fresh()
        mins.append(p)
        atoms.append(atom(fact, link + [p], rel_cols=list(range(1, k)) + [k]))
        for i in range(1, k):
            rel = _pk_relation(f"Q{q}D{i}", sizes[i], [], s, rng)
            p, p2 = fresh(), fresh()
            mins.append(p)
            atoms.append(atom(rel, [link[i - 1], p, p2], rel_cols=[0, 1, 2],
                              preds=[(2, "<", BATCH_THETA)]))
    return atoms, list(range(k)), mins


# ---------------------------------------------------------------------------
# Queries for the plan chooser: 5-relation snowflakes and 5-cycles with Zipf
# keys over a domain as large as the relation
# ---------------------------------------------------------------------------

def _zipf_col(n, domain, s, rng):
    perm = rng.permutation(domain)
    return perm[zipf_ranks(domain, s, n, rng)].astype(np.int32)


def chooser_query(q, min_rows=10_000, max_rows=50_000, base_seed=5, kind=None):
    """Query q (seed base_seed + q) for the chooser: a snowflake C(a,b),
    D1(a,c), D2(b,d), S1(c,e), S2(d,f) (q even) or a 5-cycle R1(a,b), R2(b,c),
    R3(c,d), R4(d,e), R5(e,a) (q odd), each relation with row count
    log-uniform in [min_rows, max_rows] and every column Zipf(s), s uniform
    in [0.8, 1.6], over a key domain of the relation's row count (through a
    seeded permutation).  Returns (atoms, kind)."""
    rng = _rng(base_seed + q)
    kind = kind or ("snowflake" if q % 2 == 0 else "cycle")
    s = float(rng.uniform(0.8, 1.6))
    if kind == "snowflake":
        shape = [[0, 1], [0, 2], [1, 3], [2, 4], [3, 5]]
    else:
        shape = [[0, 1], [1, 2], [2, 3], [3, 4], [4, 0]]
    atoms = []
    for i, vs in enumerate(shape):
        n = int(round(np.exp(rng.uniform(np.log(min_rows), np.log(max_rows)))))
        rel = {"name": f"C{q}R{i}", "cols": [_zipf_col(n, n, s, rng) for _ in vs]}
        atoms.append(atom(rel, vs))
    return atoms, kind


def chooser_pool(n_rel, min_rows=1_000_000, max_rows=16_000_000, seed=17):
    """n_rel two-column relations to compose chooser training queries from
    (pool_query): row count log-uniform in [min_rows, max_rows], each with
    its own Zipf exponent s uniform in [0.8, 1.6], both columns Zipf(s) over
    a key domain of the relation's row count through a seeded permutation
    (the columns of chooser_query)."""
    rng = _rng(seed)
    pool = []
    for i in range(n_rel):
        n = int(round(np.exp(rng.uniform(np.log(min_rows), np.log(max_rows)))))
        s = float(rng.uniform(0.8, 1.6))
        pool.append({"name": f"P{i}", "cols": [_zipf_col(n, n, s, rng) for _ in range(2)]})
    return pool


def pool_query(pool, q, base_seed=11):
    """Query q (seed base_seed + q) over the relations of a pool, with the
    shapes of chooser_query: a snowflake (q even) or a 5-cycle (q odd), each
    atom a different pool relation drawn at random, its two columns bound in
    random order.  Returns (atoms, kind)."""
    rng = _rng(base_seed + q)
    kind = "snowflake" if q % 2 == 0 else "cycle"
    if kind == "snowflake":
        shape = [[0, 1], [0, 2], [1, 3], [2, 4], [3, 5]]
    else:
        shape = [[0, 1], [1, 2], [2, 3], [3, 4], [4, 0]]
    idx = rng.choice(len(pool), len(shape), replace=False)
    atoms = []
    for i, vs in zip(idx, shape):
        cols = [0, 1] if rng.random() < 0.5 else [1, 0]
        atoms.append(atom(pool[int(i)], vs, rel_cols=cols))
    return atoms, kind


# ---------------------------------------------------------------------------
# Small random queries for property tests
# ---------------------------------------------------------------------------

def random_query(seed, max_atoms=4, max_rows=12, domain=4, max_vars=5, max_arity=3):
    """A random full conjunctive query over small relations drawn from a small
    value domain, so duplicates, skew and empty results all occur.  Every
    atom has distinct variables; relations are separate tables."""
    rng = _rng(seed)
    n_vars = int(rng.integers(1, max_vars + 1))
    n_atoms = int(rng.integers(1, max_atoms + 1))
    atoms = []
    used = set()
    for i in range(n_atoms):
        k = int(rng.integers(1, min(max_arity, n_vars) + 1))
        vars_ = [int(v) for v in rng.choice(n_vars, size=k, replace=False)]
        used |= set(vars_)
        n = int(rng.integers(0, max_rows + 1))
        cols = [rng.integers(0, domain, size=n).astype(np.int32) for _ in range(k)]
        preds = []
        if rng.random() < 0.25 and n:
            preds.append((int(rng.integers(0, k)), str(rng.choice(["<", "<=", ">", ">=", "==", "!="])),
                          int(rng.integers(0, domain))))
        atoms.append(atom({"name": f"R{i}", "cols": cols}, vars_, preds=preds))
    # Renumber variables densely in order of first appearance.
    ren = {}
    for a in atoms:
        for v in a["vars"]:
            ren.setdefault(v, len(ren))
    for a in atoms:
        a["vars"] = [ren[v] for v in a["vars"]]
    return atoms
