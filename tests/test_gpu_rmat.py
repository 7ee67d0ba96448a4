"""Cyclic queries on seeded R-MAT graphs (a, b, c = 0.57, 0.19, 0.19; 16
edges per vertex, self-loops and duplicates removed).

* Scales 14-18: exact triangle counts against the stored oracle counts in
  golden/rmat_counts.json (written by golden/make_rmat_counts.py from the
  oracle's Generic Join alone), for every plan shape and both cover
  policies; 4-cycles at scales 14 and 16 against the oracle's 2-path form
  (which equals the Generic Join count at scale 14).
* Full size (2^20 vertices, 2^24 edges): the oracle cannot enumerate it in
  seconds, so the test checks what holds at any size -- every valid plan
  gives the same triangle count, the triangles with x below a cutoff that
  leaves at most LIST_LIMIT of them are listed exactly once each (count of
  the listing = the count query with the same selection), and a sample of
  the listed rows, checked one by one against the edge set, are triangles;
  the listings below two small cutoffs equal the oracle's
  (golden/rmat_listing.json, written by golden/make_rmat_listing.py from
  the oracle's hash join alone).
"""

import json
import os

import numpy as np
import pytest

from fjtest import device_atoms, gj_plan, sort_rows
from paper_2301_10841_gb300 import datagen as G

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
# The triangle plan printed in Section 3.3 (Q_tri with R, S, T = E1, E2, E3).
TRI_PLAN = [[(0, (0, 1)), (1, (1,)), (2, (0,))], [(1, (2,)), (2, (2,))]]
LIST_LIMIT = 100_000_000  # the first 100M triangles (config 3)
FOUR_CYCLE_MAX_SCALE = 16  # 4-cycle counts checked up to this scale


@pytest.fixture(scope="module")
def golden():
    with open(os.path.join(HERE, "golden", "rmat_counts.json")) as f:
        return json.load(f)["graphs"]


def test_rmat_counts_match_oracle(fj, ctx, golden):
    for g in golden:
        e = G.rmat(g["scale"], g["n_edges"], seed=g["seed"])
        tri = G.triangle_query(e)
        dev, cache = device_atoms(fj, ctx, tri)
        for plan in (TRI_PLAN, fj.binary_to_free_plan(dev, [0, 1, 2]),
                     gj_plan([a["vars"] for a in tri], [0, 1, 2])):
            for cover in ("static", "fewest"):
                got = fj.execute(ctx, dev, plan, out_mode="count", cover=cover).count
                assert got == g["triangles"], (g["scale"], plan, cover)
        if "four_cycles" in g and "four_cycles_two_paths" in g:
            # the two oracle paths (enumeration, sparse 2-path products) agree
            assert g["four_cycles"] == g["four_cycles_two_paths"]
        want4 = g.get("four_cycles", g.get("four_cycles_two_paths"))
        if want4 is not None and g["scale"] <= FOUR_CYCLE_MAX_SCALE:
            cyc = G.four_cycle_query(e)
            dev4, _ = device_atoms(fj, ctx, cyc, cache)
            plans = [fj.binary_to_free_plan(dev4, [0, 1, 2, 3])]
            if g["scale"] <= 14:
                plans.append(gj_plan([a["vars"] for a in cyc], [0, 1, 2, 3]))
            for plan in plans:
                got = fj.execute(ctx, dev4, plan, out_mode="count", cover="fewest").count
                assert got == want4, (g["scale"], plan)


def _with_x_below(atoms, theta):
    """The triangle atoms with the selection x < theta on E1(x, y) and
    E3(z, x) (variable 0 is x)."""
    out = []
    for a in atoms:
        b = dict(a)
        b["preds"] = [(a["vars"].index(0), "<", int(theta))] if 0 in a["vars"] else []
        out.append(b)
    return out


def test_rmat_full_scale_triangles(fj, ctx):
    import torch
    e = G.rmat(20, 16 << 20, seed=3)
    tri = G.triangle_query(e)
    dev, _ = device_atoms(fj, ctx, tri)
    counts = {fj.execute(ctx, dev, plan, out_mode="count", cover=cover).count
              for plan in (TRI_PLAN, fj.binary_to_free_plan(dev, [0, 1, 2]))
              for cover in ("static", "fewest")}
    assert len(counts) == 1
    total = counts.pop()
    assert total > LIST_LIMIT

    # Largest cutoff theta (a vertex id) whose prefix x < theta holds at most
    # LIST_LIMIT triangles, by bisection on count queries.
    lo, hi = 0, int(max(e["cols"][0].max(), e["cols"][1].max())) + 1
    while hi - lo > 1:
        mid = (lo + hi) // 2
        c = fj.execute(ctx, _with_x_below(dev, mid), TRI_PLAN, out_mode="count",
                       cover="fewest").count
        lo, hi = (mid, hi) if c <= LIST_LIMIT else (lo, mid)
    sel = _with_x_below(dev, lo)
    want = fj.execute(ctx, sel, TRI_PLAN, out_mode="count", cover="fewest").count
    assert 0 < want <= LIST_LIMIT
    got = fj.execute(ctx, sel, TRI_PLAN, out_mode="materialize", cover="fewest")
    assert got.count == want
    rows = got.tuples  # (want, 3) int32 on the device: x, y, z
    assert rows.shape == (want, 3)
    assert bool((rows[:, 0] < lo).all())
    # Each listed exactly once: no two rows equal.
    key = (rows[:, 0].long() << 42) | (rows[:, 1].long() << 21) | rows[:, 2].long()
    assert torch.unique(key).numel() == want
    # A sample, one by one against the edge set.
    src, dst = e["cols"]
    codes = np.sort(src.astype(np.int64) << 32 | dst.astype(np.int64))

    def has(u, v):
        c = (np.int64(u) << 32) | np.int64(v)
        i = np.searchsorted(codes, c)
        return i < len(codes) and codes[i] == c

    rng = np.random.default_rng(7)
    sample = rows[torch.from_numpy(rng.integers(0, want, 2000)).cuda()].cpu().numpy()
    for x, y, z in sample:
        assert has(x, y) and has(y, z) and has(z, x)


def test_rmat_full_scale_listing_against_oracle(fj, ctx):
    """The listing of the triangles with x below a cutoff on the full-size
    graph equals the oracle's (tests/golden/rmat_listing.json, written by
    make_rmat_listing.py from the oracle alone): count, SHA-256 of the
    sorted rows, first and last rows."""
    import hashlib
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "rmat_listing.json")) as f:
        gold = json.load(f)["listings"]
    e = G.rmat(20, 16 << 20, seed=3)
    dev, _ = device_atoms(fj, ctx, G.triangle_query(e))
    for rec in gold:
        sel = _with_x_below(dev, rec["cutoff"])
        for plan in (TRI_PLAN, fj.binary_to_free_plan(sel, [0, 1, 2])):
            got = fj.execute(ctx, sel, plan, out_mode="materialize", cover="fewest")
            assert got.count == rec["count"]
            rows = np.ascontiguousarray(sort_rows(got.tuples.cpu().numpy()), dtype="<i4")
            assert rows[:5].tolist() == rec["first"] and rows[-5:].tolist() == rec["last"]
            assert hashlib.sha256(rows.tobytes()).hexdigest() == rec["sha256"]
