"""GPU parity on the launch configurations and sizes the benchmarks use:

* the star join at its full size (10M fact rows), in the launch sequence
  bench.py times (prepared plan, reset + asynchronous execution, timing
  events), against the direct-address semi-join;
* random queries with three-column keys over every hash-level load factor
  {0.25, 0.5, 0.7} and cover-batch size {256, 1024, 8192} the autotuner
  offers, against the oracle's sorted bag, COUNT and MIN;
* the batched PK-FK workload at its real sizes (up to 2M rows per
  relation), graph-captured, against direct-address key lookups.
"""

import numpy as np
import pytest

import oracle
from oracle import closed
from paper_2301_10841_gb300 import datagen as G

from fjtest import device_atoms, plans_for, sort_rows

pytestmark = pytest.mark.gpu


def test_star_join_full_size_as_benchmarked(fj, ctx):
    import torch
    fact, dims = G.star_schema(n_fact=10_000_000, dims=G.STAR_DIMS, s=1.1, seed=2)
    atoms = G.star_query(fact, dims, theta=G.STAR_THETA)
    want = closed.star_join_direct(fact["cols"], [tuple(d["cols"]) for d in dims],
                                   [G.STAR_THETA] * 4)
    dev, _ = device_atoms(fj, ctx, atoms)
    plan = fj.binary_to_free_plan(dev, [0, 1, 2, 3, 4], factor=True)
    mins = [4, 5, 6, 7]
    prep = fj.Prepared(ctx, dev, plan, out_mode="count_min", min_vars=mins, batch_size=1024,
                       flags=fj.FLAG_TIMING)
    for _ in range(3):
        prep.reset()
        prep.execute_async()
        got = prep.result()
        assert (got.count, got.mins) == want
    torch.cuda.synchronize()
    got = fj.execute(ctx, dev, plan, out_mode="count_min", min_vars=mins)
    assert (got.count, got.mins) == want
    got = fj.execute(ctx, dev, plan, out_mode="count_min", min_vars=mins, cover="fewest")
    assert (got.count, got.mins) == want
    prep.free()


@pytest.mark.parametrize("seed", range(16))
def test_random_wide_keys_every_load_and_batch(fj, ctx, seed):
    atoms = G.random_query(900 + seed, max_atoms=4, max_rows=60, domain=5, max_vars=5,
                           max_arity=3)
    atom_vars = [a["vars"] for a in atoms]
    rng = np.random.default_rng(seed)
    head = oracle.query_vars(atoms)
    mins = head[:2]
    want_c, want_m, want_t = oracle.binary_join(atoms, head=head, min_vars=mins,
                                                materialize=True)
    dev, _ = device_atoms(fj, ctx, atoms)
    for name, plan in plans_for(atom_vars, rng, n_orders=1):
        for lf in (0.25, 0.5, 0.7):
            for bs in (256, 1024, 8192):
                for cover in ("static", "fewest"):
                    got = fj.execute(ctx, dev, plan, head=head, out_mode="materialize",
                                     cover=cover, batch_size=bs, load_factor=lf)
                    assert got.count == want_c, (name, lf, bs, cover)
                    np.testing.assert_array_equal(sort_rows(got.tuples.cpu().numpy()), want_t)
                    got = fj.execute(ctx, dev, plan, head=head, out_mode="count_min",
                                     min_vars=mins, cover=cover, batch_size=bs, load_factor=lf)
                    assert (got.count, got.mins) == (want_c, want_m), (name, lf, bs, cover)


def test_wide_three_column_levels_larger(fj, ctx):
    """Three-column hash levels below the root (wide 32-byte slots) on
    inputs large enough to span many blocks and probe chains."""
    rng = np.random.default_rng(77)
    n = 200_000
    r = {"name": "R", "cols": [rng.integers(0, 40, n).astype(np.int32) for _ in range(4)]}
    s = {"name": "S", "cols": [rng.integers(0, 40, n // 4).astype(np.int32) for _ in range(3)]}
    atoms = [G.atom(r, [0, 1, 2, 3]), G.atom(s, [1, 2, 3])]
    want = oracle.binary_join(atoms, min_vars=[0, 3])[:2]
    dev, _ = device_atoms(fj, ctx, atoms)
    plans = [fj.binary_to_free_plan(dev, [0, 1]), fj.binary_to_free_plan(dev, [1, 0]),
             [[(0, (0,))], [(0, (1, 2, 3)), (1, (1, 2, 3))]],
             [[(1, (1,)), (0, (1,))], [(1, (2, 3)), (0, (2, 3))], [(0, (0,))]]]
    for plan in plans:
        for lf in (0.25, 0.7):
            for cover in ("static", "fewest"):
                got = fj.execute(ctx, dev, plan, out_mode="count_min", min_vars=[0, 3],
                                 cover=cover, load_factor=lf)
                assert (got.count, got.mins) == want, (plan, lf, cover)


def test_batched_workload_real_sizes(fj, ctx):
    """Queries of the batched workload at up to 2M rows per relation, run as
    one graph-captured batch with several cover-batch sizes and load
    factors, each against closed.pkfk_direct."""
    import torch
    picks = list(range(0, 256, 16))
    preps, wants = [], []
    cfgs = [(256, 0.25), (1024, 0.5), (8192, 0.7), (4096, 0.25)]
    keep = []
    for i, q in enumerate(picks):
        atoms, order, mins = G.batch_query(q, max_rows=2_000_000)
        wants.append(closed.pkfk_direct(atoms, mins))
        dev, cache = device_atoms(fj, ctx, atoms)
        keep.append(cache)
        plan = fj.binary_to_free_plan(dev, order, factor=True)
        bs, lf = cfgs[i % len(cfgs)]
        preps.append(fj.Prepared(ctx, dev, plan, out_mode="count_min", min_vars=mins,
                                 batch_size=bs, load_factor=lf))
    for conc in (False, True):
        batch = fj.Batch(ctx, preps, graph=True, concurrent=conc)
        for _ in range(2):
            res = batch.execute()
            for q, r, w in zip(picks, res, wants):
                assert (r.count, r.mins) == w, (q, conc)
        batch.free()
    for p, w in zip(preps, wants):
        p.reset()
        r = p.execute()
        assert (r.count, r.mins) == w
        p.free()
    torch.cuda.synchronize()


def test_star_join_from_host_columns(fj, ctx):
    """Relations copied from host memory (fj_load_relation_host, pinned and
    pageable sources alike) give the direct-address star join's COUNT and
    MINs."""
    import torch
    fact, dims = G.star_schema(n_fact=3_000_007, dims=(1000, 2500, 5000, 10_000), s=1.1, seed=5)
    want = closed.star_join_direct(fact["cols"], [tuple(d["cols"]) for d in dims],
                                   [G.STAR_THETA] * 4)
    for pinned in (True, False):
        def host(cols):
            ts = [torch.from_numpy(np.ascontiguousarray(c)) for c in cols]
            return [t.pin_memory() for t in ts] if pinned else ts
        rels = {r["name"]: ctx.relation_host(host(r["cols"]), r["name"]) for r in [fact] + dims}
        q = G.star_query(fact, dims, theta=G.STAR_THETA)
        atoms = [{"rel": rels[a["rel"]["name"]], "vars": a["vars"], "preds": a["preds"]}
                 for a in q]
        plan = fj.binary_to_free_plan(atoms, [0, 1, 2, 3, 4], factor=True)
        r = fj.execute(ctx, atoms, plan, out_mode="count_min", min_vars=[4, 5, 6, 7])
        assert (r.count, r.mins) == want, pinned
        for h in rels.values():
            h.release()


def test_star_join_first_probe_bitmap_and_its_fallback(fj, ctx):
    """The first probe of the one-launch scan tests an exact key bitmap when
    every key of its root level lies in the bitmap's range (D1's keys
    0..39,999), and falls back to the Bloom filter and hash lookup when one
    does not (the same keys times 7: up to 279,993, past the 262,144 bits);
    both give the direct-address star join's COUNT and MINs, executed twice
    on one prepared plan."""
    fact, dims = G.star_schema(n_fact=500_000, dims=(40_000, 2500, 5000, 10_000), s=1.1, seed=9)
    for scale in (1, 7):
        f = dict(fact, cols=[fact["cols"][0] * scale] + list(fact["cols"][1:]))
        d = [dict(dims[0], cols=[dims[0]["cols"][0] * scale, dims[0]["cols"][1]])] + dims[1:]
        want = closed.star_join_direct(f["cols"], [tuple(x["cols"]) for x in d],
                                       [G.STAR_THETA] * 4)
        atoms = G.star_query(f, d, theta=G.STAR_THETA)
        dev, _ = device_atoms(fj, ctx, atoms)
        plan = fj.binary_to_free_plan(dev, list(range(5)), factor=True)
        p = fj.Prepared(ctx, dev, plan, out_mode="count_min", min_vars=[4, 5, 6, 7])
        for _ in range(2):
            p.reset()
            r = p.execute()
            assert (r.count, r.mins) == want, scale
        p.free()
