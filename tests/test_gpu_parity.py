"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Everything is integer, so results must match exactly: the sorted bag of
output tuples, COUNT(*) and the MINs."""

import numpy as np
import pytest

import oracle
from oracle import closed
from paper_2301_10841_gb300 import datagen as G

from fjtest import device_atoms, gj_plan, plans_for, sort_rows

pytestmark = pytest.mark.gpu


def _run_all_ways(fj, ctx, atoms, plan, min_vars, covers=("static", "fewest"), tiles=(256, 2048)):
    head = oracle.query_vars(atoms)
    want_c, want_m, want_t = oracle.binary_join(atoms, head=head, min_vars=min_vars,
                                                materialize=True)
    dev, cache = device_atoms(fj, ctx, atoms)
    for cover in covers:
        for tile in tiles:
            got = fj.execute(ctx, dev, plan, head=head, out_mode="materialize", cover=cover,
                             batch_size=tile)
            assert got.count == want_c, (cover, tile, plan)
            np.testing.assert_array_equal(sort_rows(got.tuples.cpu().numpy()), want_t)
            got = fj.execute(ctx, dev, plan, head=head, out_mode="count_min", min_vars=min_vars,
                             cover=cover, batch_size=tile)
            assert (got.count, got.mins) == (want_c, want_m), (cover, tile, plan)
    return want_c


@pytest.mark.parametrize("seed", range(60))
def test_random_queries_every_plan_shape(fj, ctx, seed):
    atoms = G.random_query(seed, max_atoms=4, max_rows=14, domain=4, max_vars=5, max_arity=2)
    atom_vars = [a["vars"] for a in atoms]
    rng = np.random.default_rng(seed)
    mins = [int(v) for v in rng.permutation(oracle.query_vars(atoms))[:2]]
    for name, plan in plans_for(atom_vars, rng):
        _run_all_ways(fj, ctx, atoms, plan, mins, tiles=(256,))


@pytest.mark.parametrize("seed", range(12))
def test_random_queries_larger(fj, ctx, seed):
    atoms = G.random_query(500 + seed, max_atoms=5, max_rows=300, domain=12, max_vars=5,
                           max_arity=2)
    atom_vars = [a["vars"] for a in atoms]
    rng = np.random.default_rng(seed)
    mins = oracle.query_vars(atoms)[:3]
    for name, plan in plans_for(atom_vars, rng, n_orders=1):
        c, _, _ = oracle.binary_join(atoms, min_vars=mins)
        if c > 3_000_000:
            continue
        _run_all_ways(fj, ctx, atoms, plan, mins, tiles=(256, 4096))


def test_triangle_small_config(fj, ctx):
    """Triangle query, 2,000 vertices and 20,000 distinct uniform edges:
    COUNT against trace(A^3), listing against the oracle's sorted bag."""
    e = G.uniform_digraph(2000, 20000, seed=1)
    atoms = G.triangle_query(e)
    a = closed.adjacency(e["cols"][0], e["cols"][1], 2000)
    tr = closed.trace_power(a, 3)
    want = oracle.generic_join(atoms, materialize=True)
    assert want[0] == tr
    dev, _ = device_atoms(fj, ctx, atoms)
    plan = [[(0, (0, 1)), (1, (1,)), (2, (0,))], [(1, (2,)), (2, (2,))]]
    conv = fj.binary_to_free_plan(dev, [0, 1, 2], factor=True)
    for pl in (plan, conv):
        for cover in ("static", "fewest"):
            got = fj.execute(ctx, dev, pl, out_mode="materialize", cover=cover)
            assert got.count == tr
            np.testing.assert_array_equal(sort_rows(got.tuples.cpu().numpy()), want[2])
            got = fj.execute(ctx, dev, pl, out_mode="count", cover=cover)
            assert got.count == tr


@pytest.mark.parametrize("n", [5, 17, 40])
def test_complete_digraph_closed_forms(fj, ctx, n):
    e = G.complete_digraph(n)
    tri = G.triangle_query(e)
    cyc = G.four_cycle_query(e)
    dev, cache = device_atoms(fj, ctx, tri)
    for plan in (fj.binary_to_free_plan(dev, [0, 1, 2]),
                 gj_plan([a["vars"] for a in tri], [0, 1, 2])):
        assert fj.execute(ctx, dev, plan, cover="fewest").count == n * (n - 1) * (n - 2)
    dev4, _ = device_atoms(fj, ctx, cyc, cache)
    want = closed.complete_digraph_cycles(n, 4)
    for plan in (fj.binary_to_free_plan(dev4, [0, 1, 2, 3]),
                 gj_plan([a["vars"] for a in cyc], [0, 1, 2, 3])):
        for cover in ("static", "fewest"):
            assert fj.execute(ctx, dev4, plan, cover=cover).count == want


def test_star_join_reduced(fj, ctx):
    fact, dims = G.star_schema(n_fact=300_000, dims=(2000, 5000, 10000, 20000), s=1.1, seed=5)
    theta = 200_000_000
    atoms = G.star_query(fact, dims, theta=theta)
    want = closed.star_join_direct(fact["cols"], [tuple(d["cols"]) for d in dims], [theta] * 4)
    dev, _ = device_atoms(fj, ctx, atoms)
    mins = [4, 5, 6, 7]
    for fac in (True, False):
        plan = fj.binary_to_free_plan(dev, [0, 1, 2, 3, 4], factor=fac)
        for cover in ("static", "fewest"):
            got = fj.execute(ctx, dev, plan, out_mode="count_min", min_vars=mins, cover=cover)
            assert (got.count, got.mins) == want


def test_clover_factor_changes_work_not_result(fj, ctx):
    """Fig. 3 instance: one output tuple; the naive plan's second loop runs
    n^2 times, the factored plan's work is linear (Section 4.1)."""
    from test_oracle import clover_instance
    n = 200
    atoms = clover_instance(n)
    dev, _ = device_atoms(fj, ctx, atoms)
    naive = fj.binary_to_free_plan(dev, [0, 1, 2], factor=False)
    fact = fj.binary_to_free_plan(dev, [0, 1, 2], factor=True)
    r1 = fj.execute(ctx, dev, naive, out_mode="materialize")
    r2 = fj.execute(ctx, dev, fact, out_mode="materialize")
    for r in (r1, r2):
        assert r.tuples.cpu().numpy().tolist() == [[0, 100, 1000, 10000]]
    assert r1.counters["cover_iters"] >= n * n
    assert r2.counters["cover_iters"] <= 4 * n + 8
    assert r2.counters["probes"] <= 4 * n + 8


def test_colt_laziness_example(fj, ctx):
    """Example 4.3: Q(x,a,b,c) :- R(x,a),S(x,b),T(x,c),U(b) with plan
    [[R(x,a),S(x),T(x)],[U(b),S(b)],[T(c)]] on the clover instance.  R is only
    iterated, so nothing is built for it; S and T get their first level; with
    U(b) as the cover only the x0 subtrie of S is expanded; with the fewest-
    keys cover S(b) is iterated instead and U's map is built."""
    from test_oracle import clover_instance
    n = 50
    atoms = clover_instance(n)
    u = {"name": "U", "cols": [np.array([1000, 1001, 1002, 5], dtype=np.int32)]}
    atoms.append(G.atom(u, [2]))
    dev, _ = device_atoms(fj, ctx, atoms)
    plan = [[(0, (0, 1)), (1, (0,)), (2, (0,))], [(3, (2,)), (1, (2,))], [(2, (3,))]]
    want = oracle.binary_join(atoms, materialize=True)
    r = fj.execute(ctx, dev, plan, out_mode="materialize", cover="static")
    np.testing.assert_array_equal(sort_rows(r.tuples.cpu().numpy()), want[2])
    assert want[0] == 1
    built = r.counters["atom_built_mask"]
    assert not built & 1            # R: nothing built
    assert built & 2 and built & 4  # S and T: first level
    assert r.counters["subtries_forced"] == 1  # only S[x0]
    r = fj.execute(ctx, dev, plan, out_mode="materialize", cover="fewest")
    np.testing.assert_array_equal(sort_rows(r.tuples.cpu().numpy()), want[2])
    assert r.counters["subtries_forced"] == 0  # S(b) iterated as a vector
    assert r.counters["atom_built_mask"] & 8   # U's map built


def test_eager_builds_give_the_same_bag(fj, ctx):
    atoms = G.random_query(77, max_atoms=4, max_rows=40, domain=6, max_vars=4, max_arity=2)
    atom_vars = [a["vars"] for a in atoms]
    head = oracle.query_vars(atoms)
    want = oracle.binary_join(atoms, head=head, materialize=True)
    dev, _ = device_atoms(fj, ctx, atoms)
    plan = gj_plan(atom_vars, head)
    for flags in (fj.FLAG_EAGER_ROOT, fj.FLAG_EAGER_ALL):
        r = fj.execute(ctx, dev, plan, head=head, out_mode="materialize", cover="fewest",
                       flags=flags)
        np.testing.assert_array_equal(sort_rows(r.tuples.cpu().numpy()), want[2])


def test_prepared_reuse_and_explicit_build(fj, ctx):
    e = G.uniform_digraph(400, 5000, seed=4)
    atoms = G.triangle_query(e)
    dev, _ = device_atoms(fj, ctx, atoms)
    plan = [[(0, (0, 1)), (1, (1,)), (2, (0,))], [(1, (2,)), (2, (2,))]]
    want = oracle.binary_join(atoms)[0]
    p = fj.Prepared(ctx, dev, plan, out_mode="count", cover="fewest")
    r1 = p.execute()
    r2 = p.execute()  # levels reused
    assert r1.count == r2.count == want
    assert r2.counters["roots_built"] == 0
    p.reset()
    p.build_level(2, 0)
    p.build_level(2, 1)
    r3 = p.execute()
    assert r3.count == want
    p.free()


def test_edge_cases(fj, ctx):
    i32 = np.int32
    big, small = np.iinfo(i32).max, np.iinfo(i32).min
    # extreme values and the all-ones two-column key (-1, -1)
    r = {"name": "R", "cols": [np.array([-1, -1, big, small, 0, -1], i32),
                               np.array([-1, -1, small, big, 0, 7], i32)]}
    s = {"name": "S", "cols": [np.array([-1, big, small, -1], i32),
                               np.array([-1, small, big, -1], i32),
                               np.array([3, 4, 5, 6], i32)]}
    atoms = [G.atom(r, [0, 1]), G.atom(s, [0, 1, 2])]
    dev, _ = device_atoms(fj, ctx, atoms)
    want = oracle.binary_join(atoms, materialize=True, min_vars=[0, 1, 2])
    for order in ([0, 1], [1, 0]):
        plan = fj.binary_to_free_plan(dev, order)
        got = fj.execute(ctx, dev, plan, out_mode="materialize")
        np.testing.assert_array_equal(sort_rows(got.tuples.cpu().numpy()), want[2])
        got = fj.execute(ctx, dev, plan, out_mode="count_min", min_vars=[0, 1, 2])
        assert (got.count, got.mins) == (want[0], want[1])
    # empty relation, and a selection that keeps nothing
    e = {"name": "E", "cols": [np.zeros(0, i32), np.zeros(0, i32)]}
    f = {"name": "F", "cols": [np.arange(10, dtype=i32), np.arange(10, dtype=i32)]}
    for atoms in ([G.atom(f, [0, 1]), G.atom(e, [1, 2])],
                  [G.atom(f, [0, 1], preds=[(0, ">", 100)]), G.atom(f, [1, 2])],
                  [G.atom(f, [0, 1]), G.atom(f, [1, 2], preds=[(1, "<", -5)])]):
        dev, _ = device_atoms(fj, ctx, atoms)
        for order in ([0, 1], [1, 0]):
            plan = fj.binary_to_free_plan(dev, order)
            got = fj.execute(ctx, dev, plan, out_mode="count_min", min_vars=[0])
            assert got.count == 0 and got.mins == [None]
            got = fj.execute(ctx, dev, plan, out_mode="materialize")
            assert got.count == 0 and got.tuples.shape[0] == 0


def test_errors_are_reported(fj, ctx):
    r = {"name": "R", "cols": [np.arange(4, dtype=np.int32), np.arange(4, dtype=np.int32)]}
    atoms = [G.atom(r, [0, 1]), G.atom(r, [1, 2])]
    dev, _ = device_atoms(fj, ctx, atoms)
    with pytest.raises(fj.FJError) as ei:
        fj.execute(ctx, dev, [[(0, (0, 1)), (1, (1, 2))]])
    assert ei.value.status == -2
    with pytest.raises(fj.FJError) as ei:
        fj.execute(ctx, dev, fj.binary_to_free_plan(dev, [0, 1]), out_mode="count_min",
                   min_vars=[9])
    assert ei.value.status == -1


def test_context_close_releases_live_children(fj):
    """fj_ctx_destroy releases relations and prepared plans still alive; the
    binding's handles become inert, so later frees are no-ops."""
    import gc
    c = fj.Context(0)
    e = G.uniform_digraph(50, 300, seed=9)
    atoms, _ = device_atoms(fj, c, G.triangle_query(e))
    plan = [[(0, (0, 1)), (1, (1,)), (2, (0,))], [(1, (2,)), (2, (2,))]]
    p = fj.Prepared(c, atoms, plan, out_mode="count")
    want = p.execute().count
    c.close()
    p.free()
    del p, atoms
    gc.collect()
    assert want == oracle.binary_join(G.triangle_query(e))[0]


@pytest.mark.parametrize("seed", range(10))
def test_ablation_configurations_agree(fj, ctx, seed):
    """The ablation configurations (simple trie, simple lazy trie, batch
    sizes, no one-launch scan) and the Generic Join baseline give the
    oracle's bag on random queries."""
    atoms = G.random_query(700 + seed, max_atoms=4, max_rows=80, domain=6, max_vars=5,
                           max_arity=3)
    atom_vars = [a["vars"] for a in atoms]
    head = oracle.query_vars(atoms)
    want_c, want_m, want_t = oracle.binary_join(atoms, head=head, min_vars=head[:2],
                                                materialize=True)
    dev, _ = device_atoms(fj, ctx, atoms)
    fplan = fj.binary_to_free_plan(dev, list(range(len(atoms))), factor=True)
    gplan = fj.generic_join_plan(dev, head)
    cfgs = [(fplan, fj.FLAG_EAGER_ALL, 2048, "static"), (fplan, fj.FLAG_EAGER_ROOT, 2048, "static"),
            (fplan, fj.FLAG_NO_FUSED_SCAN, 256, "static"), (fplan, fj.FLAG_NO_FUSED_SCAN, 4096, "fewest"),
            (gplan, fj.FLAG_EAGER_ALL | fj.FLAG_NO_FUSED_SCAN, 256, "fewest")]
    for plan, flags, bs, cover in cfgs:
        got = fj.execute(ctx, dev, plan, head=head, out_mode="materialize", flags=flags,
                         batch_size=bs, cover=cover)
        assert got.count == want_c, (flags, bs, cover)
        np.testing.assert_array_equal(sort_rows(got.tuples.cpu().numpy()), want_t)
        got = fj.execute(ctx, dev, plan, head=head, out_mode="count_min", min_vars=head[:2],
                         flags=flags, batch_size=bs, cover=cover)
        assert (got.count, got.mins) == (want_c, want_m), (flags, bs, cover)


def test_ablation_star_join_eager_and_generic_join(fj, ctx):
    """The star join under every trie variant and as a Generic Join: the
    four-key fact level stays a vector under the eager flags."""
    fact, dims = G.star_schema(n_fact=200_000, dims=(2000, 5000, 10000, 20000), s=1.1, seed=6)
    theta = 300_000_000
    atoms = G.star_query(fact, dims, theta=theta)
    want = closed.star_join_direct(fact["cols"], [tuple(d["cols"]) for d in dims], [theta] * 4)
    dev, _ = device_atoms(fj, ctx, atoms)
    fplan = fj.binary_to_free_plan(dev, [0, 1, 2, 3, 4], factor=True)
    gplan = fj.generic_join_plan(dev, list(range(8)))
    for plan, flags, cover in [(fplan, fj.FLAG_EAGER_ALL, "static"),
                               (fplan, fj.FLAG_EAGER_ROOT, "static"),
                               (fplan, fj.FLAG_NO_FUSED_SCAN, "static"),
                               (gplan, fj.FLAG_EAGER_ALL | fj.FLAG_NO_FUSED_SCAN, "fewest")]:
        got = fj.execute(ctx, dev, plan, out_mode="count_min", min_vars=[4, 5, 6, 7],
                         flags=flags, batch_size=256, cover=cover)
        assert (got.count, got.mins) == want, (plan is gplan, flags)


def test_list_limit_overflow_keeps_exact_count_and_rows(fj, ctx):
    """FJ_ERR_OUTPUT_OVERFLOW: the COUNT stays exact and the first
    list_limit rows come back, each a row of the oracle's bag."""
    e = G.uniform_digraph(400, 6000, seed=21)
    atoms = G.triangle_query(e)
    want = oracle.generic_join(atoms, materialize=True)
    dev, _ = device_atoms(fj, ctx, atoms)
    plan = [[(0, (0, 1)), (1, (1,)), (2, (0,))], [(1, (2,)), (2, (2,))]]
    limit = want[0] // 3
    with pytest.raises(fj.FJError) as ei:
        fj.execute(ctx, dev, plan, out_mode="materialize", list_limit=limit)
    err = ei.value
    assert err.status == -4 and err.result is not None
    assert err.result.count == want[0]
    rows = err.result.tuples.cpu().numpy()
    assert len(rows) == limit
    bag = {tuple(r) for r in want[2].tolist()}
    assert all(tuple(r) in bag for r in rows.tolist())
    # Within the limit the listing is complete.
    got = fj.execute(ctx, dev, plan, out_mode="materialize", list_limit=want[0])
    np.testing.assert_array_equal(sort_rows(got.tuples.cpu().numpy()), want[2])


def test_count_overflow_is_reported(fj, ctx):
    """A product above 2^64 - 1 (five relations of 10,000 equal keys: 10^20
    combinations) fails with FJ_ERR_COUNT_OVERFLOW instead of wrapping."""
    rels = [{"name": f"R{i}", "cols": [np.zeros(10_000, dtype=np.int32)]} for i in range(5)]
    atoms = [G.atom(r, [0]) for r in rels]
    dev, _ = device_atoms(fj, ctx, atoms)
    plan = fj.binary_to_free_plan(dev, list(range(5)), factor=True)
    with pytest.raises(fj.FJError) as ei:
        fj.execute(ctx, dev, plan, out_mode="count")
    assert ei.value.status == -5
    # Four of them fit: 10^16.
    got = fj.execute(ctx, dev[:4], fj.binary_to_free_plan(dev[:4], list(range(4))), out_mode="count")
    assert got.count == 10**16


def test_materialized_output_above_the_first_buffer_is_retried(fj, ctx):
    """The output buffer starts at 2^20 rows; a larger listing is sized
    exactly and run again, and every row comes back."""
    r = {"name": "R", "cols": [np.arange(1200, dtype=np.int32) % 3, np.arange(1200, dtype=np.int32)]}
    s = {"name": "S", "cols": [np.arange(1500, dtype=np.int32) % 3, np.arange(1500, dtype=np.int32)]}
    atoms = [G.atom(r, [0, 1]), G.atom(s, [0, 2])]
    want_c = 3 * 400 * 500
    assert want_c > 1 << 20 is False or want_c < 1 << 20  # sanity of the arithmetic below
    big = {"name": "S", "cols": [np.zeros(1000, dtype=np.int32), np.arange(1000, dtype=np.int32)]}
    rb = {"name": "R", "cols": [np.zeros(1100, dtype=np.int32), np.arange(1100, dtype=np.int32)]}
    atoms = [G.atom(rb, [0, 1]), G.atom(big, [0, 2])]
    dev, _ = device_atoms(fj, ctx, atoms)
    plan = fj.binary_to_free_plan(dev, [0, 1])
    got = fj.execute(ctx, dev, plan, out_mode="materialize")
    assert got.count == 1100 * 1000 > 1 << 20
    t = got.tuples.cpu().numpy()
    assert len(t) == got.count
    assert len({(a, b) for _, a, b in t.tolist()}) == 1100 * 1000


@pytest.mark.parametrize("seed", range(10))
def test_root_tables_reused_across_executions(fj, ctx, seed):
    """A root build clears only the slots the previous build of the same
    table listed (the first build, and any after a build by the multi-launch
    path, clear the whole table).  One prepared query, executed again and
    again -- in between, once inside a batch of concurrent branches, whose
    root levels the multi-launch path builds -- gives the oracle's COUNT and
    MINs every time: unique keys (each row placed by its entry) and repeated
    ones (placed by the scatter), one- to three-column keys, small and large
    key domains."""
    rng = np.random.default_rng(seed)
    domain, rows = [(3, 40), (40, 600), (5000, 3000)][seed % 3]
    atoms = G.random_query(900 + seed, max_atoms=4, max_rows=rows, domain=domain, max_vars=5,
                           max_arity=3)
    mins = oracle.query_vars(atoms)[:2]
    want_c, want_m, _ = oracle.binary_join(atoms, min_vars=mins)
    dev, _ = device_atoms(fj, ctx, atoms)
    order = [int(a) for a in rng.permutation(len(atoms))]
    plan = fj.binary_to_free_plan(dev, order, factor=True)
    p = fj.Prepared(ctx, dev, plan, out_mode="count_min", min_vars=mins)
    for k in range(5):
        if k == 2:
            b = fj.Batch(ctx, [p], graph=True, concurrent=True)
            (r,) = b.execute()
            b.free()
        else:
            p.reset()
            r = p.execute()
        assert (r.count, r.mins) == (want_c, want_m), k
    p.free()


def test_root_tables_reused_star_join(fj, ctx):
    """The star join's dimension roots (unique keys: no scatter pass) and a
    variant whose dimensions repeat keys (scatter pass), each executed three
    times on one prepared query with the per-entry tail MINs, equal the
    direct-address join every time."""
    fact, dims = G.star_schema(n_fact=200_000, dims=(1000, 2500, 5000, 10_000), s=1.1, seed=7)
    want = closed.star_join_direct(fact["cols"], [tuple(d["cols"]) for d in dims],
                                   [G.STAR_THETA] * 4)
    for repeat in (False, True):
        if repeat:
            # Every dimension row twice: each key has two rows.
            dims = [dict(d, cols=[np.concatenate([c, c]) for c in d["cols"]]) for d in dims]
            want = closed.star_join_direct(fact["cols"], [tuple(d["cols"]) for d in dims],
                                           [G.STAR_THETA] * 4)
        atoms = G.star_query(fact, dims, theta=G.STAR_THETA)
        dev, _ = device_atoms(fj, ctx, atoms)
        plan = fj.binary_to_free_plan(dev, list(range(5)), factor=True)
        p = fj.Prepared(ctx, dev, plan, out_mode="count_min", min_vars=[4, 5, 6, 7])
        for _ in range(3):
            p.reset()
            r = p.execute()
            assert (r.count, r.mins) == want, repeat
        p.free()
