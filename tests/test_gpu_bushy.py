"""Bushy plans (Section 2.2; the materialized intermediates of Section 5.2):
fj_execute_bushy against the oracle on random queries with random join
trees, the 4-cycle as (E1 E2)(E3 E4) against trace(A^4), and the star join
with a bushy dimension pair against direct addressing."""

import numpy as np
import pytest

import oracle
from oracle import closed
from paper_2301_10841_gb300 import datagen as G

from fjtest import device_atoms, sort_rows

pytestmark = pytest.mark.gpu


def _random_tree(atoms, rng):
    """A random binary join tree whose every subtree is connected (no
    Cartesian products inside an intermediate)."""
    sets = [set(a["vars"]) for a in atoms]
    items = [(i, set(s)) for i, s in enumerate(sets)]
    while len(items) > 1:
        pairs = [(i, j) for i in range(len(items)) for j in range(len(items))
                 if i != j and items[i][1] & items[j][1]]
        if not pairs:
            pairs = [(i, j) for i in range(len(items)) for j in range(len(items)) if i != j]
        i, j = pairs[int(rng.integers(len(pairs)))]
        t = ((items[i][0], items[j][0]), items[i][1] | items[j][1])
        items = [x for k, x in enumerate(items) if k not in (i, j)] + [t]
    return items[0][0]


def _is_bushy(t):
    return not isinstance(t, int) and (not isinstance(t[1], int) or _is_bushy(t[0]))


@pytest.mark.parametrize("seed", range(30))
def test_random_bushy_trees(fj, ctx, seed):
    atoms = G.random_query(1300 + seed, max_atoms=5, max_rows=25, domain=4, max_vars=5,
                           max_arity=2)
    rng = np.random.default_rng(seed)
    tree = _random_tree(atoms, rng)
    head = oracle.query_vars(atoms)
    want_c, want_m, want_t = oracle.binary_join(atoms, head=head, min_vars=head[:2],
                                                materialize=True)
    dev, _ = device_atoms(fj, ctx, atoms)
    got = fj.execute_bushy(ctx, dev, tree, head=head, out_mode="materialize")
    assert got.count == want_c, tree
    np.testing.assert_array_equal(sort_rows(got.tuples.cpu().numpy()), want_t)
    got = fj.execute_bushy(ctx, dev, tree, head=head, out_mode="count_min", min_vars=head[:2],
                           cover="fewest")
    assert (got.count, got.mins) == (want_c, want_m), tree


def test_four_cycle_bushy_against_trace(fj, ctx):
    e = G.uniform_digraph(300, 3000, seed=7)
    atoms = G.four_cycle_query(e)
    want = closed.trace_power(closed.adjacency(e["cols"][0], e["cols"][1], 300), 4)
    dev, _ = device_atoms(fj, ctx, atoms)
    for tree in [((0, 1), (2, 3)), (((0, 1), 2), 3), (0, (1, (2, 3)))]:
        assert fj.execute_bushy(ctx, dev, tree, out_mode="count").count == want, tree


def test_snowflake_bushy(fj, ctx):
    """A snowflake C(a,b), D1(a,c), D2(b,d), S1(c,e), S2(d,f) with its two
    branches joined first and then together: ((C D1) S1)(D2 S2)."""
    for q in (0, 2, 4):
        atoms, kind = G.chooser_query(q, 2_000, 8_000)
        assert kind == "snowflake"
        head = oracle.query_vars(atoms)
        want = oracle.binary_join(atoms, head=head, min_vars=head[:3])[:2]
        dev, _ = device_atoms(fj, ctx, atoms)
        for tree in [(((0, 1), 3), (2, 4)), (((2, 4), 0), (1, 3)), ((((0, 1), 3), 2), 4)]:
            got = fj.execute_bushy(ctx, dev, tree, head=head, out_mode="count_min",
                                   min_vars=head[:3], cover="fewest")
            assert (got.count, got.mins) == (want[0], want[1]), tree


def test_bushy_rejects_bad_trees(fj, ctx):
    atoms = G.random_query(5, max_atoms=3, max_rows=5, domain=3, max_vars=3, max_arity=2)
    dev, _ = device_atoms(fj, ctx, atoms)
    if len(atoms) < 2:
        atoms = G.triangle_query(G.uniform_digraph(20, 60, seed=1))
        dev, _ = device_atoms(fj, ctx, atoms)
    with pytest.raises(fj.FJError):
        fj.execute_bushy(ctx, dev, (0, 0), out_mode="count")  # an atom twice, one missing
