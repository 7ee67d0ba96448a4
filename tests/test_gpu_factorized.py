"""Factorized output (FJ_OUT_FACTORIZED; the trie-form result of Section
4.4): the union of products a prepared plan returns expands to exactly the
oracle's bag, its COUNT is the bag size, and on output-heavy queries it holds
far fewer rows than the flat listing."""

import numpy as np
import pytest

import oracle
from paper_2301_10841_gb300 import datagen as G

from fjtest import device_atoms, plans_for, sort_rows

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed", range(30))
def test_factorized_expands_to_the_bag(fj, ctx, seed):
    atoms = G.random_query(1700 + seed, max_atoms=4, max_rows=30, domain=4, max_vars=5,
                           max_arity=2)
    head = oracle.query_vars(atoms)
    want_c, _, want_t = oracle.binary_join(atoms, head=head, materialize=True)
    dev, _ = device_atoms(fj, ctx, atoms)
    rng = np.random.default_rng(seed)
    for name, plan in plans_for([a["vars"] for a in atoms], rng, n_orders=1):
        for cover in ("static", "fewest"):
            prep = fj.Prepared(ctx, dev, plan, head=head, out_mode="factorized", cover=cover)
            r = prep.execute()
            assert r.count == want_c, (name, cover)
            width, pre, tails = prep.factor_layout()
            assert r.tuples.shape[1] == width == len(pre) + 2 + 2 * len(tails)
            flat = prep.expand(r).cpu().numpy()
            np.testing.assert_array_equal(sort_rows(flat), want_t)
            prep.free()


def test_factorized_two_path_is_compact(fj, ctx):
    """Q(a,b,c) :- R(a,b), S(b,c) with heavy fan-out: the factorized result
    has one row per R row, the flat one |R| x deg(b) rows."""
    rng = np.random.default_rng(3)
    r = {"name": "R", "cols": [rng.integers(0, 5000, 4000).astype(np.int32),
                               rng.integers(0, 50, 4000).astype(np.int32)]}
    s = {"name": "S", "cols": [rng.integers(0, 50, 20000).astype(np.int32),
                               rng.integers(0, 10**6, 20000).astype(np.int32)]}
    atoms = [G.atom(r, [0, 1]), G.atom(s, [1, 2])]
    want_c, _, want_t = oracle.binary_join(atoms, head=[0, 1, 2], materialize=True)
    dev, _ = device_atoms(fj, ctx, atoms)
    plan = fj.binary_to_free_plan(dev, [0, 1], factor=True)
    prep = fj.Prepared(ctx, dev, plan, head=[0, 1, 2], out_mode="factorized")
    res = prep.execute()
    assert res.count == want_c
    assert res.tuples.shape[0] <= len(r["cols"][0])
    assert res.tuples.shape[0] * 50 < want_c
    np.testing.assert_array_equal(sort_rows(prep.expand(res).cpu().numpy()), want_t)
    with pytest.raises(fj.FJError):  # one-shot execution cannot keep the vectors
        fj.execute(ctx, dev, plan, out_mode="factorized")
