"""Several prepared plans with different expansion shared-memory needs
coexist: the dynamic shared-memory limit of a kernel is one setting for the
whole process, so preparing a plan that needs less must not lower it under
a plan prepared earlier that needs more."""

import pytest

import oracle
from fjtest import device_atoms
from paper_2301_10841_gb300 import datagen as G

pytestmark = pytest.mark.gpu


def test_plans_prepared_in_any_order_run(fj, ctx):
    e = G.uniform_digraph(400, 5000, seed=4)
    tri = G.triangle_query(e)
    dev, cache = device_atoms(fj, ctx, tri)
    # Three subatoms in node 0, then a two-relation path with two; at a
    # batch of 4096 (16 elements per thread) they need 128 KB and 112 KB of
    # dynamic shared memory, above the 48 KB default.
    big_plan = [[(0, (0, 1)), (1, (1,)), (2, (0,))], [(1, (2,)), (2, (2,))]]
    big = fj.Prepared(ctx, dev, big_plan, out_mode="count", batch_size=4096)
    path = [G.atom(e, [0, 1]), G.atom(e, [1, 2])]
    dpath, _ = device_atoms(fj, ctx, path, cache)
    small = fj.Prepared(ctx, dpath, fj.binary_to_free_plan(dpath, [0, 1]), out_mode="count",
                        batch_size=4096)
    assert big.execute().count == oracle.generic_join(tri)[0]
    assert small.execute().count == oracle.generic_join(path)[0]
    assert big.execute().count == oracle.generic_join(tri)[0]
