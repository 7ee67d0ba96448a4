"""The bounded waits of the cooperative root build: with FJ_FLAG_TEST_TIMEOUT
its first grid barrier waits for a block that does not exist, every block
gives up after its spin limit, the execution fails with FJ_ERR_TIMEOUT
instead of hanging, and the same context then answers correctly."""

import pytest

from fjtest import device_atoms
from oracle import closed
from paper_2301_10841_gb300 import datagen as G

pytestmark = pytest.mark.gpu


def test_timeout_is_reported_and_the_context_recovers(fj, ctx):
    fact, dims = G.star_schema(n_fact=50_000, dims=(500, 1000, 2000, 4000), s=1.1, seed=6)
    theta = 300_000_000
    atoms = G.star_query(fact, dims, theta=theta)
    dev, _ = device_atoms(fj, ctx, atoms)
    plan = fj.binary_to_free_plan(dev, [0, 1, 2, 3, 4], factor=True)
    mins = [4, 5, 6, 7]
    with pytest.raises(fj.FJError) as ei:
        fj.execute(ctx, dev, plan, out_mode="count_min", min_vars=mins,
                   flags=fj.FLAG_TEST_TIMEOUT)
    assert ei.value.status == -6
    want = closed.star_join_direct(fact["cols"], [tuple(d["cols"]) for d in dims], [theta] * 4)
    got = fj.execute(ctx, dev, plan, out_mode="count_min", min_vars=mins)
    assert (got.count, got.mins) == want
    p = fj.Prepared(ctx, dev, plan, out_mode="count_min", min_vars=mins)
    for _ in range(2):
        p.reset()
        r = p.execute()
        assert (r.count, r.mins) == want
