"""Batches of independent PK-FK chain and star queries (fj_batch_*): every
query's COUNT and MINs equal the oracle's hash join of the same query, run
eagerly, as one captured CUDA graph and as one graph of concurrent branches
(each replayed twice); a query whose
output size the host would decide (materialized output) is refused with
FJ_ERR_UNSUPPORTED."""

import pytest

import oracle
from fjtest import device_atoms
from paper_2301_10841_gb300 import datagen as G

pytestmark = pytest.mark.gpu


def test_batch_matches_oracle(fj, ctx):
    preps, want = [], []
    for q in range(48):
        atoms, order, mins = G.batch_query(q, max_rows=60_000)
        c, m, _ = oracle.binary_join(atoms, order=order, min_vars=mins)
        want.append((c, m))
        dev, _ = device_atoms(fj, ctx, atoms)
        plan = fj.binary_to_free_plan(dev, order, factor=True)
        preps.append(fj.Prepared(ctx, dev, plan, out_mode="count_min", min_vars=mins))
    assert len(preps) == 48
    for graph, conc in ((False, False), (True, False), (True, True)):
        b = fj.Batch(ctx, preps, graph=graph, concurrent=conc)
        for _ in range(2):
            got = [(r.count, r.mins) for r in b.execute()]
            assert got == want, (graph, conc)
        b.free()
    # A prepared query still runs on its own after the batches (the
    # concurrent capture's settings are put back).
    for p, w in zip(preps[:4], want[:4]):
        p.reset()
        r = p.execute()
        assert (r.count, r.mins) == w
    with pytest.raises(fj.FJError):
        fj.Batch(ctx, preps, graph=False, concurrent=True)


def test_batch_refuses_host_decisions(fj, ctx):
    atoms, order, mins = G.batch_query(0, max_rows=5_000)  # chain
    dev, _ = device_atoms(fj, ctx, atoms)
    plan = fj.binary_to_free_plan(dev, order, factor=True)
    ok = fj.Prepared(ctx, dev, plan, out_mode="count_min", min_vars=mins)
    m = fj.Prepared(ctx, dev, plan, out_mode="materialize")
    with pytest.raises(fj.FJError) as ei:
        fj.Batch(ctx, [ok, m])
    assert ei.value.status == -8 and "batch query 1" in str(ei.value)


def test_prepared_keeps_its_relations(fj, ctx):
    """A prepared query borrows device columns: it must keep the relations
    alive after the caller drops them (the allocator would reuse them)."""
    import gc

    import torch

    def make():
        atoms, order, mins = G.batch_query(1, max_rows=20_000)
        dev, _ = device_atoms(fj, ctx, atoms)
        plan = fj.binary_to_free_plan(dev, order, factor=True)
        want = oracle.binary_join(atoms, order=order, min_vars=mins)[:2]
        return fj.Prepared(ctx, dev, plan, out_mode="count_min", min_vars=mins), want

    p, want = make()
    gc.collect()
    junk = [torch.full((1 << 20,), 7, dtype=torch.int32, device="cuda") for _ in range(8)]
    r = p.execute()
    assert (r.count, r.mins) == want
    del junk



def test_autotuner_picks_the_fastest_candidate(fj, ctx):
    """The autotuner times every (cover-batch size, load factor) candidate
    -- {256, 1024, 4096, 8192} x {0.25, 0.5, 0.7} -- and keeps the one with
    the shortest time, configured as chosen; whatever it picks gives the
    oracle's COUNT and MINs."""
    for q in (0, 1, 5):
        atoms, order, mins = G.batch_query(q, max_rows=200_000)
        want = oracle.binary_join(atoms, order=order, min_vars=mins)[:2]
        dev, _ = device_atoms(fj, ctx, atoms)
        plan = fj.binary_to_free_plan(dev, order, factor=True)
        times = {}
        p, cfg, ms = fj.autotune(ctx, dev, plan, out_mode="count_min", min_vars=mins,
                                 times=times)
        assert set(times) == {(b, l) for b in (256, 1024, 4096, 8192) for l in (0.25, 0.5, 0.7)}
        assert ms == min(times.values()) and times[cfg] == ms
        assert (p.batch_size, p.load_factor) == cfg
        p.reset()
        r = p.execute()
        assert (r.count, r.mins) == tuple(want)
        p.free()
