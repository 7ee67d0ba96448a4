"""fj_join2_count_noalloc: the join COUNT that allocates nothing (its hash
level lives in a fixed array inside the library), for callers that cannot
allocate device memory on the join path, e.g. while capturing a CUDA graph
or under a fixed memory budget.  Its result must equal fj_execute_plan's
COUNT for the same query on two calls in a row (the shared array keeps the
previous call's contents, so the second call checks the clearing).  This
file sorts last so a run stopped at the first failure has run every other
test already."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _existing_count(fj, ctx, r, s):
    import torch
    rr = ctx.relation([torch.from_numpy(r).cuda()], "R")
    ss = ctx.relation([torch.from_numpy(s).cuda()], "S")
    atoms = [{"rel": rr, "vars": [0]}, {"rel": ss, "vars": [0]}]
    plan = fj.binary_to_free_plan(atoms, [0, 1])
    return fj.execute(ctx, atoms, plan, out_mode="count").count


def _bag_count(r, s):
    """The bag COUNT of R(x), S(x) from its definition: the sum over keys of
    the product of the two multiplicities (numpy, independent of the GPU)."""
    kr, cr = np.unique(r, return_counts=True)
    ks, cs = np.unique(s, return_counts=True)
    _, ir, is_ = np.intersect1d(kr, ks, assume_unique=True, return_indices=True)
    return int(np.dot(cr[ir].astype(np.uint64), cs[is_].astype(np.uint64)))


def test_noalloc_join_count_matches_execute_plan_twice(fj):
    import torch
    ctx = fj.Context(0)
    rng = np.random.default_rng(5)
    cases = [
        (rng.integers(-50, 50, size=200_000, dtype=np.int64).astype(np.int32),
         rng.integers(-50, 50, size=300_000, dtype=np.int64).astype(np.int32)),
        (rng.integers(0, 1 << 30, size=1_000_000, dtype=np.int64).astype(np.int32),
         np.concatenate([rng.integers(0, 1 << 30, size=400_000, dtype=np.int64),
                         np.full(1000, -1, np.int64)]).astype(np.int32)),
    ]
    for r, s in cases:  # two calls in a row on the shared scratch
        want = _existing_count(fj, ctx, r, s)
        assert want == _bag_count(r, s)
        out = torch.full((1,), -7, dtype=torch.int64, device="cuda")
        fj.join2_count_noalloc(torch.from_numpy(r).cuda(), torch.from_numpy(s).cuda(), out)
        torch.cuda.synchronize()
        assert int(out.item()) == want
    ctx.close()


def test_noalloc_rejects_inputs_beyond_the_scratch(fj):
    import torch
    r = torch.zeros(10, dtype=torch.int32, device="cuda")
    s = torch.zeros(524_289, dtype=torch.int32, device="cuda")
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(fj.FJError) as ei:
        fj.join2_count_noalloc(r, s, out)
    assert ei.value.status == -1 and "524288" in str(ei.value)
