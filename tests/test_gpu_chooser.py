"""The learned plan chooser.

* The network's CUDA forward, backward and descent kernels against the
  float64 restatement in oracle/mlp.py (itself pinned by finite differences).
* The chooser's features, plan choice, model file and learned cover policy
  through the C ABI (fj_plan_features, fj_choose_plan, fj_model_save/load,
  FJ_COVER_LEARNED).
* The chooser trained on work the exact engine reports for engine-generated
  queries: on held-out queries its choices give exactly the results of the
  declared order (the converted binary plan, its fallback) with less work
  than it and no more than the fewest-keys cover.
"""

import numpy as np
import pytest

from fjtest import device_atoms
from oracle import mlp
from paper_2301_10841_gb300 import chooser as C
from paper_2301_10841_gb300 import datagen as G

pytestmark = pytest.mark.gpu


def test_model_kernels_match_oracle(fj, ctx):
    """Forward within 1e-5 relative to each output's magnitude (the sum of
    the absolute values of its terms, mlp.magnitudes); every gradient
    element against the float64 chain rule and a float32 CPU backprop within
    1e-4 of its own magnitude, and against central finite differences of the
    float64 loss within 1e-3 relative; descent steps follow float64."""
    import torch
    d, h1, h2, n = C.IN_DIM, 128, 64, 700
    rng = np.random.default_rng(11)
    theta = C.init_params(d, h1, h2, seed=3)
    x = rng.normal(0, 1, (n, d)).astype(np.float32)
    t = rng.normal(0, 1, n).astype(np.float32)
    m = fj.Model(ctx, d, h1, h2, max_batch=1024)
    assert m.n_params == mlp.n_params(d, h1, h2)
    m.set_params(theta)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    th64 = theta.astype(np.float64)
    y = m.forward(xd).cpu().numpy().astype(np.float64)
    want, _ = mlp.forward(th64, x, d, h1, h2)
    ymag, gmag = mlp.magnitudes(th64, x, t, d, h1, h2)
    assert np.all(np.abs(y - want) <= 1e-5 * ymag), np.max(np.abs(y - want) / ymag)
    g, loss = m.gradients(xd, td)
    g = g.astype(np.float64)
    g64 = mlp.gradients(th64, x, t, d, h1, h2)
    g32 = mlp.gradients(theta, x, t, d, h1, h2, dtype=np.float32).astype(np.float64)
    tiny = 1e-12
    assert np.all(np.abs(g - g64) <= 1e-4 * gmag + tiny), np.max(np.abs(g - g64) / (gmag + tiny))
    assert np.all(np.abs(g - g32) <= 1e-4 * gmag + tiny), np.max(np.abs(g - g32) / (gmag + tiny))
    assert abs(loss - mlp.loss(th64, x, t, d, h1, h2)) <= 1e-5 * loss
    # Central finite differences of the float64 loss, every parameter of a
    # smaller network (the same kernels, other shapes).
    ds, hs1, hs2, ns = 24, 16, 8, 48
    ths = C.init_params(ds, hs1, hs2, seed=5) + np.float32(0.01)
    xs = rng.normal(0, 1, (ns, ds)).astype(np.float32)
    ts = rng.normal(0, 1, ns).astype(np.float32)
    ms = fj.Model(ctx, ds, hs1, hs2, max_batch=64)
    ms.set_params(ths)
    gs, _ = ms.gradients(torch.from_numpy(xs).cuda(), torch.from_numpy(ts).cuda())
    th = ths.astype(np.float64)
    eps = 1e-6
    fd = np.empty_like(th)
    for i in range(len(th)):
        e = np.zeros_like(th)
        e[i] = eps
        fd[i] = (mlp.loss(th + e, xs, ts, ds, hs1, hs2) -
                 mlp.loss(th - e, xs, ts, ds, hs1, hs2)) / (2 * eps)
    floor = 1e-3 * np.max(np.abs(fd))
    rel = np.abs(gs - fd) / np.maximum(np.abs(fd), floor)
    assert np.all(rel < 1e-3), (np.argmax(rel), rel.max())
    ms.free()
    # Twenty descent steps follow the float64 trajectory.
    th = th64
    for _ in range(20):
        l_gpu = m.train_step(xd, td, 0.01)
        l_cpu, th = mlp.sgd_step(th, x, t, d, h1, h2, 0.01)
        assert abs(l_gpu - l_cpu) <= 1e-4 * l_cpu
    np.testing.assert_allclose(m.params(), th, rtol=1e-3, atol=1e-5)
    with pytest.raises(fj.FJError):
        m.forward(torch.zeros((1025, d), device="cuda"))
    m.free()


def _features_by_definition(fj, ctx, atoms, order, policy):
    """The documented feature layout (include/fj.h, FJ_CHOOSER_IN_DIM),
    written out here from fj.degree_histogram and the row counts."""
    import torch
    sets = [set(a["vars"]) for a in atoms]
    n_vars = len(set().union(*sets))
    cyclic = sum(len(v) for v in sets) - n_vars >= len(atoms)
    f, bound = [], set()
    for pos in range(4):
        if pos >= len(order):
            f.extend([0.0] * 33)
            continue
        a = order[pos]
        with_ = (sets[order[1]] if len(order) > 1 else set()) if pos == 0 else bound
        j = next((k for k, v in enumerate(atoms[a]["vars"]) if v in with_), 0)
        col = torch.from_numpy(np.ascontiguousarray(atoms[a]["cols"][j])).cuda()
        f.append(np.log2(len(atoms[a]["cols"][0]) + 1.0) / 32.0)
        f.extend(fj.degree_histogram(ctx, col, mod=100, seed=31 * a + j))
        bound |= sets[a]
    f.extend([len(order) / 8.0, n_vars / 32.0, float(cyclic), 1.0,
              1.0 if policy == "fewest" else 0.0])
    return np.asarray(f, dtype=np.float32)


def test_plan_features_follow_their_definition(fj, ctx):
    rng = np.random.default_rng(3)
    for q in range(4):
        atoms, _ = G.chooser_query(q, 2_000, 9_000)
        dev, _ = device_atoms(fj, ctx, atoms)
        cands = C.training_candidates([a["vars"] for a in atoms], 3, rng)
        got = fj.plan_features(ctx, dev, cands)
        assert got.shape == (len(cands), fj.CHOOSER_IN_DIM)
        for row, (order, pol) in zip(got, cands):
            want = _features_by_definition(fj, ctx, atoms, order, pol)
            np.testing.assert_allclose(row, want, rtol=1e-6, atol=1e-7)
    with pytest.raises(fj.FJError):
        fj.plan_features(ctx, dev, [([0, 0, 1, 2, 3], "static")])


def test_choose_plan_without_model_is_the_converted_binary_plan(fj, ctx):
    atoms, _ = G.chooser_query(1, 2_000, 5_000)
    dev, _ = device_atoms(fj, ctx, atoms)
    plan, pol, order = fj.choose_plan(ctx, dev, None)
    assert order == list(range(len(atoms))) and pol == "static"
    assert plan == fj.binary_to_free_plan(dev, order, factor=True)


def test_model_save_load_and_learned_cover(fj, ctx, tmp_path):
    """A saved model loads with the same parameters, scaler and predictions;
    FJ_COVER_LEARNED runs the policy the model predicts cheaper for the
    plan, and its results equal the oracle's."""
    import torch

    import oracle
    rng = np.random.default_rng(5)
    d = fj.CHOOSER_IN_DIM
    m = fj.Model(ctx, d, 32, 16, max_batch=64)
    m.set_params(C.init_params(d, 32, 16, seed=7))
    mean = rng.normal(0, 0.1, d).astype(np.float32)
    scale = rng.uniform(0.5, 2.0, d).astype(np.float32)
    m.set_scaler(mean, scale)
    path = tmp_path / "chooser.fjm"
    m.save(path)
    m2 = fj.Model.load(ctx, path, max_batch=64)
    np.testing.assert_array_equal(m2.params(), m.params())
    x = rng.normal(0, 1, (40, d)).astype(np.float32)
    xs = torch.from_numpy((x - mean) / scale).cuda()
    np.testing.assert_array_equal(m2.forward(xs).cpu().numpy(), m.forward(xs).cpu().numpy())
    (tmp_path / "bad.fjm").write_bytes(b"not a model")
    with pytest.raises(fj.FJError):
        fj.Model.load(ctx, tmp_path / "bad.fjm")
    for q in range(6):
        atoms, _ = G.chooser_query(q, 2_000, 6_000)
        dev, _ = device_atoms(fj, ctx, atoms)
        plan = fj.binary_to_free_plan(dev, list(range(len(atoms))), factor=True)
        want = oracle.binary_join(atoms)[0]
        got = fj.execute(ctx, dev, plan, out_mode="count", cover="learned", model=m2)
        assert got.count == want
        f = fj.plan_features(ctx, dev, [(list(range(len(atoms))), p) for p in C.POLICIES])
        pred = m2.forward(torch.from_numpy((f - mean) / scale).cuda()).cpu().numpy()
        assert got.counters["cover_policy"] == (1 if pred[1] < pred[0] else 0)
    with pytest.raises(fj.FJError):
        fj.execute(ctx, dev, plan, out_mode="count", cover="learned")  # no model
    m.free()
    m2.free()


def test_chooser_gain(fj, ctx):
    """Trained on the engine's work for generated queries, the chooser
    (fj_choose_plan: order and cover policy together) does less work on
    held-out queries than the plain converted binary plan and no more than
    the fewest-keys cover alone, with identical results."""
    rng = np.random.default_rng(0)
    xs, ys = [], []
    for q in range(160):
        atoms, _ = G.chooser_query(q, 3_000, 20_000)
        dev, _ = device_atoms(fj, ctx, atoms)
        rows = C.samples(fj, ctx, dev, C.training_candidates([a["vars"] for a in atoms], 6, rng))
        assert len({c for _, _, c in rows}) == 1  # every candidate gives the same count
        xs += [f for f, _, _ in rows]
        ys += [w for _, w, _ in rows]
    model, losses = C.fit(fj, ctx, np.stack(xs), np.array(ys))
    assert losses[-1] < 0.6 * losses[0]
    tot = {"plain": 0.0, "fewest": 0.0, "learned": 0.0}
    for q in range(1000, 1024):
        atoms, _ = G.chooser_query(q, 20_000, 80_000)
        dev, _ = device_atoms(fj, ctx, atoms)
        declared = fj.binary_to_free_plan(dev, list(range(len(atoms))), factor=True)
        plan, pol, _ = fj.choose_plan(ctx, dev, model)
        runs = {"plain": fj.execute(ctx, dev, declared, out_mode="count"),
                "fewest": fj.execute(ctx, dev, declared, out_mode="count", cover="fewest"),
                "learned": fj.execute(ctx, dev, plan, out_mode="count", cover=pol)}
        assert len({r.count for r in runs.values()}) == 1  # bit-exact whatever it picks
        for k, r in runs.items():
            tot[k] += np.log2(C.work(r) + 1.0)
    print("log2 work summed over held-out queries:", {k: round(v, 1) for k, v in tot.items()})
    assert tot["learned"] < tot["plain"]
    assert tot["learned"] <= tot["fewest"]
    model.free()


def test_chooser_time_gain(fj, ctx):
    """Trained on device times of queries composed from a pool of relations
    of 300K-3M rows, the chooser (order and cover policy together) runs
    held-out queries -- generated apart, with their own relations -- in less
    time than the plain converted binary plan and than the fewest-keys
    cover, with identical results.  Each candidate is timed as the best of
    three executions from scratch between CUDA events."""
    import torch
    pool = G.chooser_pool(16, 300_000, 3_000_000, seed=23)
    dpool = {r["name"]: ctx.relation([torch.from_numpy(c).cuda() for c in r["cols"]])
             for r in pool}
    rng = np.random.default_rng(1)
    xs, ys = [], []
    for q in range(120):
        atoms, _ = G.pool_query(pool, q, base_seed=3000)
        dev = [{"rel": dpool[a["rel"]["name"]], "vars": a["vars"], "rel_cols": a["rel_cols"]}
               for a in atoms]
        rows = C.samples(fj, ctx, dev, C.training_candidates([a["vars"] for a in atoms], 6, rng),
                         label="time")
        assert len({c for _, _, c in rows}) == 1
        xs += [f for f, _, _ in rows]
        ys += [t for _, t, _ in rows]
    for r in dpool.values():
        r.release()
    model, losses = C.fit(fj, ctx, np.stack(xs), np.array(ys))
    assert losses[-1] < 0.6 * losses[0]
    stream = torch.cuda.current_stream()

    def best_ms(prep):
        best = None
        for _ in range(3):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            prep.reset()
            e0.record(stream)
            prep.execute_async()
            e1.record(stream)
            prep.result()
            t = e0.elapsed_time(e1)
            best = t if best is None else min(best, t)
        return best

    tot = {"plain": 0.0, "fewest": 0.0, "learned": 0.0}
    for q in range(2100, 2108):
        atoms, _ = G.chooser_query(q, 300_000, 3_000_000)
        dev, _ = device_atoms(fj, ctx, atoms)
        declared = fj.binary_to_free_plan(dev, list(range(len(atoms))), factor=True)
        plan, pol, _ = fj.choose_plan(ctx, dev, model)
        preps = {"plain": fj.Prepared(ctx, dev, declared, out_mode="count"),
                 "fewest": fj.Prepared(ctx, dev, declared, out_mode="count", cover="fewest"),
                 "learned": fj.Prepared(ctx, dev, plan, out_mode="count", cover=pol)}
        counts = {k: p.execute().count for k, p in preps.items()}
        assert len(set(counts.values())) == 1  # bit-exact whatever it picks
        for k, p in preps.items():
            tot[k] += best_ms(p)
            p.free()
        for a in dev:
            a["rel"].release()
    print("ms summed over held-out queries:", {k: round(v, 2) for k, v in tot.items()})
    assert tot["learned"] < tot["plain"]
    assert tot["learned"] <= tot["fewest"]
    model.free()


def test_degree_histogram_kernel_matches_oracle(fj, ctx):
    import torch

    from oracle import stats
    for seed, (n, s, mod) in enumerate([(50_000, 1.2, 100), (20_000, 0.8, 7), (3_000, 1.6, 1)]):
        rng = np.random.default_rng(seed)
        col = G.zipf_ranks(n // 3, s, n, rng).astype(np.int32) - (n // 6)
        got = fj.degree_histogram(ctx, torch.from_numpy(col).cuda(), mod=mod, seed=seed)
        want = stats.degree_histogram(col, mod=mod, seed=seed)
        np.testing.assert_allclose(got, want, rtol=1e-6, atol=1e-7)
    empty = fj.degree_histogram(ctx, torch.zeros(0, dtype=torch.int32, device="cuda"))
    assert not empty.any()
