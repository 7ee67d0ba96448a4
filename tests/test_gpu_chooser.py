"""The learned plan chooser.

* The network's CUDA forward, backward and descent kernels against the
  float64 restatement in oracle/mlp.py (itself pinned by finite differences).
* The chooser trained on work the exact engine reports for engine-generated
  queries: on held-out queries its orders give exactly the results of the
  declared order (the converted binary plan, its fallback) and less work.
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


def _engine_samples(fj, ctx, queries):
    """(features, log2 work, count) of every candidate order of each query."""
    out = []
    for atoms, _ in queries:
        dev, _ = device_atoms(fj, ctx, atoms)
        hists = C.atom_histograms(ctx, atoms)
        orders = C.candidate_orders([a["vars"] for a in atoms])
        rows = []
        for o in orders:
            r = fj.execute(ctx, dev, fj.binary_to_free_plan(dev, o, factor=True),
                           out_mode="count")
            rows.append((C.order_features(atoms, o, hists), np.log2(C.work(r) + 1.0), r.count))
        out.append((atoms, dev, hists, orders, rows))
    return out


def test_chooser_gain(fj, ctx):
    import torch
    train_q = [G.chooser_query(q, 3_000, 20_000) for q in range(120)]
    test_q = [G.chooser_query(q, 20_000, 80_000) for q in range(1000, 1016)]
    train = _engine_samples(fj, ctx, train_q)
    for *_, rows in train:  # every order of a query gives the same count
        assert len({c for _, _, c in rows}) == 1
    x = np.stack([f for *_, rows in train for f, _, _ in rows])
    y = np.array([w for *_, rows in train for _, w, _ in rows], dtype=np.float32)
    scaler = C.fit_scaler(x)
    mu, sd = float(y.mean()), float(y.std() + 1e-6)
    model = fj.Model(ctx, C.IN_DIM, 128, 64, max_batch=8192)
    model.set_params(C.init_params(C.IN_DIM, 128, 64, seed=1))
    losses = C.train(model, torch.from_numpy(C.standardize(x, scaler)).cuda(),
                     torch.from_numpy((y - mu) / sd).cuda())
    assert losses[-1] < 0.6 * losses[0]
    tot_declared = tot_chosen = tot_best = 0.0
    for atoms, dev, hists, orders, rows in _engine_samples(fj, ctx, test_q):
        chosen = C.choose(model, atoms, orders, hists, scaler)
        i = orders.index(chosen)
        assert rows[i][2] == rows[0][2]          # bit-exact whatever it picks
        tot_declared += rows[0][1]
        tot_chosen += rows[i][1]
        tot_best += min(w for _, w, _ in rows)
    print(f"log2 work summed over held-out queries: declared {tot_declared:.1f}, "
          f"chosen {tot_chosen:.1f}, best {tot_best:.1f}")
    assert tot_chosen < tot_declared
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
