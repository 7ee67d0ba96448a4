"""The learned plan chooser: picks the left-deep join order that binary2fj
converts into the Free Join plan, by predicting each candidate's work with
the library's three-layer perceptron (fj.Model, trained by the library's
own CUDA kernels) from sampled degree histograms.

* Features of a candidate order (in_dim = 4 * 33 + 4): for each of its
  first four relations, log2 of the row count and the 32-bucket histogram of
  log2 key degrees of the column it joins on (fj.degree_histogram: a seeded,
  counter-based 1% sample, on the GPU), then four shape scalars.
* Label: log2 of the work the exact engine does on the plan (cover elements
  iterated plus probes, from its counters) -- deterministic, unlike a time.
* Choice: the candidate with the smallest prediction; without a model, the
  declared order (the converted binary plan) is the fallback.  Every order
  gives the same result, so a wrong prediction costs time, never exactness.
"""

from __future__ import annotations

import itertools

import numpy as np

N_BUCKETS = 32
POSITIONS = 4
IN_DIM = POSITIONS * (N_BUCKETS + 1) + 4


def atom_histograms(ctx, atoms, seed=0):
    """{(atom index, variable): the sampled key-degree histogram of that
    atom's column (1% sample), from the library's kernel}."""
    import torch

    from paper_2301_10841_gb300 import fj
    out = {}
    for i, a in enumerate(atoms):
        for j, v in enumerate(a["vars"]):
            col = torch.from_numpy(np.ascontiguousarray(a["cols"][j], dtype=np.int32)).cuda()
            out[(i, v)] = fj.degree_histogram(ctx, col, mod=100, seed=seed + 31 * i + j)
    return out


def candidate_orders(atom_vars, limit=24, seed=0):
    """Left-deep orders whose every prefix is connected (no Cartesian
    product), the declared order first; at most `limit` (seeded sample)."""
    m = len(atom_vars)
    sets = [set(v) for v in atom_vars]
    out = []
    for perm in itertools.permutations(range(m)):
        bound = set(sets[perm[0]])
        ok = True
        for a in perm[1:]:
            if not (sets[a] & bound):
                ok = False
                break
            bound |= sets[a]
        if ok:
            out.append(list(perm))
    declared = list(range(m))
    rest = [o for o in out if o != declared]
    rng = np.random.Generator(np.random.PCG64(seed))
    if len(rest) > limit - 1:
        rest = [rest[i] for i in sorted(rng.choice(len(rest), limit - 1, replace=False))]
    return [declared] + rest


def order_features(atoms, order, hists):
    sets = [set(a["vars"]) for a in atoms]
    cyclic = sum(len(s) for s in sets) - len(set().union(*sets)) >= len(atoms)
    f = []
    bound = set()
    for pos in range(POSITIONS):
        if pos < len(order):
            a = order[pos]
            vs = atoms[a]["vars"]
            if pos == 0:
                nxt = sets[order[1]] if len(order) > 1 else set()
                join = [v for v in vs if v in nxt] or vs
            else:
                join = [v for v in vs if v in bound] or vs
            f.append(np.log2(len(atoms[a]["cols"][0]) + 1.0) / 32.0)
            f.extend(hists[(a, join[0])])
            bound |= sets[a]
        else:
            f.extend([0.0] * (N_BUCKETS + 1))
    f.extend([len(order) / 8.0, len(set().union(*sets)) / 32.0, float(cyclic), 1.0])
    return np.asarray(f, dtype=np.float32)


def work(result):
    c = result.counters
    return c["cover_iters"] + c["probes"]


def init_params(n_in, h1, h2, seed=0):
    """He-normal weights, zero biases, in the model's parameter layout."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = [rng.normal(0, np.sqrt(2.0 / n_in), h1 * n_in), np.zeros(h1),
             rng.normal(0, np.sqrt(2.0 / h1), h2 * h1), np.zeros(h2),
             rng.normal(0, np.sqrt(1.0 / h2), h2), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)


def train(model, x, y, epochs=60, lr=0.03, batch=256, seed=0):
    """Plain gradient descent on the library's kernels, minibatches of
    `batch` rows (x, y float32 CUDA tensors).  Returns the loss curve."""
    import torch
    n = x.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    losses = []
    for _ in range(epochs):
        perm = torch.randperm(n, generator=g).to(x.device)
        ep = 0.0
        for i in range(0, n, batch):
            idx = perm[i:i + batch]
            ep += model.train_step(x[idx], y[idx], lr) * len(idx)
        losses.append(ep / n)
    return losses


def fit_scaler(x):
    """Per-feature mean and spread of the training rows (the network sees
    standardized features)."""
    x = np.asarray(x, dtype=np.float32)
    return x.mean(axis=0), x.std(axis=0) + 1e-3


def standardize(x, scaler):
    return ((np.asarray(x, dtype=np.float32) - scaler[0]) / scaler[1]).astype(np.float32)


def choose(model, atoms, orders, hists, scaler):
    """The candidate order with the smallest predicted work (the first order,
    the converted binary plan, when no model is given)."""
    import torch
    if model is None:
        return orders[0]
    feats = standardize(np.stack([order_features(atoms, o, hists) for o in orders]), scaler)
    pred = model.forward(torch.from_numpy(feats).cuda()).cpu().numpy()
    return orders[int(np.argmin(pred))]
