"""Training driver of the learned plan chooser.

The chooser itself lives in the library (include/fj.h): the features of a
candidate (left-deep order, cover policy) come from ``fj_plan_features``, the
candidate enumeration, the network's predictions and the argmin from
``fj_choose_plan``, the network's forward, backward and descent kernels from
``fj_model_*``, and ``FJ_COVER_LEARNED`` applies the network to the cover
policy of any prepared plan.  This module only marshals data for training:

* a training sample is a candidate of an engine-generated query, labelled
  with log2 of the work the exact engine does on it (cover elements
  iterated plus probes, from its counters; deterministic) or of the device
  time it takes;
* the network is pretrained on many small work-labelled queries and then
  fine-tuned on time-labelled queries at the scale it is used on (work is
  a poor proxy for time there: the candidate with the least work is often
  no faster than the declared plan);
* the network is trained on standardized features and labels by the
  library's own kernels, and its feature scaler is stored in the model
  (``Model.set_scaler``) so that the library can standardize by itself.

Every candidate gives the same result, so a wrong prediction costs time,
never exactness; without a model the chooser returns the declared order with
the static cover (the plain converted binary plan).
"""

from __future__ import annotations

import itertools

import numpy as np

IN_DIM = 137  # FJ_CHOOSER_IN_DIM
POLICIES = ("static", "fewest")


def connected_orders(atom_vars):
    """Every left-deep order whose prefixes are connected (no Cartesian
    product)."""
    sets = [set(v) for v in atom_vars]
    out = []
    for perm in itertools.permutations(range(len(atom_vars))):
        bound = set(sets[perm[0]])
        ok = True
        for a in perm[1:]:
            if not (sets[a] & bound):
                ok = False
                break
            bound |= sets[a]
        if ok:
            out.append(list(perm))
    return out


def training_candidates(atom_vars, n_orders, rng):
    """The declared order and up to n_orders - 1 random connected others,
    each with both cover policies."""
    m = len(atom_vars)
    declared = list(range(m))
    rest = [o for o in connected_orders(atom_vars) if o != declared]
    if len(rest) > n_orders - 1:
        rest = [rest[i] for i in sorted(rng.choice(len(rest), n_orders - 1, replace=False))]
    return [(o, p) for o in [declared] + rest for p in POLICIES]


def work(result):
    c = result.counters
    return c["cover_iters"] + c["probes"]


def samples(fj, ctx, dev_atoms, candidates, label="work", reps=2):
    """(features, label, count) of each candidate, run by the engine.  The
    label is log2 of the engine's work (``label="work"``: deterministic) or
    of its device time in microseconds (``label="time"``: the best of
    ``reps`` executions from scratch after a warm one, between CUDA events
    on the context's stream)."""
    import torch
    feats = fj.plan_features(ctx, dev_atoms, candidates)
    rows = []
    stream = torch.cuda.current_stream()
    for f, (order, pol) in zip(feats, candidates):
        plan = fj.binary_to_free_plan(dev_atoms, order, factor=True)
        if label == "work":
            r = fj.execute(ctx, dev_atoms, plan, out_mode="count", cover=pol)
            rows.append((f, np.log2(work(r) + 1.0), r.count))
            continue
        prep = fj.Prepared(ctx, dev_atoms, plan, out_mode="count", cover=pol)
        r = prep.execute()
        best = None
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            prep.reset()
            e0.record(stream)
            prep.execute_async()
            e1.record(stream)
            r = prep.result()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        prep.free()
        rows.append((f, np.log2(best * 1000.0 + 1.0), r.count))
    return rows


def init_params(n_in, h1, h2, seed=0):
    """He-normal weights, zero biases, in the model's parameter layout."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = [rng.normal(0, np.sqrt(2.0 / n_in), h1 * n_in), np.zeros(h1),
             rng.normal(0, np.sqrt(2.0 / h1), h2 * h1), np.zeros(h2),
             rng.normal(0, np.sqrt(1.0 / h2), h2), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)


def train(model, x, y, epochs=60, lr=0.03, batch=256, seed=0):
    """Plain gradient descent on the library's kernels, minibatches of
    `batch` rows (x, y float32 CUDA tensors, already standardized).  Returns
    the loss curve."""
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


def fit(fj, ctx, x, y, h1=128, h2=64, epochs=60, lr=0.03, seed=1, scaler_rows=None):
    """A model trained on (features, log2 cost) rows, with its feature
    scaler set (the library standardizes features itself when it chooses);
    the labels are standardized for training -- the argmin does not depend
    on that affine map.  The scaler is fitted on ``scaler_rows`` when given
    (every row the model will see, fine-tuning rows included: a feature
    that never varies in the first rows would otherwise blow up later),
    else on x.  Returns (model, losses); the scaler is also kept on the
    model object (``model.scaler``) for fine-tuning."""
    import torch
    x = np.asarray(x, dtype=np.float32)
    y = np.asarray(y, dtype=np.float32)
    xr = x if scaler_rows is None else np.asarray(scaler_rows, dtype=np.float32)
    mean, scale = xr.mean(axis=0), xr.std(axis=0) + 1e-3
    model = fj.Model(ctx, x.shape[1], h1, h2, max_batch=8192)
    model.set_params(init_params(x.shape[1], h1, h2, seed=seed))
    model.set_scaler(mean, scale)
    model.scaler = (mean, scale)
    xs = torch.from_numpy(((x - mean) / scale).astype(np.float32)).cuda()
    ys = torch.from_numpy(((y - y.mean()) / (y.std() + 1e-6)).astype(np.float32)).cuda()
    return model, train(model, xs, ys, epochs=epochs, lr=lr)


def finetune(model, x, y, epochs=40, lr=0.01):
    """Continue training a fitted model on new (features, log2 cost) rows --
    the time-labelled queries at the scale the chooser is used on -- under
    its existing feature scaler, with the new labels standardized on their
    own.  Returns the loss curve."""
    import torch
    mean, scale = model.scaler
    x = np.asarray(x, dtype=np.float32)
    y = np.asarray(y, dtype=np.float32)
    xs = torch.from_numpy(((x - mean) / scale).astype(np.float32)).cuda()
    ys = torch.from_numpy(((y - y.mean()) / (y.std() + 1e-6)).astype(np.float32)).cuda()
    return train(model, xs, ys, epochs=epochs, lr=lr, batch=128)
