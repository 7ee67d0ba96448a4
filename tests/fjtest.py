"""Helpers shared by the GPU tests: move datagen relations to the device,
build binding atoms, generate plans, and compare with the oracle."""

import numpy as np

from oracle import plan as P


def device_atoms(fj, ctx, atoms, cache=None):
    """Binding atoms over device copies of the atoms' relations (one
    relation handle per distinct relation, so self-joins share columns)."""
    import torch
    cache = {} if cache is None else cache
    out = []
    for a in atoms:
        rel = a["rel"]
        key = id(rel)
        if key not in cache:
            cols = [torch.from_numpy(np.ascontiguousarray(c, dtype=np.int32)).cuda()
                    for c in rel["cols"]]
            cache[key] = ctx.relation(cols, rel.get("name", ""))
        out.append({"rel": cache[key], "vars": list(a["vars"]), "rel_cols": a["rel_cols"],
                    "preds": list(a.get("preds", []))})
    return out, cache


def gj_plan(atom_vars, var_order):
    """The Generic Join plan for a total variable order (Section 3.2, Eq. 3
    shape): one node per variable holding R(x) for every atom containing x."""
    plan = []
    for x in var_order:
        node = [(a, (x,)) for a, vs in enumerate(atom_vars) if x in vs]
        plan.append(node)
    return plan


def plans_for(atom_vars, rng, n_orders=2):
    """A mix of valid plans: binary2fj with and without factor for random
    left-deep orders, and Generic Join plans for random variable orders."""
    out = []
    nvars = sorted({v for vs in atom_vars for v in vs})
    for _ in range(n_orders):
        order = [int(i) for i in rng.permutation(len(atom_vars))]
        bj = P.binary2fj(atom_vars, order)
        out.append(("bj", bj))
        out.append(("factored", P.factor(bj)))
        vo = [int(v) for v in rng.permutation(nvars)]
        out.append(("gj", gj_plan(atom_vars, vo)))
    return out


def sort_rows(t):
    t = np.asarray(t)
    if t.size == 0:
        return t.reshape(0, t.shape[1] if t.ndim == 2 else 0)
    return t[np.lexsort(t.T[::-1])]
