"""Free Join plans, written out from the paper -- TEST INFRASTRUCTURE ONLY.

A plan is a list of nodes; a node is a list of subatoms; a subatom is a pair
``(atom_index, tuple_of_vars)``.  The first subatom of a node is its
designated cover (Section 3.2, the convention after Def. 3.7).  Atoms are the
query's atoms, given as their variable lists (``atom_vars[i]``).

Readings of passages the paper leaves open:

* ``binary2fj`` (Fig. 9): the "available variables" used while building the
  current node are all variables bound so far, including those of the
  current node -- otherwise the chain example of Section 4.1 would not come
  out as printed.  A relation whose variables are already all bound gets an
  empty subatom ``s()`` as its own node; it stands for the leaf vector, whose
  length is the bag multiplicity.
* ``factor`` (Fig. 10): only the non-cover subatoms of a node are candidates
  to move, visited in order, and the first one that cannot move stops the
  node (the conservative rule).  Otherwise the clover plan printed in
  Section 4.1 would not come out as printed.  Nodes are visited from the last
  to the second; a moved subatom is appended to the previous node and may
  move again when that node is visited.
* Subatoms keep the variables in the order of the atom's columns.
"""

from __future__ import annotations


def _ordered(atom_vars, a, subset):
    return tuple(v for v in atom_vars[a] if v in subset)


def vs(node):
    """vs(phi): all variables of all subatoms of a node (Def. 3.5)."""
    out = set()
    for _, vars_ in node:
        out |= set(vars_)
    return out


def avs(plan, k):
    """avs(phi_k): union of vs(phi_j) for j < k (Def. 3.5)."""
    out = set()
    for j in range(k):
        out |= vs(plan[j])
    return out


def binary2fj(atom_vars, order):
    """Left-deep binary plan ``order`` -> Free Join plan (Section 4.1, Fig. 9)."""
    r = order[0]
    phi = [(r, tuple(atom_vars[r]))]
    bound = set(atom_vars[r])
    plan = []
    for s in order[1:]:
        phi.append((s, _ordered(atom_vars, s, bound)))  # probe with available vars
        plan.append(phi)
        phi = [(s, _ordered(atom_vars, s, set(atom_vars[s]) - bound))]  # iterate the rest
        bound |= set(atom_vars[s])
    plan.append(phi)
    return plan


def factor(plan):
    """Move probes one node earlier, conservatively (Section 4.1, Fig. 10)."""
    plan = [list(node) for node in plan]
    n = len(plan)
    for i in range(n - 1, 0, -1):
        phi, prev = plan[i], plan[i - 1]
        available = avs(plan, i)
        for alpha in list(phi[1:]):
            prev_atoms = {a for a, _ in prev}
            if set(alpha[1]) <= available and alpha[0] not in prev_atoms:
                phi.remove(alpha)
                prev.append(alpha)
            else:
                break
    return plan


def covers(plan, k):
    """Subatoms of node k containing vs(phi_k) - avs(phi_k) (Def. 3.7)."""
    need = vs(plan[k]) - avs(plan, k)
    return [i for i, (_, vars_) in enumerate(plan[k]) if need <= set(vars_)]


def is_valid(atom_vars, plan):
    """Partition requirement (Def. 3.5) and validity (Def. 3.7)."""
    seen = {a: [] for a in range(len(atom_vars))}
    for node in plan:
        if not node:
            return False
        atoms_here = [a for a, _ in node]
        if len(atoms_here) != len(set(atoms_here)):
            return False  # (a) no two subatoms of one relation in a node
        for a, vars_ in node:
            if a not in seen:
                return False
            seen[a].extend(vars_)
    for a, got in seen.items():
        if sorted(got) != sorted(atom_vars[a]):
            return False  # the subatoms of each atom partition its variables
        if not any(a == b for node in plan for b, _ in node):
            return False
    return all(covers(plan, k) for k in range(len(plan)))  # (b) a cover exists


def ght_schemas(atom_vars, plan):
    """GHT schema of each atom for the build phase (Section 3.3).

    The subatoms of atom R in plan order give levels y0..y(l-1); a final empty
    level is appended unless the last subatom is the (designated) cover of its
    node.
    """
    out = []
    for a in range(len(atom_vars)):
        levels, last_is_cover = [], False
        for node in plan:
            for pos, (b, vars_) in enumerate(node):
                if b == a:
                    levels.append(list(vars_))
                    last_is_cover = pos == 0
        if not last_is_cover:
            levels.append([])
        out.append(levels)
    return out
