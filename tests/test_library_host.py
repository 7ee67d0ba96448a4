"""Host-side checks of libfj.so that need no GPU: the library loads, exports
every entry point declared in include/fj.h, and its plan logic (binary2fj,
factor, validity, covers, GHT schemas) agrees with the paper's printed
examples and with the oracle's plain-Python restatement."""

import os
import re
import subprocess

import numpy as np
import pytest

from oracle import plan as P
from paper_2301_10841_gb300 import datagen as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fjm():
    from paper_2301_10841_gb300 import build
    build.build()
    from paper_2301_10841_gb300 import fj
    return fj


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(fj_[a-z0-9_]+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol(fjm):
    so = os.path.join(ROOT, "paper_2301_10841_gb300", "libfj.so")
    out = subprocess.check_output(["nm", "-D", "--defined-only", so]).decode()
    exported = set(re.findall(r"\bT (fj_[a-z0-9_]+)", out))
    declared = _declared()
    assert declared, "no declarations found"
    assert declared <= exported, sorted(declared - exported)
    # the binding wires up every declared function
    assert declared <= set(fjm.EXPORTED), sorted(declared - set(fjm.EXPORTED))


def _atoms(atom_vars):
    return [{"vars": list(v)} for v in atom_vars]


def test_planner_matches_printed_examples(fjm):
    clover = [[0, 1], [0, 2], [0, 3]]  # R(x,a), S(x,b), T(x,c)
    assert fjm.binary_to_free_plan(_atoms(clover), [0, 1, 2], factor=False) == \
        [[(0, (0, 1)), (1, (0,))], [(1, (2,)), (2, (0,))], [(2, (3,))]]
    assert fjm.binary_to_free_plan(_atoms(clover), [0, 1, 2], factor=True) == \
        [[(0, (0, 1)), (1, (0,)), (2, (0,))], [(1, (2,))], [(2, (3,))]]
    chain = [[0, 1], [1, 2], [2, 3], [3, 4]]
    want = [[(0, (0, 1)), (1, (1,))], [(1, (2,)), (2, (2,))], [(2, (3,)), (3, (3,))], [(3, (4,))]]
    assert fjm.binary_to_free_plan(_atoms(chain), [0, 1, 2, 3], factor=False) == want
    assert fjm.binary_to_free_plan(_atoms(chain), [0, 1, 2, 3], factor=True) == want
    gj = [[(0, (0,)), (1, (0,)), (2, (0,))], [(0, (1,))], [(1, (2,))], [(2, (3,))]]
    assert [fjm.node_covers(_atoms(clover), gj, k) for k in range(4)] == [[0, 1, 2], [0], [0], [0]]
    ok, why = fjm.validate_plan(_atoms(clover), [[(0, (0, 1)), (1, (0, 2)), (2, (0, 3))]])
    assert not ok and "cover" in why
    tri = [[0, 1], [1, 2], [2, 0]]
    plan = [[(0, (0, 1)), (1, (1,)), (2, (0,))], [(1, (2,)), (2, (2,))]]
    assert [fjm.ght_schema(_atoms(tri), plan, a) for a in range(3)] == \
        [[[0, 1]], [[1], [2]], [[0], [2], []]]


@pytest.mark.parametrize("seed", range(150))
def test_planner_matches_oracle_restatement(fjm, seed):
    atoms = G.random_query(seed, max_atoms=6, max_vars=7)
    atom_vars = [a["vars"] for a in atoms]
    rng = np.random.default_rng(seed)
    order = [int(i) for i in rng.permutation(len(atoms))]
    for fac in (False, True):
        want = P.binary2fj(atom_vars, order)
        if fac:
            want = P.factor(want)
        got = fjm.binary_to_free_plan(_atoms(atom_vars), order, factor=fac)
        assert got == [[(a, tuple(v)) for a, v in node] for node in want]
        ok, why = fjm.validate_plan(_atoms(atom_vars), got)
        assert ok, why
        for k in range(len(got)):
            assert fjm.node_covers(_atoms(atom_vars), got, k) == P.covers(want, k)
        for a in range(len(atoms)):
            assert fjm.ght_schema(_atoms(atom_vars), got, a) == P.ght_schemas(atom_vars, want)[a]


def test_invalid_plans_are_rejected(fjm):
    tri = _atoms([[0, 1], [1, 2], [2, 0]])
    bad = {
        "two subatoms of one atom": [[(0, (0, 1)), (0, ())], [(1, (1, 2)), (2, (2, 0))]],
        "not a partition": [[(0, (0, 1)), (1, (1,)), (2, (0,))], [(1, (2,))]],
        "no cover": [[(1, (1,)), (0, (0,))], [(0, (1,)), (1, (2,)), (2, (2, 0))]],
    }
    for name, plan in bad.items():
        ok, why = fjm.validate_plan(tri, plan)
        assert not ok, name
        assert why


def test_generic_join_plan_is_one_node_per_variable(fjm):
    """fj_generic_join_plan (Section 3.2, Eq. 3): node k holds R(x_k) of every
    atom containing x_k, in atom order; every such plan is valid."""
    import sys
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from fjtest import gj_plan
    rng = np.random.default_rng(4)
    for seed in range(60):
        atoms = G.random_query(seed, max_atoms=5, max_vars=6, max_arity=3)
        atom_vars = [a["vars"] for a in atoms]
        nv = sorted({v for vs in atom_vars for v in vs})
        order = [int(v) for v in rng.permutation(nv)]
        plan = fjm.generic_join_plan(_atoms(atom_vars), order)
        want = [[(a, (x,)) for a, vs in enumerate(atom_vars) if x in vs] for x in order]
        assert plan == want == gj_plan(atom_vars, order)
        assert fjm.validate_plan(_atoms(atom_vars), plan)[0]
    with pytest.raises(fjm.FJError):
        fjm.generic_join_plan(_atoms([[0, 1], [1, 2]]), [0, 1])      # a variable missing
    with pytest.raises(fjm.FJError):
        fjm.generic_join_plan(_atoms([[0, 1], [1, 2]]), [0, 1, 1])   # a variable twice
