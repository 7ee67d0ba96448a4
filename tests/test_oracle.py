"""Pins for the CPU oracle (runs without a GPU).

Each test ties the oracle to something other than itself: the paper's worked
examples, closed forms, a library routine, or the plain definition by brute
force on tiny inputs.
"""

import json
import os

import numpy as np
import pytest

import oracle
from oracle import closed
from oracle import plan as P
from paper_2301_10841_gb300 import datagen as G

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_plans.json")


def _all_three(atoms, head=None, min_vars=None):
    bj = oracle.binary_join(atoms, head=head, min_vars=min_vars, materialize=True)
    gj = oracle.generic_join(atoms, head=head, min_vars=min_vars, materialize=True)
    bf = oracle.brute_force(atoms, head=head, min_vars=min_vars)
    return bj, gj, bf


def _same(a, b):
    assert a[0] == b[0]
    assert a[1] == b[1]
    np.testing.assert_array_equal(a[2], b[2])


# --- the plain definition, three ways --------------------------------------

@pytest.mark.parametrize("seed", range(120))
def test_random_queries_agree_with_brute_force(seed):
    atoms = G.random_query(seed)
    head = oracle.query_vars(atoms)
    mins = head[: 2]
    bj, gj, bf = _all_three(atoms, head=head, min_vars=mins)
    _same(bj, bf)
    _same(gj, bf)


@pytest.mark.parametrize("seed", range(20))
def test_join_order_and_var_order_do_not_change_the_bag(seed):
    atoms = G.random_query(1000 + seed, max_atoms=4, max_rows=10)
    head = oracle.query_vars(atoms)
    rng = np.random.default_rng(seed)
    base = oracle.brute_force(atoms, head=head)
    for _ in range(3):
        order = list(rng.permutation(len(atoms)))
        _same(oracle.binary_join(atoms, order=order, head=head, materialize=True), base)
        vo = list(rng.permutation(head))
        _same(oracle.generic_join(atoms, var_order=vo, head=head, materialize=True), base)


def test_bag_semantics_duplicates_multiply():
    # R has (1,2) twice, S has (2,3) three times: the tuple (1,2,3) has
    # multiplicity 6 under bag semantics (Section 2.1; Section 2.3 footnote).
    r = {"cols": [np.array([1, 1], np.int32), np.array([2, 2], np.int32)]}
    s = {"cols": [np.array([2, 2, 2], np.int32), np.array([3, 3, 3], np.int32)]}
    atoms = [G.atom(r, [0, 1]), G.atom(s, [1, 2])]
    for res in _all_three(atoms):
        assert res[0] == 6
        assert res[2].tolist() == [[1, 2, 3]] * 6


def test_empty_result_min_is_null():
    r = {"cols": [np.array([1], np.int32)]}
    s = {"cols": [np.array([2], np.int32)]}
    atoms = [G.atom(r, [0]), G.atom(s, [0])]
    for res in _all_three(atoms, min_vars=[0]):
        assert res[0] == 0 and res[1] == [None]


def test_predicates_are_applied():
    r = {"cols": [np.arange(10, dtype=np.int32)]}
    for op, want in [("<", 3), ("<=", 4), (">", 6), (">=", 7), ("==", 1), ("!=", 9)]:
        atoms = [G.atom(r, [0], preds=[(0, op, 3)])]
        for res in _all_three(atoms):
            assert res[0] == want, op


# --- the paper's worked example: the clover instance (Fig. 3) ---------------

def clover_instance(n):
    """Fig. 3: R = {(x0,a0)} u {(x1,a_i^l),(x2,a_i^r)}, S = {(x0,b0)} u
    {(x2,b_i^l),(x3,b_i^r)}, T = {(x0,c0)} u {(x3,c_i^l),(x1,c_i^r)}.
    x_j -> j; a0 -> 100, a_i^l -> 100+i, a_i^r -> 100+n+i; b and c likewise
    from 1000 and 10000 (n < 100)."""
    i = np.arange(1, n + 1)

    def rel(x_l, x_r, base):
        x = np.concatenate([[0], np.full(n, x_l), np.full(n, x_r)]).astype(np.int32)
        y = np.concatenate([[base], base + i, base + n + i]).astype(np.int32)
        return {"cols": [x, y]}

    R, S, T = rel(1, 2, 100), rel(2, 3, 1000), rel(3, 1, 10000)
    return [G.atom(R, [0, 1]), G.atom(S, [0, 2]), G.atom(T, [0, 3])]


@pytest.mark.parametrize("n", [1, 2, 5, 20])
def test_clover_has_exactly_one_output(n):
    atoms = clover_instance(n)
    for res in _all_three(atoms, min_vars=[1, 2, 3]):
        assert res[0] == 1
        assert res[2].tolist() == [[0, 100, 1000, 10000]]


# --- closed forms and library routines --------------------------------------

@pytest.mark.parametrize("n", [3, 4, 7, 12])
def test_complete_digraph_triangles_and_four_cycles(n):
    e = G.complete_digraph(n)
    tri = G.triangle_query(e)
    cyc = G.four_cycle_query(e)
    assert closed.complete_digraph_cycles(n, 3) == n * (n - 1) * (n - 2)
    for fn in (oracle.binary_join, oracle.generic_join):
        assert fn(tri)[0] == n * (n - 1) * (n - 2)
        assert fn(cyc)[0] == (n - 1) ** 4 + (n - 1)


@pytest.mark.parametrize("seed", range(4))
def test_triangle_and_four_cycle_count_equal_trace_of_adjacency_powers(seed):
    e = G.uniform_digraph(60, 700, seed)
    # add duplicates so multiplicities matter
    e["cols"] = [np.concatenate([c, c[:50]]) for c in e["cols"]]
    a = closed.adjacency(e["cols"][0], e["cols"][1], 60)
    assert oracle.binary_join(G.triangle_query(e))[0] == closed.trace_power(a, 3)
    assert oracle.generic_join(G.triangle_query(e))[0] == closed.trace_power(a, 3)
    assert oracle.binary_join(G.four_cycle_query(e))[0] == closed.trace_power(a, 4)
    assert oracle.generic_join(G.four_cycle_query(e))[0] == closed.trace_power(a, 4)


@pytest.mark.parametrize("seed", range(3))
def test_star_join_matches_direct_addressing(seed):
    fact, dims = G.star_schema(n_fact=20000, dims=(50, 120, 300, 700), s=1.1, seed=seed)
    # Duplicate some dimension rows so per-key counts exceed one.
    dims[1]["cols"] = [np.concatenate([c, c[:40]]) for c in dims[1]["cols"]]
    theta = 300_000_000
    atoms = G.star_query(fact, dims, theta=theta)
    want = closed.star_join_direct(fact["cols"], [tuple(d["cols"]) for d in dims], [theta] * 4)
    mins = [4, 5, 6, 7]
    for fn in (oracle.binary_join, oracle.generic_join):
        c, m, _ = fn(atoms, min_vars=mins)
        assert (c, m) == want


def test_trace_pin_catches_a_transposed_atom():
    # A mistaken triangle E(x,y),E(y,z),E(x,z) (transposed last atom) counts
    # transitive triples, not 3-cycles: the trace pin must tell them apart.
    e = G.uniform_digraph(40, 400, 7)
    a = closed.adjacency(e["cols"][0], e["cols"][1], 40)
    wrong = [G.atom(e, [0, 1]), G.atom(e, [1, 2]), G.atom(e, [0, 2])]
    assert oracle.binary_join(wrong)[0] != closed.trace_power(a, 3)


# --- plans: the paper's printed examples -------------------------------------

def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


def _names(atoms_named):
    names = sorted({v for a in atoms_named for v in a})
    return {n: i for i, n in enumerate(names)}


def _to_ids(plan, ids):
    return [[(a, tuple(ids[v] for v in vs_)) for a, vs_ in node] for node in plan]


def test_binary2fj_and_factor_match_printed_plans():
    g = _golden()
    for q in ("clover", "chain"):
        ids = _names(g[q]["atoms"])
        atom_vars = [[ids[v] for v in a] for a in g[q]["atoms"]]
        got = P.binary2fj(atom_vars, g[q]["binary2fj_order"])
        assert got == _to_ids(g[q]["binary2fj"]["plan"], ids), g[q]["binary2fj"]["cite"]
        assert P.is_valid(atom_vars, got)
    ids = _names(g["clover"]["atoms"])
    atom_vars = [[ids[v] for v in a] for a in g["clover"]["atoms"]]
    naive = P.binary2fj(atom_vars, [0, 1, 2])
    assert P.factor(naive) == _to_ids(g["clover"]["factor"]["plan"], ids)
    # The chain plan has nothing to factor: each probe needs a variable bound
    # by its own node's cover.
    ids = _names(g["chain"]["atoms"])
    atom_vars = [[ids[v] for v in a] for a in g["chain"]["atoms"]]
    chain = P.binary2fj(atom_vars, [0, 1, 2, 3])
    assert P.factor(chain) == chain


def test_covers_validity_and_schemas_match_printed_examples():
    g = _golden()
    c = g["clover"]
    ids = _names(c["atoms"])
    atom_vars = [[ids[v] for v in a] for a in c["atoms"]]
    for key in ("bj_plan_covers", "gj_plan_covers"):
        plan = _to_ids(c[key]["plan"], ids)
        assert P.is_valid(atom_vars, plan)
        assert [P.covers(plan, k) for k in range(len(plan))] == c[key]["covers"], c[key]["cite"]
    assert not P.is_valid(atom_vars, _to_ids(c["invalid_plan"]["plan"], ids))
    plan = _to_ids(c["bj_plan_schemas"]["plan"], ids)
    want = [[[ids[v] for v in lvl] for lvl in s] for s in c["bj_plan_schemas"]["schemas"]]
    assert P.ght_schemas(atom_vars, plan) == want
    t = g["triangle"]
    ids = _names(t["atoms"])
    atom_vars = [[ids[v] for v in a] for a in t["atoms"]]
    plan = _to_ids(t["schemas_plan"]["plan"], ids)
    want = [[[ids[v] for v in lvl] for lvl in s] for s in t["schemas_plan"]["schemas"]]
    assert P.ght_schemas(atom_vars, plan) == want


def test_star_plan_factors_into_one_probe_node():
    # binary2fj([F,D1..D4]) then factor moves every dimension probe into
    # node 0 (conservative rule, applied node by node from the end).
    atom_vars = [[0, 1, 2, 3], [0, 4], [1, 5], [2, 6], [3, 7]]
    plan = P.factor(P.binary2fj(atom_vars, [0, 1, 2, 3, 4]))
    assert plan == [[(0, (0, 1, 2, 3)), (1, (0,)), (2, (1,)), (3, (2,)), (4, (3,))],
                    [(1, (4,))], [(2, (5,))], [(3, (6,))], [(4, (7,))]]
    assert P.is_valid(atom_vars, plan)


def test_binary2fj_emits_empty_subatom_for_fully_bound_relation():
    # Triangle [E1,E2,E3]: E3(z,x) is fully bound after E2, so its own node is
    # the empty subatom E3(), which iterates the leaf (the multiplicity).
    atom_vars = [[0, 1], [1, 2], [2, 0]]
    plan = P.binary2fj(atom_vars, [0, 1, 2])
    assert plan == [[(0, (0, 1)), (1, (1,))], [(1, (2,)), (2, (2, 0))], [(2, ())]]
    assert P.is_valid(atom_vars, plan)


def test_factor_never_breaks_validity_on_random_queries():
    for seed in range(200):
        atoms = G.random_query(seed, max_atoms=5)
        atom_vars = [a["vars"] for a in atoms]
        rng = np.random.default_rng(seed)
        order = [int(i) for i in rng.permutation(len(atoms))]
        plan = P.binary2fj(atom_vars, order)
        assert P.is_valid(atom_vars, plan)
        assert P.is_valid(atom_vars, P.factor(plan))


def test_pkfk_direct_equals_hash_join_on_batch_queries():
    """closed.pkfk_direct (follow every foreign key to its key row by direct
    addressing) equals the oracle's hash join on chains and stars of the
    batched workload, small sizes, with selections and empty results."""
    from oracle import closed
    n_empty = 0
    for q in range(40):
        atoms, _, mins = G.batch_query(q, min_rows=50, max_rows=4000)
        want = oracle.binary_join(atoms, min_vars=mins)[:2]
        got = closed.pkfk_direct(atoms, mins)
        assert got == (want[0], want[1]), q
        n_empty += want[0] == 0
    assert n_empty < 40


def test_pkfk_direct_catches_a_wrong_key():
    """A planted mistake (one key row renumbered) changes the result."""
    from oracle import closed
    atoms, _, mins = G.batch_query(3, min_rows=500, max_rows=2000)
    base = closed.pkfk_direct(atoms, mins)
    bad = [dict(a) for a in atoms]
    key = np.array(bad[1]["cols"][0], copy=True)
    key = key[::-1].copy()  # keys still unique, rows now point elsewhere
    bad[1]["cols"] = [key] + list(bad[1]["cols"][1:])
    assert closed.pkfk_direct(bad, mins) != base


@pytest.mark.parametrize("seed", range(4))
def test_four_cycles_from_two_paths_equal_trace_of_a4(seed):
    """The 2-path form (sum of P2[w,y] P2[y,w], sparse integer products) --
    the oracle used for 4-cycles where enumeration is too slow -- against
    trace(A^4) by dense matmul, multiplicities and self-loops included, and
    against the complete digraph's closed form."""
    e = G.uniform_digraph(80, 900, seed)
    src = np.concatenate([e["cols"][0], e["cols"][0][:60], np.arange(5)])
    dst = np.concatenate([e["cols"][1], e["cols"][1][:60], np.arange(5)])
    a = closed.adjacency(src, dst, 80)
    want = closed.trace_power(a, 4)
    assert closed.four_cycles_two_paths(src, dst, 80) == want
    assert closed.four_cycles_two_paths(src, dst, 80, block=7) == want  # rows in blocks
    c = G.complete_digraph(9)
    assert closed.four_cycles_two_paths(c["cols"][0], c["cols"][1], 9) == \
        closed.complete_digraph_cycles(9, 4)
