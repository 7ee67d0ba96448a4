"""Free Join oracle -- TEST INFRASTRUCTURE ONLY.

Only the test suite, the smoke check and the CPU-baseline leg of ``bench.py``
may import this package.  The product library never loads it and shares no
code with it.

Contents (each function cites the paper passage it follows):

* :func:`binary_join`   -- left-deep pipelined hash join (Section 2.2, Fig. 2a),
                           C++ in ``fj_oracle.cpp``.
* :func:`generic_join`  -- textbook Generic Join over full hash tries
                           (Section 2.3, Fig. 2b), C++ in ``fj_oracle.cpp``.
* :func:`brute_force`   -- nested loop over every combination of rows, the
                           plain definition of the bag join (Section 2.1, Eq. 1).
* :mod:`oracle.plan`    -- ``binary2fj`` (Fig. 9), ``factor`` (Fig. 10),
                           plan validity and covers (Def. 3.5-3.7) and GHT
                           schemas (Section 3.3), in plain Python.
* :mod:`oracle.closed`  -- closed forms and library routines used as pins
                           (trace of adjacency powers, complete-graph counts,
                           direct-address star join).

A query is plain data: a list of atoms, each a dict with
``cols`` (list of 1-D int32 numpy arrays, one per variable), ``vars`` (list of
distinct variable ids) and optional ``preds`` (list of ``(j, op, value)`` with
``j`` an index into ``cols`` and ``op`` one of ``"<" "<=" ">" ">=" "==" "!="``).
Results are ``(count, mins, tuples)``: ``count`` an int, ``mins`` a list with
``None`` for an empty result (SQL NULL), ``tuples`` an ``(n, len(head))`` int32
array sorted lexicographically (or ``None`` when not materialized).
"""

from __future__ import annotations

import ctypes
import itertools
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "fj_oracle.cpp")

OPS = {"<": 0, "<=": 1, ">": 2, ">=": 3, "==": 4, "!=": 5}


def build(force: bool = False) -> str:
    """Compile the C++ oracle into ``oracle/liboracle.so`` (plain g++)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


class _Atom(ctypes.Structure):
    _fields_ = [
        ("n_vars", ctypes.c_int),
        ("cols", ctypes.POINTER(ctypes.c_void_p)),
        ("n_rows", ctypes.c_uint64),
        ("vars", ctypes.POINTER(ctypes.c_int)),
        ("n_preds", ctypes.c_int),
        ("pred_col", ctypes.POINTER(ctypes.c_int)),
        ("pred_op", ctypes.POINTER(ctypes.c_int)),
        ("pred_val", ctypes.POINTER(ctypes.c_int32)),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        common = [ctypes.c_int, ctypes.POINTER(_Atom)]
        tail = [
            ctypes.c_int, ctypes.POINTER(ctypes.c_int),  # head
            ctypes.c_int, ctypes.POINTER(ctypes.c_int),  # min vars
            ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_int32),
            ctypes.POINTER(ctypes.c_uint8), ctypes.c_void_p, ctypes.c_uint64,
            ctypes.POINTER(ctypes.c_uint64),
        ]
        lib.oracle_binary_join.argtypes = common + [ctypes.POINTER(ctypes.c_int)] + tail
        lib.oracle_binary_join.restype = ctypes.c_int
        lib.oracle_generic_join.argtypes = (
            common + [ctypes.POINTER(ctypes.c_int), ctypes.c_int] + tail)
        lib.oracle_generic_join.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ints(xs):
    arr = (ctypes.c_int * max(1, len(xs)))(*xs)
    return arr


def query_vars(atoms):
    """Variables in order of first appearance across atoms (the default head)."""
    out = []
    for a in atoms:
        for v in a["vars"]:
            if v not in out:
                out.append(v)
    return out


def _marshal(atoms):
    keep = []
    arr = (_Atom * len(atoms))()
    for i, a in enumerate(atoms):
        cols = [np.ascontiguousarray(c, dtype=np.int32) for c in a["cols"]]
        n = len(cols[0]) if cols else 0
        for c in cols:
            if len(c) != n:
                raise ValueError("columns of one atom must have equal length")
        ptrs = (ctypes.c_void_p * len(cols))(*[c.ctypes.data for c in cols])
        preds = a.get("preds", [])
        pc = _ints([p[0] for p in preds])
        po = _ints([OPS[p[1]] for p in preds])
        pv = (ctypes.c_int32 * max(1, len(preds)))(*[int(p[2]) for p in preds])
        vs = _ints(list(a["vars"]))
        keep += [cols, ptrs, pc, po, pv, vs]
        arr[i] = _Atom(len(cols), ctypes.cast(ptrs, ctypes.POINTER(ctypes.c_void_p)), n,
                       ctypes.cast(vs, ctypes.POINTER(ctypes.c_int)), len(preds),
                       ctypes.cast(pc, ctypes.POINTER(ctypes.c_int)),
                       ctypes.cast(po, ctypes.POINTER(ctypes.c_int)),
                       ctypes.cast(pv, ctypes.POINTER(ctypes.c_int32)))
    return arr, keep


def _run(fn, atoms, extra, head, min_vars, materialize, cap):
    lib = _load()
    head = list(query_vars(atoms) if head is None else head)
    min_vars = list(min_vars or [])
    arr, keep = _marshal(atoms)
    count = ctypes.c_uint64(0)
    mins = (ctypes.c_int32 * max(1, len(min_vars)))()
    valid = (ctypes.c_uint8 * max(1, len(min_vars)))()
    n_out = ctypes.c_uint64(0)
    out = None
    if materialize:
        if cap is None:
            # First pass counts, second pass writes.
            rc = fn(len(atoms), arr, *extra, len(head), _ints(head), len(min_vars),
                    _ints(min_vars), ctypes.byref(count), mins, valid, None, 0,
                    ctypes.byref(n_out))
            if rc != 0:
                raise RuntimeError(f"oracle failed: {rc}")
            cap = count.value
        out = np.zeros((max(1, cap), len(head)), dtype=np.int32)
        ptr = out.ctypes.data
    else:
        ptr = None
        cap = 0
    rc = fn(len(atoms), arr, *extra, len(head), _ints(head), len(min_vars), _ints(min_vars),
            ctypes.byref(count), mins, valid, ptr, cap, ctypes.byref(n_out))
    del keep
    if rc not in (0, -4):
        raise RuntimeError(f"oracle failed: {rc}")
    mv = [int(mins[i]) if valid[i] else None for i in range(len(min_vars))]
    tup = None
    if materialize:
        tup = out[: min(count.value, cap)]
    return int(count.value), mv, tup


def binary_join(atoms, order=None, head=None, min_vars=None, materialize=False, cap=None):
    """O1: left-deep pipelined hash join in ``order`` (Section 2.2, Fig. 2a)."""
    order = list(range(len(atoms))) if order is None else list(order)
    lib = _load()
    return _run(lib.oracle_binary_join, atoms, [_ints(order)], head, min_vars, materialize, cap)


def generic_join(atoms, var_order=None, head=None, min_vars=None, materialize=False, cap=None):
    """O2: Generic Join over full hash tries (Section 2.3, Fig. 2b)."""
    var_order = list(query_vars(atoms) if var_order is None else var_order)
    lib = _load()
    return _run(lib.oracle_generic_join, atoms, [_ints(var_order), len(var_order)], head,
                min_vars, materialize, cap)


_PY_OPS = {
    "<": lambda a, b: a < b, "<=": lambda a, b: a <= b, ">": lambda a, b: a > b,
    ">=": lambda a, b: a >= b, "==": lambda a, b: a == b, "!=": lambda a, b: a != b,
}


def brute_force(atoms, head=None, min_vars=None):
    """O3: the plain definition of the bag join (Section 2.1, Eq. 1).

    Every combination of one row per atom whose values agree on all shared
    variables contributes one output tuple.  Pure Python; tiny inputs only.
    """
    head = list(query_vars(atoms) if head is None else head)
    min_vars = list(min_vars or [])
    rows_per_atom = []
    for a in atoms:
        n = len(a["cols"][0])
        rows = []
        for r in range(n):
            ok = all(_PY_OPS[op](int(a["cols"][j][r]), int(v)) for j, op, v in a.get("preds", []))
            if ok:
                rows.append([int(c[r]) for c in a["cols"]])
        rows_per_atom.append(rows)
    out = []
    for combo in itertools.product(*rows_per_atom):
        bind = {}
        ok = True
        for a, row in zip(atoms, combo):
            for v, val in zip(a["vars"], row):
                if bind.setdefault(v, val) != val:
                    ok = False
                    break
            if not ok:
                break
        if ok:
            out.append(tuple(bind[v] for v in head))
    out.sort()
    mins = []
    for v in min_vars:
        i = head.index(v)
        mins.append(min(t[i] for t in out) if out else None)
    tup = np.array(out, dtype=np.int32).reshape(len(out), len(head))
    return len(out), mins, tup
