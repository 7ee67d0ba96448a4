"""ctypes binding of libfj.so (declared in include/fj.h).

Argument marshalling only: every step of the join runs in the library's CUDA
kernels.  Importing this module loads ``libfj.so`` and raises ImportError if it
is missing -- there is no fallback.

Queries use plain data: an atom is a dict with ``rel`` (a :class:`Relation`),
``vars`` (distinct variable ids), optional ``rel_cols`` (column of the relation
per variable) and optional ``preds`` (``(j, op, value)`` with ``op`` one of
``"<" "<=" ">" ">=" "==" "!="``).  A plan is a list of nodes, a node a list of
``(atom_index, vars)`` subatoms whose first entry is the node's cover.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libfj.so")
if not os.path.exists(_SO):
    raise ImportError(f"libfj.so not built ({_SO}); run __graft_entry__.build()")
_lib = ctypes.CDLL(_SO)

MAX_VARS = 32
OPS = {"<": 0, "<=": 1, ">": 2, ">=": 3, "==": 4, "!=": 5}
COVER = {"static": 0, "fewest": 1, "learned": 2}
OUT = {"materialize": 0, "count": 1, "count_min": 2, "factorized": 3}
FLAG_EAGER_ALL = 1
FLAG_EAGER_ROOT = 2
FLAG_TIMING = 4
FLAG_TEST_TIMEOUT = 8
FLAG_NO_FUSED_SCAN = 16
CTR = {"cover_iters": 0, "probes": 1, "probe_hits": 2, "roots_built": 3, "subtries_forced": 4,
       "rows_regrouped": 5, "survivors": 6, "chunks": 7, "kernels": 8, "atom_built_mask": 9,
       "expand_ns": 10, "expand_launches": 11, "build_ns": 12, "span_ns": 13, "cover_policy": 14}
CHOOSER_IN_DIM = 137

ERRORS = {0: "OK", -1: "INVALID_ARG", -2: "INVALID_PLAN", -3: "OOM", -4: "OUTPUT_OVERFLOW",
          -5: "COUNT_OVERFLOW", -6: "TIMEOUT", -7: "CUDA", -8: "UNSUPPORTED"}


class FJError(RuntimeError):
    """A failed library call.  ``result`` is set for FJ_ERR_OUTPUT_OVERFLOW of
    a materialized execution: the exact COUNT and the first list_limit rows."""

    def __init__(self, status, msg, result=None):
        super().__init__(f"{ERRORS.get(status, status)}: {msg}")
        self.status = status
        self.result = result


class _Pred(ctypes.Structure):
    _fields_ = [("col", ctypes.c_int), ("op", ctypes.c_int), ("value", ctypes.c_int32)]


class _Atom(ctypes.Structure):
    _fields_ = [("rel", ctypes.c_void_p), ("n_vars", ctypes.c_int),
                ("vars", ctypes.POINTER(ctypes.c_int)), ("cols", ctypes.POINTER(ctypes.c_int)),
                ("n_preds", ctypes.c_int), ("preds", ctypes.POINTER(_Pred))]


class _Query(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int), ("atoms", ctypes.POINTER(_Atom)),
                ("n_head", ctypes.c_int), ("head_vars", ctypes.POINTER(ctypes.c_int))]


class _Sub(ctypes.Structure):
    _fields_ = [("atom", ctypes.c_int), ("n_vars", ctypes.c_int),
                ("vars", ctypes.POINTER(ctypes.c_int))]


class _Node(ctypes.Structure):
    _fields_ = [("n_sub", ctypes.c_int), ("sub", ctypes.POINTER(_Sub))]


class _Plan(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int), ("nodes", ctypes.POINTER(_Node))]


class _Opts(ctypes.Structure):
    _fields_ = [("batch_size", ctypes.c_uint32), ("load_factor", ctypes.c_float),
                ("cover_policy", ctypes.c_int), ("out_mode", ctypes.c_int),
                ("list_limit", ctypes.c_uint64), ("n_min_vars", ctypes.c_int),
                ("min_vars", ctypes.POINTER(ctypes.c_int)), ("spin_limit", ctypes.c_uint64),
                ("model", ctypes.c_void_p), ("flags", ctypes.c_uint32)]


class _BushyNode(ctypes.Structure):
    _fields_ = [("atom", ctypes.c_int), ("left", ctypes.c_int), ("right", ctypes.c_int)]


class _Result(ctypes.Structure):
    _fields_ = [("count", ctypes.c_uint64), ("mins", ctypes.c_int32 * MAX_VARS),
                ("min_valid", ctypes.c_uint8 * MAX_VARS), ("n_head", ctypes.c_int),
                ("n_out", ctypes.c_uint64), ("d_tuples", ctypes.c_void_p),
                ("tuples_owned", ctypes.c_int), ("counters", ctypes.c_uint64 * 16)]


_P = ctypes.POINTER
_vp = ctypes.c_void_p
_sig = {
    "fj_ctx_create": ([ctypes.c_int, _vp, _P(_vp)], ctypes.c_int),
    "fj_ctx_destroy": ([_vp], None),
    "fj_ctx_set_stream": ([_vp, _vp], ctypes.c_int),
    "fj_last_error": ([], ctypes.c_char_p),
    "fj_load_relation": ([_vp, ctypes.c_char_p, ctypes.c_int, _P(_vp), ctypes.c_uint64, _P(_vp)],
                         ctypes.c_int),
    "fj_load_relation_host": ([_vp, ctypes.c_char_p, ctypes.c_int, _P(_vp), ctypes.c_uint64,
                               _P(_vp)], ctypes.c_int),
    "fj_release_relation": ([_vp, _vp], None),
    "fj_relation_rows": ([_vp], ctypes.c_uint64),
    "fj_validate_plan": ([_P(_Query), _P(_Plan)], ctypes.c_int),
    "fj_binary_to_free_plan": ([_P(_Query), _P(ctypes.c_int), ctypes.c_int, ctypes.c_int,
                                _P(_P(_Plan))], ctypes.c_int),
    "fj_plan_free": ([_P(_Plan)], None),
    "fj_generic_join_plan": ([_P(_Query), _P(ctypes.c_int), ctypes.c_int, _P(_P(_Plan))],
                             ctypes.c_int),
    "fj_ght_schema": ([_P(_Query), _P(_Plan), ctypes.c_int, _P(ctypes.c_int), _P(ctypes.c_int),
                       _P(ctypes.c_int)], ctypes.c_int),
    "fj_node_covers": ([_P(_Query), _P(_Plan), ctypes.c_int, _P(ctypes.c_int), _P(ctypes.c_int)],
                       ctypes.c_int),
    "fj_execute_plan": ([_vp, _P(_Query), _P(_Plan), _P(_Opts), _P(_Result)], ctypes.c_int),
    "fj_prepare": ([_vp, _P(_Query), _P(_Plan), _P(_Opts), _P(_vp)], ctypes.c_int),
    "fj_build_colt_level": ([_vp, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "fj_execute_prepared": ([_vp, _P(_Result)], ctypes.c_int),
    "fj_reset_prepared": ([_vp], ctypes.c_int),
    "fj_execute_prepared_async": ([_vp], ctypes.c_int),
    "fj_prepared_result": ([_vp, _P(_Result)], ctypes.c_int),
    "fj_prepared_free": ([_vp], None),
    "fj_batch_create": ([_vp, ctypes.c_int, _P(_vp), ctypes.c_int, _P(_vp)], ctypes.c_int),
    "fj_batch_execute": ([_vp, _P(_Result)], ctypes.c_int),
    "fj_batch_launch": ([_vp], ctypes.c_int),
    "fj_batch_results": ([_vp, _P(_Result)], ctypes.c_int),
    "fj_batch_free": ([_vp], None),
    "fj_model_create": ([_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P(_vp)],
                        ctypes.c_int),
    "fj_model_n_params": ([_vp], ctypes.c_size_t),
    "fj_model_set_params": ([_vp, _vp, ctypes.c_size_t], ctypes.c_int),
    "fj_model_get_params": ([_vp, _vp, ctypes.c_size_t], ctypes.c_int),
    "fj_model_forward": ([_vp, _vp, ctypes.c_int, _vp], ctypes.c_int),
    "fj_model_gradients": ([_vp, _vp, _vp, ctypes.c_int, _vp, _P(ctypes.c_float)], ctypes.c_int),
    "fj_model_train_step": ([_vp, _vp, _vp, ctypes.c_int, ctypes.c_float, _P(ctypes.c_float)],
                            ctypes.c_int),
    "fj_model_last_error": ([], ctypes.c_char_p),
    "fj_model_set_scaler": ([_vp, _vp, _vp, ctypes.c_size_t], ctypes.c_int),
    "fj_model_save": ([_vp, ctypes.c_char_p], ctypes.c_int),
    "fj_model_load": ([_vp, ctypes.c_char_p, ctypes.c_int, _P(_vp)], ctypes.c_int),
    "fj_plan_features": ([_vp, _P(_Query), ctypes.c_int, _P(ctypes.c_int), _P(ctypes.c_int), _vp],
                         ctypes.c_int),
    "fj_choose_plan": ([_vp, _P(_Query), _vp, ctypes.c_int, ctypes.c_uint64, _P(_P(_Plan)),
                        _P(ctypes.c_int), _P(ctypes.c_int)], ctypes.c_int),
    "fj_chooser_last_error": ([], ctypes.c_char_p),
    "fj_model_free": ([_vp], None),
    "fj_degree_histogram": ([_vp, _vp, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, _vp],
                            ctypes.c_int),
    "fj_stats_last_error": ([], ctypes.c_char_p),
    "fj_result_copy_tuples": ([_vp, _P(_Result), _vp, ctypes.c_int], ctypes.c_int),
    "fj_prepared_factor_layout": ([_vp, _P(ctypes.c_int), _P(ctypes.c_int), _P(ctypes.c_int),
                                   _P(ctypes.c_int), _P(ctypes.c_int)], ctypes.c_int),
    "fj_prepared_expand": ([_vp, _P(_Result), _vp, ctypes.c_uint64], ctypes.c_int),
    "fj_execute_bushy": ([_vp, _P(_Query), _P(_BushyNode), ctypes.c_int, _P(_Opts), _P(_Result)],
                         ctypes.c_int),
    "fj_result_free": ([_vp, _P(_Result)], None),
    "fj_join2_count_noalloc": ([_vp, ctypes.c_uint64, _vp, ctypes.c_uint64, _vp, _vp],
                               ctypes.c_int),
    "fj_noalloc_last_error": ([], ctypes.c_char_p),
}
for _name, (_args, _res) in _sig.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res

EXPORTED = sorted(_sig)


def _check(st):
    if st != 0:
        raise FJError(st, _lib.fj_last_error().decode())


def _ints(xs):
    xs = [int(x) for x in xs]
    return (ctypes.c_int * max(1, len(xs)))(*xs)


# ---------------------------------------------------------------------------
# Marshalling of queries and plans.
# ---------------------------------------------------------------------------

class _QueryC:
    """Keeps the ctypes arrays of one query alive."""

    def __init__(self, atoms, head=None):
        self.keep = []
        arr = (_Atom * len(atoms))()
        for i, a in enumerate(atoms):
            vs = _ints(a["vars"])
            cols = a.get("rel_cols")
            cp = _ints(cols) if cols is not None else None
            preds = a.get("preds", [])
            pa = (_Pred * max(1, len(preds)))(*[_Pred(int(j), OPS[op], int(v)) for j, op, v in preds])
            rel = a.get("rel")
            handle = rel.handle if isinstance(rel, Relation) else None
            arr[i] = _Atom(handle, len(a["vars"]), ctypes.cast(vs, _P(ctypes.c_int)),
                           ctypes.cast(cp, _P(ctypes.c_int)) if cp is not None else None,
                           len(preds), ctypes.cast(pa, _P(_Pred)))
            self.keep += [vs, cp, pa]
        self.arr = arr
        self.head = None if head is None else _ints(head)
        self.q = _Query(len(atoms), ctypes.cast(arr, _P(_Atom)), 0 if head is None else len(head),
                        None if head is None else ctypes.cast(self.head, _P(ctypes.c_int)))

    @property
    def ptr(self):
        return ctypes.byref(self.q)


class _PlanC:
    def __init__(self, plan):
        self.keep = []
        nodes = (_Node * len(plan))()
        for k, node in enumerate(plan):
            subs = (_Sub * len(node))()
            for s, (atom, vars_) in enumerate(node):
                vs = _ints(vars_)
                self.keep.append(vs)
                subs[s] = _Sub(int(atom), len(vars_), ctypes.cast(vs, _P(ctypes.c_int)))
            self.keep.append(subs)
            nodes[k] = _Node(len(node), ctypes.cast(subs, _P(_Sub)))
        self.nodes = nodes
        self.p = _Plan(len(plan), ctypes.cast(nodes, _P(_Node)))

    @property
    def ptr(self):
        return ctypes.byref(self.p)


def _plan_from_c(pp):
    p = pp.contents
    out = []
    for k in range(p.n_nodes):
        n = p.nodes[k]
        out.append([(n.sub[s].atom, tuple(n.sub[s].vars[j] for j in range(n.sub[s].n_vars)))
                    for s in range(n.n_sub)])
    return out


# ---------------------------------------------------------------------------
# Plans (host only; no GPU needed).
# ---------------------------------------------------------------------------

def binary_to_free_plan(atoms, order=None, factor=True):
    """binary2fj (Fig. 9) and, if ``factor``, factor (Fig. 10)."""
    q = _QueryC(atoms)
    order = list(range(len(atoms))) if order is None else list(order)
    out = _P(_Plan)()
    _check(_lib.fj_binary_to_free_plan(q.ptr, _ints(order), len(order), int(bool(factor)),
                                       ctypes.byref(out)))
    try:
        return _plan_from_c(out)
    finally:
        _lib.fj_plan_free(out)


def generic_join_plan(atoms, var_order):
    """The Generic Join plan of a total variable order (Section 3.2, Eq. 3)."""
    q = _QueryC(atoms)
    out = _P(_Plan)()
    _check(_lib.fj_generic_join_plan(q.ptr, _ints(var_order), len(var_order), ctypes.byref(out)))
    try:
        return _plan_from_c(out)
    finally:
        _lib.fj_plan_free(out)


def validate_plan(atoms, plan):
    """Returns (True, "") or (False, reason) per Def. 3.5 / Def. 3.7."""
    q, p = _QueryC(atoms), _PlanC(plan)
    st = _lib.fj_validate_plan(q.ptr, p.ptr)
    return st == 0, _lib.fj_last_error().decode()


def ght_schema(atoms, plan, atom):
    q, p = _QueryC(atoms), _PlanC(plan)
    n = ctypes.c_int(0)
    sizes = (ctypes.c_int * 64)()
    vs = (ctypes.c_int * 64)()
    _check(_lib.fj_ght_schema(q.ptr, p.ptr, atom, ctypes.byref(n), sizes, vs))
    out, w = [], 0
    for lv in range(n.value):
        out.append([vs[w + j] for j in range(sizes[lv])])
        w += sizes[lv]
    return out


def node_covers(atoms, plan, k):
    q, p = _QueryC(atoms), _PlanC(plan)
    n = ctypes.c_int(0)
    cv = (ctypes.c_int * 64)()
    _check(_lib.fj_node_covers(q.ptr, p.ptr, k, ctypes.byref(n), cv))
    return [cv[i] for i in range(n.value)]


# ---------------------------------------------------------------------------
# Context, relations, execution.
# ---------------------------------------------------------------------------

def _current_stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


class Context:
    """A libfj context on one CUDA device, enqueuing on a torch stream."""

    def __init__(self, device=0, stream=None):
        self.handle = _vp()
        if stream is None:
            stream = _current_stream()
        _check(_lib.fj_ctx_create(int(device), _vp(stream), ctypes.byref(self.handle)))
        self.device = device
        self._children = []  # weak references to relations and prepared plans

    def set_stream(self, stream):
        _check(_lib.fj_ctx_set_stream(self.handle, _vp(stream)))

    def relation(self, cols, name=""):
        """Borrow device columns (torch int32 CUDA tensors of equal length)."""
        return Relation(self, cols, name, host=False)

    def relation_host(self, cols, name=""):
        """Copy host columns (numpy int32 arrays or CPU tensors) to the device."""
        return Relation(self, cols, name, host=True)

    def _adopt(self, obj):
        import weakref
        self._children.append(weakref.ref(obj))

    def close(self):
        if self.handle:
            # fj_ctx_destroy releases every relation and prepared plan;
            # batches are freed here.
            for ref in self._children:
                obj = ref()
                if obj is not None:
                    if isinstance(obj, Batch):
                        obj.free()
                    obj.handle = _vp()
            self._children = []
            _lib.fj_ctx_destroy(self.handle)
            self.handle = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Relation:
    def __init__(self, ctx, cols, name="", host=False):
        self.ctx = ctx
        self.keep = list(cols)
        ptrs = []
        n = None
        for c in cols:
            if hasattr(c, "data_ptr"):
                if c.dtype.__str__() != "torch.int32" or not c.is_contiguous():
                    raise ValueError("columns must be contiguous int32")
                ptrs.append(c.data_ptr())
                length = c.numel()
            else:
                c = np.ascontiguousarray(c, dtype=np.int32)
                self.keep.append(c)
                ptrs.append(c.ctypes.data)
                length = len(c)
            if n is None:
                n = length
            elif n != length:
                raise ValueError("columns of one relation must have equal length")
        arr = (_vp * len(ptrs))(*ptrs)
        self.handle = _vp()
        fn = _lib.fj_load_relation_host if host else _lib.fj_load_relation
        _check(fn(ctx.handle, name.encode(), len(ptrs), arr, int(n or 0), ctypes.byref(self.handle)))
        self.n_rows = int(n or 0)
        ctx._adopt(self)

    def release(self):
        if self.handle and self.ctx.handle:
            _lib.fj_release_relation(self.ctx.handle, self.handle)
        self.handle = _vp()


class Result:
    def __init__(self, res, tuples, min_vars):
        self._raw = res
        self.count = int(res.count)
        self.mins = [int(res.mins[i]) if res.min_valid[i] else None for i in range(len(min_vars))]
        self.tuples = tuples
        self.counters = {k: int(res.counters[v]) for k, v in CTR.items()}


def _opts(out_mode, min_vars, batch_size, load_factor, cover, list_limit, flags, model=None,
          spin_limit=0):
    mv = _ints(min_vars or [])
    o = _Opts(int(batch_size), float(load_factor), COVER[cover], OUT[out_mode], int(list_limit),
              len(min_vars or []), ctypes.cast(mv, _P(ctypes.c_int)), int(spin_limit),
              model.handle if model is not None else None, int(flags))
    return o, mv


def _take_tuples(ctx, res, n_head):
    import torch
    n = int(res.n_out)
    t = torch.empty((n, n_head), dtype=torch.int32, device=f"cuda:{ctx.device}")
    if n:
        _check(_lib.fj_result_copy_tuples(ctx.handle, ctypes.byref(res), _vp(t.data_ptr()), 1))
    return t


def execute(ctx, atoms, plan, head=None, out_mode="count", min_vars=None, batch_size=0,
            load_factor=0.0, cover="static", list_limit=0, flags=0, model=None, spin_limit=0):
    """One-shot fj_execute_plan.  Returns a :class:`Result`; materialized
    tuples come back as an (n, len(head)) int32 CUDA tensor in head order
    (unsorted).  ``cover="learned"`` needs ``model`` (a :class:`Model`)."""
    q, p = _QueryC(atoms, head), _PlanC(plan)
    o, mv = _opts(out_mode, min_vars, batch_size, load_factor, cover, list_limit, flags, model,
                  spin_limit)
    res = _Result()
    st = _lib.fj_execute_plan(ctx.handle, q.ptr, p.ptr, ctypes.byref(o), ctypes.byref(res))
    if st not in (0, -4):
        _check(st)
    msg = _lib.fj_last_error().decode()
    tuples = None
    try:
        if out_mode == "materialize" and res.d_tuples:
            tuples = _take_tuples(ctx, res, res.n_head)
    finally:
        _lib.fj_result_free(ctx.handle, ctypes.byref(res))
    out = Result(res, tuples, min_vars or [])
    if st != 0:
        raise FJError(st, msg, out)
    return out


def bushy_nodes(tree):
    """Flatten a nested join tree -- an atom index, or a pair (left, right)
    of trees -- into fj_bushy_node rows, the root last."""
    nodes = []

    def walk(t):
        if isinstance(t, int):
            nodes.append((t, -1, -1))
        else:
            left, right = walk(t[0]), walk(t[1])
            nodes.append((-1, left, right))
        return len(nodes) - 1

    walk(tree)
    return nodes


def execute_bushy(ctx, atoms, tree, head=None, out_mode="count", min_vars=None, batch_size=0,
                  load_factor=0.0, cover="static", list_limit=0, flags=0, model=None):
    """fj_execute_bushy: run a bushy join tree (nested pairs of atom indices)
    with its non-atom right children materialized first."""
    q = _QueryC(atoms, head)
    nodes = bushy_nodes(tree)
    arr = (_BushyNode * len(nodes))(*[_BushyNode(*n) for n in nodes])
    o, mv = _opts(out_mode, min_vars, batch_size, load_factor, cover, list_limit, flags, model)
    res = _Result()
    st = _lib.fj_execute_bushy(ctx.handle, q.ptr, arr, len(nodes), ctypes.byref(o),
                               ctypes.byref(res))
    if st not in (0, -4):
        _check(st)
    msg = _lib.fj_last_error().decode()
    tuples = None
    try:
        if out_mode == "materialize" and res.d_tuples:
            tuples = _take_tuples(ctx, res, res.n_head)
    finally:
        _lib.fj_result_free(ctx.handle, ctypes.byref(res))
    out = Result(res, tuples, min_vars or [])
    if st != 0:
        raise FJError(st, msg, out)
    return out


def join2_count_noalloc(r_key, s_key, out, stream=None):
    """Bag COUNT of R(x), S(x) into the int64 CUDA tensor `out` (one element),
    with no device allocation (fj_join2_count_noalloc).  `r_key` and `s_key`
    are contiguous int32 CUDA tensors; work goes on `stream` (default: the
    current torch stream) and is not waited for."""
    import torch
    dev = torch.cuda.current_device()
    for name, t, dt in (("r_key", r_key, torch.int32), ("s_key", s_key, torch.int32),
                        ("out", out, torch.int64)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dt:
            raise ValueError(f"{name} must be a {dt} CUDA tensor")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if t.device.index != dev:
            raise ValueError(f"{name} is on cuda:{t.device.index}, not the current device "
                             f"cuda:{dev}")
    if out.numel() < 1:
        raise ValueError("out must hold at least one element")
    if stream is None:
        stream = _current_stream()
    st = _lib.fj_join2_count_noalloc(_vp(r_key.data_ptr()), r_key.numel(),
                                     _vp(s_key.data_ptr()), s_key.numel(),
                                     _vp(out.data_ptr()), _vp(stream))
    if st != 0:
        raise FJError(st, _lib.fj_noalloc_last_error().decode())


class Prepared:
    """fj_prepare / fj_build_colt_level / fj_execute_prepared / fj_reset_prepared."""

    def __init__(self, ctx, atoms, plan, head=None, out_mode="count", min_vars=None,
                 batch_size=0, load_factor=0.0, cover="static", list_limit=0, flags=0,
                 model=None, spin_limit=0):
        self.ctx = ctx
        self.min_vars = list(min_vars or [])
        self.out_mode = out_mode
        self.batch_size, self.load_factor = batch_size, load_factor
        self._head = list(head) if head is not None else None
        self._atoms_vars = [list(a["vars"]) for a in atoms]
        # The library borrows the relations' columns: keep them alive.
        self._rels = [a["rel"] for a in atoms]
        q, p = _QueryC(atoms, head), _PlanC(plan)
        o, mv = _opts(out_mode, min_vars, batch_size, load_factor, cover, list_limit, flags,
                      model, spin_limit)
        self.handle = _vp()
        _check(_lib.fj_prepare(ctx.handle, q.ptr, p.ptr, ctypes.byref(o), ctypes.byref(self.handle)))
        ctx._adopt(self)

    def build_level(self, atom, level):
        _check(_lib.fj_build_colt_level(self.handle, int(atom), int(level)))

    def execute(self):
        res = _Result()
        _check(_lib.fj_execute_prepared(self.handle, ctypes.byref(res)))
        tuples = (_take_tuples(self.ctx, res, res.n_head)
                  if self.out_mode in ("materialize", "factorized") else None)
        return Result(res, tuples, self.min_vars)

    def factor_layout(self):
        """fj_prepared_factor_layout: (width, prefix variables, tail atoms)."""
        w, npre, nt = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        pv = (ctypes.c_int * MAX_VARS)()
        ta = (ctypes.c_int * 16)()
        _check(_lib.fj_prepared_factor_layout(self.handle, ctypes.byref(w), ctypes.byref(npre), pv,
                                              ctypes.byref(nt), ta))
        return w.value, [pv[i] for i in range(npre.value)], [ta[i] for i in range(nt.value)]

    def expand(self, result):
        """fj_prepared_expand: the factorized `result` (this plan's last) as
        flat head-order tuples, an (count, n_head) int32 CUDA tensor."""
        import torch
        n_head = len(self._head) if self._head is not None else None
        raw = result._raw
        if n_head is None:
            n_head = len({v for a in self._atoms_vars for v in a})
        t = torch.empty((result.count, n_head), dtype=torch.int32, device=f"cuda:{self.ctx.device}")
        _check(_lib.fj_prepared_expand(self.handle, ctypes.byref(raw), _vp(t.data_ptr()),
                                       result.count))
        return t

    def execute_async(self):
        """Enqueue an execution; :meth:`result` waits for it."""
        _check(_lib.fj_execute_prepared_async(self.handle))

    def result(self):
        res = _Result()
        _check(_lib.fj_prepared_result(self.handle, ctypes.byref(res)))
        tuples = (_take_tuples(self.ctx, res, res.n_head)
                  if self.out_mode in ("materialize", "factorized") else None)
        return Result(res, tuples, self.min_vars)

    def reset(self):
        _check(_lib.fj_reset_prepared(self.handle))

    def free(self):
        if self.handle and self.ctx.handle:
            _lib.fj_prepared_free(self.handle)
        self.handle = _vp()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Batch:
    """fj_batch_create / fj_batch_execute: prepared queries run back to back
    from scratch with one synchronization; ``graph=True`` captures them once
    into a CUDA graph (FJ_BATCH_GRAPH) so each execution is one launch;
    ``concurrent=True`` (FJ_BATCH_CONCURRENT) spreads them over independent
    branches of the graph."""

    def __init__(self, ctx, preps, graph=False, concurrent=False):
        self.ctx = ctx
        self.preps = list(preps)
        arr = (_vp * max(1, len(self.preps)))(*[p.handle for p in self.preps])
        self.handle = _vp()
        flags = (1 if graph else 0) | (2 if concurrent else 0)
        _check(_lib.fj_batch_create(ctx.handle, len(self.preps), arr, flags,
                                    ctypes.byref(self.handle)))
        ctx._adopt(self)

    def execute(self):
        res = (_Result * max(1, len(self.preps)))()
        _check(_lib.fj_batch_execute(self.handle, res))
        return [Result(res[i], None, p.min_vars) for i, p in enumerate(self.preps)]

    def launch(self):
        """Enqueue the batch (fj_batch_launch); :meth:`results` waits."""
        _check(_lib.fj_batch_launch(self.handle))

    def results(self):
        res = (_Result * max(1, len(self.preps)))()
        _check(_lib.fj_batch_results(self.handle, res))
        return [Result(res[i], None, p.min_vars) for i, p in enumerate(self.preps)]

    def free(self):
        if self.handle:
            _lib.fj_batch_free(self.handle)
        self.handle = _vp()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def autotune(ctx, atoms, plan, out_mode="count", min_vars=None, cover="static",
             batch_sizes=(256, 1024, 4096, 8192), load_factors=(0.25, 0.5, 0.7), reps=2,
             times=None):
    """Pick the cover-batch size and hash-level load factor with the shortest
    execution (device time between CUDA events, best of ``reps`` runs from
    scratch) and return ``(prepared, (batch_size, load_factor), ms)``; the
    other candidates are freed.  Results do not depend on the choice.  When
    ``times`` is a dict it receives every candidate's time."""
    import torch
    best = None
    stream = torch.cuda.current_stream()
    for bs in batch_sizes:
        for lf in load_factors:
            p = Prepared(ctx, atoms, plan, out_mode=out_mode, min_vars=min_vars,
                         batch_size=bs, load_factor=lf, cover=cover)
            t = None
            for _ in range(reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                p.reset()
                e0.record(stream)
                p.execute_async()
                e1.record(stream)
                p.result()
                ms = e0.elapsed_time(e1)
                t = ms if t is None else min(t, ms)
            if times is not None:
                times[(bs, lf)] = t
            if best is None or t < best[2]:
                if best is not None:
                    best[0].free()
                best = (p, (bs, lf), t)
            else:
                p.free()
    return best


class Model:
    """fj_model_*: the chooser's three-layer perceptron (float32) with its
    CUDA forward, backward and descent kernels.  Inputs are float32 CUDA
    tensors of shape (n, in_dim); targets (n,)."""

    def __init__(self, ctx, in_dim, h1=128, h2=64, max_batch=8192):
        self.ctx = ctx
        self.shape = (int(in_dim), int(h1), int(h2))
        self.handle = _vp()
        st = _lib.fj_model_create(ctx.handle, int(in_dim), int(h1), int(h2), int(max_batch),
                                  ctypes.byref(self.handle))
        if st != 0:
            raise FJError(st, _lib.fj_model_last_error().decode())
        self.n_params = int(_lib.fj_model_n_params(self.handle))

    def _check(self, st):
        if st != 0:
            raise FJError(st, _lib.fj_model_last_error().decode())

    def set_params(self, theta):
        a = np.ascontiguousarray(theta, dtype=np.float32)
        self._check(_lib.fj_model_set_params(self.handle, _vp(a.ctypes.data), a.size))

    def params(self):
        a = np.empty(self.n_params, dtype=np.float32)
        self._check(_lib.fj_model_get_params(self.handle, _vp(a.ctypes.data), a.size))
        return a

    def forward(self, x):
        import torch
        x = x.contiguous()
        y = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
        self._check(_lib.fj_model_forward(self.handle, _vp(x.data_ptr()), x.shape[0],
                                          _vp(y.data_ptr())))
        return y

    def gradients(self, x, t):
        x, t = x.contiguous(), t.contiguous()
        g = np.empty(self.n_params, dtype=np.float32)
        loss = ctypes.c_float()
        self._check(_lib.fj_model_gradients(self.handle, _vp(x.data_ptr()), _vp(t.data_ptr()),
                                            x.shape[0], _vp(g.ctypes.data), ctypes.byref(loss)))
        return g, float(loss.value)

    def train_step(self, x, t, lr):
        x, t = x.contiguous(), t.contiguous()
        loss = ctypes.c_float()
        self._check(_lib.fj_model_train_step(self.handle, _vp(x.data_ptr()), _vp(t.data_ptr()),
                                             x.shape[0], float(lr), ctypes.byref(loss)))
        return float(loss.value)

    def set_scaler(self, mean, scale):
        m = np.ascontiguousarray(mean, dtype=np.float32)
        sc = np.ascontiguousarray(scale, dtype=np.float32)
        self._check(_lib.fj_model_set_scaler(self.handle, _vp(m.ctypes.data), _vp(sc.ctypes.data),
                                             m.size))

    def save(self, path):
        self._check(_lib.fj_model_save(self.handle, str(path).encode()))

    @classmethod
    def load(cls, ctx, path, max_batch=8192):
        m = cls.__new__(cls)
        m.ctx = ctx
        m.handle = _vp()
        st = _lib.fj_model_load(ctx.handle, str(path).encode(), int(max_batch),
                                ctypes.byref(m.handle))
        if st != 0:
            raise FJError(st, _lib.fj_model_last_error().decode())
        m.n_params = int(_lib.fj_model_n_params(m.handle))
        return m

    def free(self):
        if self.handle and self.ctx.handle:
            _lib.fj_model_free(self.handle)
        self.handle = _vp()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def degree_histogram(ctx, col, mod=100, seed=0):
    """fj_degree_histogram: the 32-bucket sampled key-degree histogram of an
    int32 CUDA tensor, as a numpy float32 array."""
    import torch
    if not isinstance(col, torch.Tensor) or not col.is_cuda or col.dtype != torch.int32:
        raise ValueError("col must be an int32 CUDA tensor")
    if col.device.index != ctx.device:
        raise ValueError(f"col is on cuda:{col.device.index}, the context on cuda:{ctx.device}")
    col = col.contiguous()
    out = np.zeros(32, dtype=np.float32)
    st = _lib.fj_degree_histogram(ctx.handle, _vp(col.data_ptr()), col.numel(), int(mod),
                                  int(seed), _vp(out.ctypes.data))
    if st != 0:
        raise FJError(st, _lib.fj_stats_last_error().decode())
    return out


def plan_features(ctx, atoms, candidates):
    """fj_plan_features: the chooser's features of each (order, cover policy
    name) candidate, as a numpy float32 array (len(candidates), CHOOSER_IN_DIM)."""
    q = _QueryC(atoms)
    cands = list(candidates)
    out = np.zeros((len(cands), CHOOSER_IN_DIM), dtype=np.float32)
    orders = _ints([a for o, _ in cands for a in o])
    pols = _ints([COVER[p] for _, p in cands])
    st = _lib.fj_plan_features(ctx.handle, q.ptr, len(cands), orders, pols, _vp(out.ctypes.data))
    if st != 0:
        raise FJError(st, _lib.fj_chooser_last_error().decode())
    return out


def choose_plan(ctx, atoms, model=None, max_candidates=24, seed=0):
    """fj_choose_plan: (plan, cover policy name, order) -- the candidate with
    the smallest predicted work, or the declared order with the static cover
    when ``model`` is None."""
    q = _QueryC(atoms)
    out = _P(_Plan)()
    pol = ctypes.c_int(0)
    order = (ctypes.c_int * len(atoms))()
    st = _lib.fj_choose_plan(ctx.handle, q.ptr, model.handle if model is not None else None,
                             int(max_candidates), int(seed), ctypes.byref(out), ctypes.byref(pol),
                             order)
    if st != 0:
        raise FJError(st, _lib.fj_chooser_last_error().decode())
    try:
        plan = _plan_from_c(out)
    finally:
        _lib.fj_plan_free(out)
    name = {v: k for k, v in COVER.items()}[pol.value]
    return plan, name, [order[i] for i in range(len(atoms))]
