"""CPU oracle for the query-processor hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The C code in ``oracle.c`` is a plain row-at-a-
time restatement of the paper's operators (Section 3.1 filter, Section 5.1
expressions, Sections 5.2-5.3 equi-join, Section 5.4 group-by aggregation);
this module only marshals numpy arrays into it.  It shares no code with the
CUDA library and never imports it.

A plan is given as plain Python data:

* ``fact`` / ``dim``: lists of 1-D numpy arrays (int32, int64 or uint8).
* ``preds``: ``(col, op, lo, hi)`` with op in ``lt le gt ge eq ne between``
  (``between`` is inclusive); all predicates are ANDed.
* expressions: postfix token lists -- ``("col", i)``, ``("const", v)``,
  ``"add"``, ``"sub"``, ``"mul"``; column ``i`` addresses fact columns first,
  then dim columns.
* ``aggs``: ``(fn, expr)`` with fn in ``sum count avg min max``.
* string columns: 2-D uint8 arrays ``(n, width)``, one character per byte,
  right-padded with 0 (Section 4.1); they take ``(col, "in", values)``,
  ``(col, "like", pattern)`` and ``(col, "not_like", pattern)`` only (values
  and patterns as ``str`` or ``bytes``); ``(col, "in", ints)`` also applies to
  numeric columns.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
_SRC_MT = os.path.join(_HERE, "oracle_mt.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LOCK = threading.Lock()
_LIB = None

OK, ERR_INVALID, ERR_CAPACITY, ERR_OVERFLOW, ERR_NOMEM = 0, 1, 4, 5, 6
_TYPES = {np.dtype(np.int32): 0, np.dtype(np.int64): 1, np.dtype(np.uint8): 2}
_OPS = {"lt": 0, "le": 1, "gt": 2, "ge": 3, "eq": 4, "ne": 5, "between": 6, "in": 7, "like": 8, "not_like": 9}
CHAR = 3
_XK = {"col": 0, "const": 1, "add": 2, "sub": 3, "mul": 4}
_FNS = {"sum": 0, "count": 1, "avg": 2, "min": 3, "max": 4}
MAX_EXPR = 8


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (plain C11, no fast-math)."""
    newest = max(os.path.getmtime(f) for f in (_SRC, _SRC_MT, _HDR))
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fno-fast-math", "-fPIC", "-shared", "-pthread",
                               "-o", tmp, _SRC, _SRC_MT, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class Col(C.Structure):
    _fields_ = [("data", C.c_void_p), ("type", C.c_int32), ("width", C.c_int32)]


class Pred(C.Structure):
    _fields_ = [("col", C.c_int32), ("op", C.c_int32), ("lo", C.c_int64), ("hi", C.c_int64)]


class Expr(C.Structure):
    _fields_ = [("n", C.c_int32), ("kind", C.c_int32 * MAX_EXPR), ("v", C.c_int64 * MAX_EXPR)]


class Agg(C.Structure):
    _fields_ = [("fn", C.c_int32), ("pad", C.c_int32), ("expr", Expr)]


class Plan(C.Structure):
    _fields_ = [("nfact", C.c_int64), ("fact", C.POINTER(Col)), ("nfact_cols", C.c_int32), ("pad0", C.c_int32),
                ("preds", C.POINTER(Pred)), ("npreds", C.c_int32), ("pad1", C.c_int32),
                ("ndim", C.c_int64), ("dim", C.POINTER(Col)), ("ndim_cols", C.c_int32),
                ("fact_fk", C.c_int32), ("dim_key", C.c_int32), ("join_kind", C.c_int32),
                ("group_cols", C.POINTER(C.c_int32)), ("ngc", C.c_int32), ("pad3", C.c_int32),
                ("aggs", C.POINTER(Agg)), ("naggs", C.c_int32), ("pad4", C.c_int32),
                ("sum_expr", C.POINTER(Expr)),
                ("topk", C.c_int32), ("topk_agg", C.c_int32)]


class Out(C.Structure):
    _fields_ = [("row_ids", C.POINTER(C.c_int32)), ("cap_rows", C.c_int64), ("num_rows", C.c_int64),
                ("pair_fact", C.POINTER(C.c_int32)), ("pair_dim", C.POINTER(C.c_int32)),
                ("cap_pairs", C.c_int64), ("num_pairs", C.c_int64),
                ("sum", C.c_int64),
                ("keys", C.POINTER(C.c_int64)), ("ivals", C.POINTER(C.c_int64)), ("fvals", C.POINTER(C.c_double)),
                ("cap_groups", C.c_int64), ("num_groups", C.c_int64), ("total_groups", C.c_int64)]


def lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            _LIB = C.CDLL(build())
            _LIB.oracle_plan.argtypes = [C.POINTER(Plan), C.POINTER(Out)]
            _LIB.oracle_plan.restype = C.c_int
            _LIB.oracle_filter_mt.argtypes = [C.POINTER(Plan), C.POINTER(Out), C.c_int]
            _LIB.oracle_filter_mt.restype = C.c_int
    return _LIB


def _cols(arrs):
    arrs = [np.ascontiguousarray(a) for a in arrs]
    cs = (Col * max(1, len(arrs)))()
    for i, a in enumerate(arrs):
        if a.dtype not in _TYPES:
            raise TypeError(f"unsupported column dtype {a.dtype}")
        cs[i].data = a.ctypes.data
        if a.ndim == 2:  # a string column
            if a.dtype != np.uint8:
                raise TypeError("string columns are uint8 (n, width) arrays")
            cs[i].type, cs[i].width = CHAR, a.shape[1]
        else:
            cs[i].type = _TYPES[a.dtype]
    return cs, arrs


def _bytes(v) -> bytes:
    return v.encode("latin-1") if isinstance(v, str) else bytes(v)


def pad_strings(values, width: int) -> np.ndarray:
    """``(k, width)`` uint8 rows: each value's bytes, right-padded with 0."""
    out = np.zeros((len(values), width), np.uint8)
    for i, v in enumerate(values):
        b = _bytes(v)
        if len(b) > width:
            raise ValueError(f"string {b!r} longer than the column width {width}")
        out[i, :len(b)] = np.frombuffer(b, np.uint8)
    return out


def _set_pred(pred, op, col, keep):
    """lo / hi of an IN, LIKE or NOT LIKE predicate on column array ``col`` (buffers appended to ``keep``)."""
    if op == "in":
        if col.ndim == 2:
            buf = pad_strings(pred, col.shape[1])
        else:
            buf = np.ascontiguousarray(np.asarray(list(pred), dtype=np.int64))
        n = len(buf)
    else:
        buf = np.frombuffer(_bytes(pred), np.uint8).copy()
        n = len(buf)
    keep.append(buf)
    return (buf.ctypes.data if n else 0), n


def _expr(tokens) -> Expr:
    e = Expr()
    toks = list(tokens)
    if len(toks) > MAX_EXPR:
        raise ValueError("expression longer than 8 tokens")
    e.n = len(toks)
    for i, t in enumerate(toks):
        if isinstance(t, str):
            e.kind[i] = _XK[t]
        else:
            e.kind[i] = _XK[t[0]]
            e.v[i] = int(t[1])
    return e


def _ptr(a, ct):
    return a.ctypes.data_as(C.POINTER(ct)) if a is not None else None


def load_variant(so_path: str):
    """Load another build of ``oracle.c`` (used by tests that plant mistakes in a copy)."""
    L = C.CDLL(so_path)
    L.oracle_plan.argtypes = [C.POINTER(Plan), C.POINTER(Out)]
    L.oracle_plan.restype = C.c_int
    return L


_JOINS = {"inner": 0, "semi": 1, "anti": 2, "left_outer": 3}


def run_plan(fact, preds=(), dim=None, fact_fk=0, dim_key=0, group_cols=(), aggs=(), sum_expr=None,
             topk=0, topk_agg=0, want_row_ids=True, want_pairs=False, cap_groups=None, join_kind="inner",
             threads=1, _lib=None):
    """Evaluate one plan with the C oracle; returns a dict of numpy results.
    join_kind: "inner" (every equal-key pair), "semi" / "anti" (each fact row
    once if it has a / no equal-key dim row; fact columns only), "left_outer"
    (the inner pairs, and each fact row without a match once with dim row -1;
    fact columns only).
    threads > 1 (filter plans only: no join, no grouping) evaluates row ranges
    on that many threads with the same row loop (oracle_filter_mt) -- the
    all-core CPU baseline; the result is identical."""
    if threads > 1 and (dim is not None or len(group_cols) or len(aggs)):
        raise ValueError("threads > 1 is for filter plans only")
    L = _lib if _lib is not None else lib()
    fcols, fkeep = _cols(fact)
    fkeep_bufs = []  # IN lists and LIKE patterns, alive until the call returns
    nfact = len(fkeep[0]) if fkeep else 0
    dcols, dkeep = _cols(dim or [])
    pr = (Pred * max(1, len(preds)))()
    for i, (c, op, lo, *hi) in enumerate(preds):
        if op in ("in", "like", "not_like"):
            pr[i].col, pr[i].op = int(c), _OPS[op]
            pr[i].lo, pr[i].hi = _set_pred(lo, op, fkeep[int(c)], fkeep_bufs)
            continue
        pr[i].col, pr[i].op, pr[i].lo = int(c), _OPS[op], int(lo)
        pr[i].hi = int(hi[0]) if hi else 0
    gc = np.ascontiguousarray(np.asarray(group_cols, dtype=np.int32).reshape(-1))
    ag = (Agg * max(1, len(aggs)))()
    for i, (fn, ex) in enumerate(aggs):
        ag[i].fn = _FNS[fn]
        if ex is not None:
            ag[i].expr = _expr(ex)
    se = _expr(sum_expr) if sum_expr is not None else None

    p = Plan()
    p.nfact, p.fact, p.nfact_cols = nfact, fcols, len(fkeep)
    p.preds, p.npreds = pr, len(preds)
    p.ndim, p.dim, p.ndim_cols = (len(dkeep[0]) if dkeep else 0), dcols, len(dkeep)
    p.fact_fk, p.dim_key = int(fact_fk), int(dim_key)
    p.join_kind = _JOINS[join_kind]
    p.group_cols, p.ngc = gc.ctypes.data_as(C.POINTER(C.c_int32)), len(gc)
    p.aggs, p.naggs = ag, len(aggs)
    p.sum_expr = C.pointer(se) if se is not None else None
    p.topk, p.topk_agg = int(topk), int(topk_agg)

    na = len(aggs)
    ngc = len(gc)
    cap_rows = nfact if want_row_ids else 0
    cap_pairs = (nfact if dim is None else max(16, nfact)) if want_pairs else 0
    if cap_groups is None:
        cap_groups = (int(topk) if topk else min(max(nfact, 1), 1 << 16)) if (ngc or na) else 0
    for _attempt in range(3):
        row_ids = np.empty(max(cap_rows, 1), np.int32) if want_row_ids else None
        pf = np.empty(max(cap_pairs, 1), np.int32) if want_pairs else None
        pd = np.empty(max(cap_pairs, 1), np.int32) if want_pairs else None
        keys = np.empty(max(cap_groups * ngc, 1), np.int64)
        iv = np.empty(max(cap_groups * na, 1), np.int64)
        fv = np.empty(max(cap_groups * na, 1), np.float64)
        o = Out()
        o.row_ids, o.cap_rows = _ptr(row_ids, C.c_int32), cap_rows
        o.pair_fact, o.pair_dim, o.cap_pairs = _ptr(pf, C.c_int32), _ptr(pd, C.c_int32), cap_pairs
        o.keys, o.ivals, o.fvals, o.cap_groups = _ptr(keys, C.c_int64), _ptr(iv, C.c_int64), _ptr(fv, C.c_double), cap_groups
        if threads > 1:
            st = L.oracle_filter_mt(C.byref(p), C.byref(o), int(threads))
        else:
            st = L.oracle_plan(C.byref(p), C.byref(o))
        if st == ERR_CAPACITY:
            cap_rows = max(cap_rows, o.num_rows) if want_row_ids else 0
            cap_pairs = max(cap_pairs, o.num_pairs) if want_pairs else 0
            cap_groups = max(cap_groups, o.num_groups)
            continue
        break
    if st != OK:
        raise OracleError(st)
    G = o.num_groups
    res = {
        "status": st,
        "num_rows": o.num_rows,
        "num_pairs": o.num_pairs,
        "sum": o.sum,
        "num_groups": G,
        "total_groups": o.total_groups,
        "keys": keys[:G * ngc].reshape(G, ngc).copy(),
        "ivals": iv[:G * na].reshape(G, na).copy(),
        "fvals": fv[:G * na].reshape(G, na).copy(),
    }
    if want_row_ids:
        res["row_ids"] = row_ids[:o.num_rows].copy()
    if want_pairs:
        res["pair_fact"] = pf[:o.num_pairs].copy()
        res["pair_dim"] = pd[:o.num_pairs].copy()
    return res


class OracleError(RuntimeError):
    def __init__(self, status):
        super().__init__(f"oracle status {status}")
        self.status = status


# Convenience wrappers with the operator-level shapes of the library calls.

def filter_rows(fact, preds, sum_expr=None, threads=1):
    """Row ids (ascending) of rows passing every predicate, and SUM(sum_expr)."""
    r = run_plan(fact, preds, sum_expr=sum_expr, want_row_ids=True, threads=threads)
    return r["row_ids"], r["sum"]


def groupby(fact, preds, group_cols, aggs, topk=0, topk_agg=0):
    r = run_plan(fact, preds, group_cols=group_cols, aggs=aggs, topk=topk, topk_agg=topk_agg, want_row_ids=False)
    return r["keys"], r["ivals"], r["fvals"]


def join_pairs(build_keys, probe_keys, join_kind="inner"):
    """Equi-join index pairs (build_idx, probe_idx) in (probe, build) ascending order (left outer: a probe row
    without a match once, with build_idx -1)."""
    r = run_plan([probe_keys], (), dim=[build_keys], fact_fk=0, dim_key=0, want_row_ids=False, want_pairs=True,
                 join_kind=join_kind)
    return r["pair_dim"], r["pair_fact"]
