"""Python binding of libtqp (GB300 columnar relational operators).

Thin ctypes marshalling over the C ABI in ``include/tqp.h``: every function
here has the name of the C entry point it calls and only converts Python
values (torch CUDA tensors, tuples) into the C structs.  All computation runs
in the CUDA kernels of ``libtqp.so``; there is no CPU fallback -- importing
works without the library, but every call raises if it is missing.

Plan vocabulary (shared with the tests):

* predicates ``(col, op, lo[, hi])`` with op in ``lt le gt ge eq ne between``;
* expressions: postfix token lists ``("col", i)``, ``("const", v)``, ``"add"``,
  ``"sub"``, ``"mul"``;
* aggregates ``(fn, expr)`` with fn in ``sum count avg min max`` (MIN/MAX: few-group
  aggregations without a join, see include/tqp.h).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtqp.so")
_LOCK = threading.Lock()
_LIB = None

OK, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_OUT_OF_MEMORY, ERR_CAPACITY, ERR_OVERFLOW, ERR_TIMEOUT, ERR_CUDA = range(8)
I32, I64, U8, CHAR = 0, 1, 2, 3
MAX_PREDS, MAX_EXPR, MAX_GROUP_COLS, MAX_AGGS, MAX_COLS = 8, 8, 4, 8, 16
_OPS = {"lt": 0, "le": 1, "gt": 2, "ge": 3, "eq": 4, "ne": 5, "between": 6, "in": 7, "like": 8, "not_like": 9}
_XOPS = {"col": 0, "const": 1, "add": 2, "sub": 3, "mul": 4}
_FNS = {"sum": 0, "count": 1, "avg": 2, "min": 3, "max": 4}


class TqpError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"tqp status {status}: {msg}")
        self.status = status


class Column(C.Structure):
    _fields_ = [("data", C.c_void_p), ("type", C.c_int32), ("scale", C.c_int32)]


class Table(C.Structure):
    _fields_ = [("num_rows", C.c_int64), ("num_cols", C.c_int32), ("reserved", C.c_int32),
                ("cols", C.POINTER(Column))]


class Pred(C.Structure):
    _fields_ = [("col", C.c_int32), ("op", C.c_int32), ("lo", C.c_int64), ("hi", C.c_int64)]


class Expr(C.Structure):
    _fields_ = [("n", C.c_int32), ("op", C.c_int32 * MAX_EXPR), ("v", C.c_int64 * MAX_EXPR)]


class Agg(C.Structure):
    _fields_ = [("fn", C.c_int32), ("reserved", C.c_int32), ("expr", Expr)]


class Plan(C.Structure):
    _fields_ = [("fact", C.POINTER(Table)),
                ("preds", Pred * MAX_PREDS), ("npreds", C.c_int32), ("emit_row_ids", C.c_int32),
                ("dim", C.POINTER(Table)), ("fact_fk", C.c_int32), ("dim_key", C.c_int32),
                ("group_cols", C.c_int32 * MAX_GROUP_COLS), ("ngc", C.c_int32), ("naggs", C.c_int32),
                ("aggs", Agg * MAX_AGGS),
                ("has_sum", C.c_int32), ("topk", C.c_int32),
                ("sum_expr", Expr),
                ("topk_agg", C.c_int32), ("join_kind", C.c_int32), ("max_groups", C.c_int64),
                ("prepared", C.c_void_p)]


class ScanQuery(C.Structure):
    _fields_ = [("preds", Pred * MAX_PREDS), ("npreds", C.c_int32), ("has_sum", C.c_int32),
                ("sum_expr", Expr), ("d_count", C.c_void_p), ("d_sum", C.c_void_p)]


class Result(C.Structure):
    _fields_ = [("d_row_ids", C.c_void_p), ("capacity_rows", C.c_int64), ("d_num_rows", C.c_void_p),
                ("d_sum", C.c_void_p),
                ("d_keys", C.c_void_p), ("d_ivals", C.c_void_p), ("d_fvals", C.c_void_p),
                ("capacity_groups", C.c_int64), ("d_num_groups", C.c_void_p), ("d_total_groups", C.c_void_p),
                ("d_num_joined", C.c_void_p)]


_P = C.c_void_p
_SIGS = {
    "tqp_ctx_create": (C.c_int, [C.c_int, _P, C.c_size_t, C.POINTER(_P)]),
    "tqp_ctx_destroy": (C.c_int, [_P]),
    "tqp_ctx_check": (C.c_int, [_P, _P]),
    "tqp_ctx_set_wait_limit": (C.c_int, [_P, C.c_int64]),
    "tqp_ctx_arena_bytes": (C.c_size_t, [_P]),
    "tqp_ctx_set_tuning": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_int32]),
    "tqp_ctx_set_variant": (C.c_int, [_P, C.c_int32]),
    "tqp_ctx_set_jit": (C.c_int, [_P, C.c_int32]),
    "tqp_jit_stats": (None, [C.POINTER(C.c_int64)]),
    "tqp_jit_probe": (C.c_int, []),
    "tqp_last_error": (C.c_char_p, []),
    "tqp_status_string": (C.c_char_p, [C.c_int]),
    "tqp_version": (C.c_int, []),
    "tqp_filter": (C.c_int, [_P, C.POINTER(Table), C.POINTER(Pred), C.c_int32, C.POINTER(Expr), _P, _P,
                             C.c_int64, _P, _P]),
    "tqp_filter_noalloc": (C.c_int, [C.c_int, C.POINTER(Table), C.POINTER(Pred), C.c_int32, C.POINTER(Expr), _P,
                                     _P, C.c_int64, _P, _P, _P]),
    "tqp_filter_shared": (C.c_int, [_P, C.POINTER(Table), C.POINTER(ScanQuery), C.c_int32,
                                    C.POINTER(C.c_int32), _P]),
    "tqp_groupby_agg": (C.c_int, [_P, C.POINTER(Table), C.POINTER(Pred), C.c_int32, C.POINTER(C.c_int32),
                                  C.c_int32, C.POINTER(Agg), C.c_int32, _P, _P, _P, C.c_int64, _P, _P]),
    "tqp_hash_join": (C.c_int, [_P, C.POINTER(Table), C.c_int32, C.POINTER(Table), C.c_int32, _P, _P,
                                C.c_int64, _P, _P]),
    "tqp_hash_join_kind": (C.c_int, [_P, C.POINTER(Table), C.c_int32, C.POINTER(Table), C.c_int32, C.c_int32, _P,
                                     _P, C.c_int64, _P, _P]),
    "tqp_run_plan": (C.c_int, [_P, C.POINTER(Plan), C.POINTER(Result), _P]),
    "tqp_run_plans": (C.c_int, [_P, C.POINTER(Plan), C.POINTER(Result), C.c_int32, _P]),
    "tqp_batch_create": (C.c_int, [_P, C.POINTER(Plan), C.POINTER(Result), C.c_int32, C.POINTER(_P)]),
    "tqp_batch_run": (C.c_int, [_P, _P]),
    "tqp_batch_destroy": (C.c_int, [_P]),
    "tqp_dim_prepare": (C.c_int, [_P, C.POINTER(Table), C.c_int32, C.POINTER(C.c_int32), C.c_int32, C.c_int64, _P,
                                  C.POINTER(_P)]),
    "tqp_dim_groups": (C.c_int64, [_P]),
    "tqp_dim_destroy": (C.c_int, [_P]),
    "tqp_ctx_set_autotune": (C.c_int, [_P, C.c_int32]),
    "tqp_ctx_tuned_count": (C.c_int32, [_P]),
    "tqp_ctx_save_tuning": (C.c_int, [_P, C.c_char_p]),
    "tqp_ctx_load_tuning": (C.c_int, [_P, C.c_char_p]),
    "tqp_server_create": (C.c_int, [_P, C.c_void_p, C.POINTER(_P)]),
    "tqp_server_submit": (C.c_int, [_P, C.POINTER(Plan), C.POINTER(Result), C.c_uint64]),
    "tqp_server_poll": (C.c_int32, [_P, C.c_void_p, C.c_int32]),
    "tqp_server_drain": (C.c_int, [_P, C.c_double]),
    "tqp_server_destroy": (C.c_int, [_P]),
    "tqp_measure_l2_red": (C.c_int, [C.c_int, _P, C.c_int64, C.c_int64, C.c_int32, C.c_int32, C.c_int32, _P]),
    "tqp_measure_scan_rate": (C.c_int, [_P, C.POINTER(Table), C.c_int32, C.c_int32, C.c_int32, _P, _P]),
}


def lib():
    """Load libtqp.so (raises if it has not been built)."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libtqp.so not built ({LIB_PATH}); run __graft_entry__.build()")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name, None)
                if f is None:
                    continue
                f.restype = res
                f.argtypes = args
            _LIB = L
    return _LIB


def _check(status: int):
    if status != OK:
        raise TqpError(status, lib().tqp_last_error().decode())


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _dtype_code(t) -> int:
    import torch
    m = {torch.int32: I32, torch.int64: I64, torch.uint8: U8}
    if t.dtype not in m:
        raise TypeError(f"unsupported column dtype {t.dtype}")
    return m[t.dtype]


class TableRef:
    """A tqp_table over CUDA tensors (keeps the tensors and C structs alive).
    With host_ok, a column may also be a pinned CPU tensor: tqp_filter reads
    such a column in place at passing rows (a projected column); every other
    use is rejected by the library."""

    def __init__(self, cols, scales=None, host_ok=False):
        """A 2-D uint8 tensor (n, width) is a string column (one character per byte, right-padded with 0)."""
        import torch
        cols = list(cols)
        if not cols:
            raise ValueError("a table needs at least one column")
        rows = lambda c: c.shape[0] if c.dim() == 2 else c.numel()  # noqa: E731
        n = rows(cols[0])
        for c in cols:
            on_host = host_ok and not c.is_cuda and c.is_pinned()
            if not (c.is_cuda or on_host) or not c.is_contiguous() or rows(c) != n:
                raise ValueError("columns must be contiguous CUDA tensors (or pinned host tensors with host_ok) "
                                 "of equal length")
            if c.dim() == 2 and c.dtype != torch.uint8:
                raise TypeError("string columns are uint8 (n, width) tensors")
        self.tensors = cols
        self.widths = [c.shape[1] if c.dim() == 2 else 0 for c in cols]
        self.carr = (Column * len(cols))()
        for i, c in enumerate(cols):
            self.carr[i].data = c.data_ptr()
            if c.dim() == 2:
                self.carr[i].type, self.carr[i].scale = CHAR, c.shape[1]
            else:
                self.carr[i].type = _dtype_code(c)
                self.carr[i].scale = (scales[i] if scales else 0)
        self.t = Table(n, len(cols), 0, self.carr)

    @property
    def num_rows(self):
        return self.t.num_rows

    def ref(self):
        return C.byref(self.t)


def make_expr(tokens) -> Expr:
    e = Expr()
    toks = list(tokens)
    if len(toks) > MAX_EXPR:
        raise ValueError("expression longer than 8 tokens")
    e.n = len(toks)
    for i, tk in enumerate(toks):
        if isinstance(tk, str):
            e.op[i] = _XOPS[tk]
        else:
            e.op[i] = _XOPS[tk[0]]
            e.v[i] = int(tk[1])
    return e


def _bytes(v) -> bytes:
    return v.encode("latin-1") if isinstance(v, str) else bytes(v)


def _set_operand(table, col, op, v, keep):
    """lo / hi of an IN, LIKE or NOT LIKE predicate: the host address and count of its values (IN: int64
    numbers, or the column width's 0-padded strings) or of its pattern bytes; the buffer goes to `keep`."""
    import numpy as np
    width = table.widths[col] if table is not None and 0 <= col < len(table.widths) else 0
    if op == "in":
        vals = list(v)
        if width:
            buf = np.zeros((len(vals), width), np.uint8)
            for k, x in enumerate(vals):
                b = _bytes(x)
                if len(b) > width:
                    raise ValueError(f"IN value {b!r} longer than the column width {width}")
                buf[k, :len(b)] = np.frombuffer(b, np.uint8)
        elif vals and isinstance(vals[0], (str, bytes)):
            raise ValueError("IN with strings needs the table (to know the column width)")
        else:
            buf = np.asarray(vals, dtype=np.int64).reshape(-1)
    else:
        buf = np.frombuffer(_bytes(v), np.uint8).copy()
    buf = np.ascontiguousarray(buf)
    keep.append(buf)
    n = len(buf)
    return (buf.ctypes.data if n else 0), n


def _fill_pred(dst, table, pred, keep):
    c, op, lo, *hi = pred
    dst.col, dst.op = int(c), _OPS[op]
    if op in ("in", "like", "not_like"):
        dst.lo, dst.hi = _set_operand(table, int(c), op, lo, keep)
    else:
        dst.lo = int(lo)
        dst.hi = int(hi[0]) if hi else 0


def make_preds(preds, table=None):
    """Predicates (col, op, lo[, hi]); op "in" takes a list of values, "like" / "not_like" a pattern (str or
    bytes).  The array keeps the value buffers alive (``_keep``)."""
    arr = (Pred * max(1, len(preds)))()
    keep = []
    for i, pr in enumerate(preds):
        _fill_pred(arr[i], table, pr, keep)
    arr._keep = keep
    return arr


def make_aggs(aggs):
    arr = (Agg * max(1, len(aggs)))()
    for i, (fn, ex) in enumerate(aggs):
        arr[i].fn = _FNS[fn]
        if ex is not None:
            arr[i].expr = make_expr(ex)
    return arr


def tqp_jit_stats() -> dict:
    """Process-wide run-time specialisation counters."""
    out = (C.c_int64 * 4)()
    lib().tqp_jit_stats(out)
    return {"compiled": out[0], "from_disk": out[1], "launches": out[2], "failed": out[3]}


def tqp_jit_probe() -> None:
    """Raise TqpError unless NVRTC and the kernel sources are found and a sample shape compiles."""
    _check(lib().tqp_jit_probe())


class Context:
    """A libtqp context; the scratch arena is a torch CUDA allocation."""

    def __init__(self, device: int = 0, arena_bytes: int = 1 << 30):
        import torch
        self.device = device
        self.arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device=f"cuda:{device}")
        h = C.c_void_p()
        _check(lib().tqp_ctx_create(device, C.c_void_p(self.arena.data_ptr()), int(arena_bytes), C.byref(h)))
        self.h = h

    def check(self, stream=None):
        _check(lib().tqp_ctx_check(self.h, _stream(stream)))

    def status(self, stream=None) -> int:
        """Like check(), but returns the status code instead of raising."""
        return lib().tqp_ctx_check(self.h, _stream(stream))

    def set_tuning(self, tile_rows: int = 0, stages: int = 0, ctas_per_sm: int = 0):
        _check(lib().tqp_ctx_set_tuning(self.h, int(tile_rows), int(stages), int(ctas_per_sm)))

    def set_variant(self, variant: int = -1):
        """Force the algorithm of two-algorithm operators (grouped join plans: 0 radix-partitioned, 1 fused
        probe); -1 restores the default."""
        _check(lib().tqp_ctx_set_variant(self.h, int(variant)))

    def set_jit(self, mode: int = 1):
        """Run-time specialisation of the few-groups aggregate: 0 off, 1 inputs of 16M rows or more
        (default), 2 always."""
        _check(lib().tqp_ctx_set_jit(self.h, int(mode)))

    def set_autotune(self, enable: bool = True):
        _check(lib().tqp_ctx_set_autotune(self.h, int(bool(enable))))

    @property
    def tuned_count(self) -> int:
        return int(lib().tqp_ctx_tuned_count(self.h))

    def save_tuning(self, path: str):
        _check(lib().tqp_ctx_save_tuning(self.h, os.fsencode(path)))

    def load_tuning(self, path: str):
        _check(lib().tqp_ctx_load_tuning(self.h, os.fsencode(path)))

    def set_wait_limit(self, polls: int):
        _check(lib().tqp_ctx_set_wait_limit(self.h, int(polls)))

    def close(self):
        if getattr(self, "h", None):
            lib().tqp_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- entry points (same names as the C ABI) ---------------------------------

def tqp_filter(ctx: Context, table: TableRef, preds=(), sum_expr=None, d_sum=None, d_row_ids=None,
               capacity: int = 0, d_count=None, stream=None):
    pa = make_preds(preds, table)
    se = C.byref(make_expr(sum_expr)) if sum_expr is not None else None
    _check(lib().tqp_filter(ctx.h, table.ref(), pa, len(preds), se, _ptr(d_sum), _ptr(d_row_ids),
                            int(capacity), _ptr(d_count), _stream(stream)))


def tqp_filter_noalloc(device: int, table: TableRef, preds=(), sum_expr=None, d_sum=None, d_row_ids=None,
                       capacity: int = 0, d_count=None, d_status=None, stream=None):
    """tqp_filter without a context, for callers that cannot allocate device
    memory; its scratch is a fixed array inside libtqp (see include/tqp.h)."""
    pa = make_preds(preds, table)
    se = C.byref(make_expr(sum_expr)) if sum_expr is not None else None
    _check(lib().tqp_filter_noalloc(int(device), table.ref(), pa, len(preds), se, _ptr(d_sum), _ptr(d_row_ids),
                                    int(capacity), _ptr(d_count), _ptr(d_status), _stream(stream)))


def make_scan_queries(queries, table=None):
    """queries: (preds, sum_expr or None, d_count, d_sum or None) tuples."""
    arr = (ScanQuery * max(1, len(queries)))()
    keep = []
    arr._keep = keep
    for i, (preds, ex, d_count, d_sum) in enumerate(queries):
        if len(preds) > MAX_PREDS:
            raise ValueError("more than 8 predicates")
        for j, pr in enumerate(preds):
            _fill_pred(arr[i].preds[j], table, pr, keep)
        arr[i].npreds = len(preds)
        if ex is not None:
            arr[i].has_sum = 1
            arr[i].sum_expr = make_expr(ex)
        arr[i].d_count = None if d_count is None else d_count.data_ptr()
        arr[i].d_sum = None if d_sum is None else d_sum.data_ptr()
    return arr


class ScanQueries:
    """Queries marshalled once (make_scan_queries) for repeated tqp_filter_shared calls."""

    def __init__(self, queries, table=None):
        self.n = len(queries)
        self.arr = make_scan_queries(queries, table)
        self.launch_of = (C.c_int32 * max(1, self.n))()


def tqp_filter_shared(ctx: Context, table: TableRef, queries, stream=None):
    """Shared scans: each (preds, sum_expr, d_count, d_sum) query gets what
    tqp_filter without row ids gives it.  `queries` is a list of such tuples or
    a ScanQueries.  Returns each query's launch index (-1: it ran alone through
    the single-query scan)."""
    q = queries if isinstance(queries, ScanQueries) else ScanQueries(queries, table)
    _check(lib().tqp_filter_shared(ctx.h, table.ref(), q.arr, q.n, q.launch_of, _stream(stream)))
    return [int(q.launch_of[i]) for i in range(q.n)]


def tqp_groupby_agg(ctx: Context, table: TableRef, preds, group_cols, aggs, d_keys, d_ivals, d_fvals,
                    capacity_groups: int, d_num_groups, stream=None):
    pa = make_preds(preds, table)
    gc = (C.c_int32 * max(1, len(group_cols)))(*[int(c) for c in group_cols])
    ag = make_aggs(aggs)
    _check(lib().tqp_groupby_agg(ctx.h, table.ref(), pa, len(preds), gc, len(group_cols), ag, len(aggs),
                                 _ptr(d_keys), _ptr(d_ivals), _ptr(d_fvals), int(capacity_groups),
                                 _ptr(d_num_groups), _stream(stream)))


def tqp_hash_join(ctx: Context, build: TableRef, build_key: int, probe: TableRef, probe_key: int,
                  d_build_idx, d_probe_idx, capacity: int, d_count, stream=None):
    _check(lib().tqp_hash_join(ctx.h, build.ref(), int(build_key), probe.ref(), int(probe_key),
                               _ptr(d_build_idx), _ptr(d_probe_idx), int(capacity), _ptr(d_count),
                               _stream(stream)))


JOIN_KINDS = {"inner": 0, "semi": 1, "anti": 2, "left_outer": 3}


def tqp_hash_join_kind(ctx: Context, build: TableRef, build_key: int, probe: TableRef, probe_key: int, join_kind,
                       d_build_idx, d_probe_idx, capacity: int, d_count, stream=None):
    """tqp_hash_join for a join kind ("inner", "semi", "anti", "left_outer" or its tqp_join_kind code)."""
    kind = JOIN_KINDS[join_kind] if isinstance(join_kind, str) else int(join_kind)
    _check(lib().tqp_hash_join_kind(ctx.h, build.ref(), int(build_key), probe.ref(), int(probe_key), kind,
                                    _ptr(d_build_idx), _ptr(d_probe_idx), int(capacity), _ptr(d_count),
                                    _stream(stream)))


def make_plan(fact: TableRef, preds=(), dim: TableRef | None = None, fact_fk=0, dim_key=0, group_cols=(),
              aggs=(), sum_expr=None, topk=0, topk_agg=0, emit_row_ids=False, max_groups=0,
              prepared: "PreparedDim | None" = None, join_kind="inner") -> Plan:
    p = Plan()
    p.fact = C.pointer(fact.t)
    if len(preds) > MAX_PREDS or len(group_cols) > MAX_GROUP_COLS or len(aggs) > MAX_AGGS:
        raise ValueError("plan exceeds the fixed plan limits")
    pa = make_preds(preds, fact)
    for i in range(len(preds)):
        p.preds[i] = pa[i]
    p._keep = pa._keep
    p.npreds = len(preds)
    p.emit_row_ids = int(bool(emit_row_ids))
    p.dim = C.pointer(dim.t) if dim is not None else None
    p.fact_fk, p.dim_key = int(fact_fk), int(dim_key)
    for i, c in enumerate(group_cols):
        p.group_cols[i] = int(c)
    p.ngc = len(group_cols)
    ag = make_aggs(aggs)
    for i in range(len(aggs)):
        p.aggs[i] = ag[i]
    p.naggs = len(aggs)
    if sum_expr is not None:
        p.has_sum = 1
        p.sum_expr = make_expr(sum_expr)
    p.topk, p.topk_agg = int(topk), int(topk_agg)
    p.max_groups = int(max_groups)
    p.join_kind = JOIN_KINDS[join_kind] if isinstance(join_kind, str) else int(join_kind)
    p.prepared = prepared.h if prepared is not None else None
    p._keep = (fact, dim, prepared)  # keep the tables' C structs alive
    return p


def make_result(d_row_ids=None, capacity_rows=0, d_num_rows=None, d_sum=None, d_keys=None, d_ivals=None,
                d_fvals=None, capacity_groups=0, d_num_groups=None, d_total_groups=None,
                d_num_joined=None) -> Result:
    r = Result(_ptr(d_row_ids), int(capacity_rows), _ptr(d_num_rows), _ptr(d_sum), _ptr(d_keys), _ptr(d_ivals),
               _ptr(d_fvals), int(capacity_groups), _ptr(d_num_groups), _ptr(d_total_groups), _ptr(d_num_joined))
    r._keep = (d_row_ids, d_num_rows, d_sum, d_keys, d_ivals, d_fvals, d_num_groups, d_total_groups, d_num_joined)
    return r


def tqp_run_plan(ctx: Context, plan: Plan, result: Result, stream=None):
    _check(lib().tqp_run_plan(ctx.h, C.byref(plan), C.byref(result), _stream(stream)))


def tqp_run_plans(ctx: Context, plans, results, stream=None):
    n = len(plans)
    pa = (Plan * n)(*plans)
    ra = (Result * n)(*results)
    _check(lib().tqp_run_plans(ctx.h, pa, ra, n, _stream(stream)))


class Batch:
    """A lowered, graph-captured batch of plans (tqp_batch_create).

    Holds the plans, results and context alive until ``tqp_batch_destroy``;
    the device buffers they point to are re-read on every run."""

    def __init__(self, ctx: Context, plans, results):
        n = len(plans)
        if n != len(results):
            raise ValueError("one result per plan")
        pa = (Plan * n)(*plans)
        ra = (Result * n)(*results)
        h = C.c_void_p()
        _check(lib().tqp_batch_create(ctx.h, pa, ra, n, C.byref(h)))
        self.h = h
        self.ctx = ctx
        self._keep = (list(plans), list(results))

    def close(self):
        if getattr(self, "h", None):
            lib().tqp_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tqp_batch_create(ctx: Context, plans, results) -> Batch:
    return Batch(ctx, plans, results)


def tqp_batch_run(batch: Batch, stream=None):
    if not batch.h:
        raise ValueError("batch was destroyed")
    _check(lib().tqp_batch_run(batch.h, _stream(stream)))


def tqp_batch_destroy(batch: Batch):
    batch.close()


class PreparedDim:
    """A dimension table prepared once for many joined plans (tqp_dim_prepare)."""

    def __init__(self, ctx: Context, dim: TableRef, key_col: int, group_cols=(), max_groups: int = 0, stream=None):
        gc = (C.c_int32 * max(1, len(group_cols)))(*[int(c) for c in group_cols])
        h = C.c_void_p()
        _check(lib().tqp_dim_prepare(ctx.h, C.byref(dim.t), int(key_col), gc, len(group_cols), int(max_groups),
                                     _stream(stream), C.byref(h)))
        self.h = h
        self.ctx = ctx
        self.dim = dim

    @property
    def groups(self) -> int:
        return int(lib().tqp_dim_groups(self.h))

    def close(self):
        if getattr(self, "h", None):
            lib().tqp_dim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tqp_dim_prepare(ctx: Context, dim: TableRef, key_col: int, group_cols=(), max_groups: int = 0,
                    stream=None) -> PreparedDim:
    return PreparedDim(ctx, dim, key_col, group_cols, max_groups, stream)


def tqp_dim_destroy(d: PreparedDim):
    d.close()


class ServerConfig(C.Structure):
    _fields_ = [("max_batch", C.c_int32), ("max_inflight", C.c_int32), ("budget_bytes", C.c_int64)]


class Completion(C.Structure):
    _fields_ = [("tag", C.c_uint64), ("status", C.c_int32), ("batch_size", C.c_int32), ("queue_s", C.c_double),
                ("latency_s", C.c_double)]


class Server:
    """Continuous batching of submitted plans (tqp_server_*).

    The caller keeps each submitted plan's tables and result buffers alive until
    its completion is polled."""

    def __init__(self, ctx: Context, max_batch: int = 64, max_inflight: int = 2, budget_bytes: int = 1 << 30):
        cfg = ServerConfig(int(max_batch), int(max_inflight), int(budget_bytes))
        h = C.c_void_p()
        _check(lib().tqp_server_create(ctx.h, C.byref(cfg), C.byref(h)))
        self.h = h
        self.ctx = ctx
        self._buf = (Completion * 4096)()

    def submit(self, plan: Plan, result: Result, tag: int):
        _check(lib().tqp_server_submit(self.h, C.byref(plan), C.byref(result), int(tag)))

    def poll(self):
        """Finished requests since the last poll: list of (tag, status, batch_size, queue_s, latency_s)."""
        out = []
        while True:
            k = lib().tqp_server_poll(self.h, self._buf, len(self._buf))
            out.extend((c.tag, c.status, c.batch_size, c.queue_s, c.latency_s) for c in self._buf[:k])
            if k < len(self._buf):
                return out

    def drain(self, timeout_s: float = 60.0):
        _check(lib().tqp_server_drain(self.h, float(timeout_s)))

    def close(self):
        if getattr(self, "h", None):
            lib().tqp_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tqp_server_create(ctx: Context, max_batch: int = 64, max_inflight: int = 2, budget_bytes: int = 1 << 30) -> Server:
    return Server(ctx, max_batch, max_inflight, budget_bytes)


def tqp_server_submit(server: Server, plan: Plan, result: Result, tag: int):
    server.submit(plan, result, tag)


def tqp_server_poll(server: Server):
    return server.poll()


def tqp_server_drain(server: Server, timeout_s: float = 60.0):
    server.drain(timeout_s)


def tqp_server_destroy(server: Server):
    server.close()


def tqp_measure_l2_red(device: int, d_table, rows: int, adds_per_row: int = 2, blocks_per_sm: int = 2,
                       threads: int = 256, stream=None):
    """Random 8-byte L2 reductions into d_table (an int64 CUDA tensor): the joined aggregation's roofline."""
    _check(lib().tqp_measure_l2_red(int(device), _ptr(d_table), d_table.numel(), int(rows), int(adds_per_row),
                                    int(blocks_per_sm), int(threads), _stream(stream)))


def tqp_measure_scan_rate(ctx: Context, table: TableRef, tile_rows: int, stages: int, ctas_per_sm: int, d_out,
                          stream=None):
    """The staged scan engine over every column of `table` with a body that only reads the stages: the
    ceiling of the scans on those columns at that launch shape (see include/tqp.h)."""
    _check(lib().tqp_measure_scan_rate(ctx.h, table.ref(), int(tile_rows), int(stages), int(ctas_per_sm),
                                       _ptr(d_out), _stream(stream)))
