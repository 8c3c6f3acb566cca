"""Pins for the oracle's filter and expression evaluation (CPU only).

The filter is the selection-vector form of Section 3.1 (Listing 1 uses a
comparison mask then ``masked_select``; the selection-vector variant uses
``nonzero``): rows whose predicates all hold, in ascending row order.  The
oracle is checked against numpy's boolean-mask + ``flatnonzero`` (a library
special case of the same definition), against hand-worked values, and against
statistical closed forms of the generated workloads.
"""
import math

import numpy as np
import pytest

import datagen
import oracle

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

NP_OPS = {
    "lt": lambda x, lo, hi: x < lo,
    "le": lambda x, lo, hi: x <= lo,
    "gt": lambda x, lo, hi: x > lo,
    "ge": lambda x, lo, hi: x >= lo,
    "eq": lambda x, lo, hi: x == lo,
    "ne": lambda x, lo, hi: x != lo,
    "between": lambda x, lo, hi: (x >= lo) & (x <= hi),
}


def np_mask(cols, preds):
    m = np.ones(len(cols[0]), dtype=bool)
    for c, op, lo, *hi in preds:
        m &= NP_OPS[op](cols[c].astype(np.int64), lo, hi[0] if hi else 0)
    return m


def test_hand_worked_example():
    # quantity < 24 on six rows (the running example of Section 3.1):
    # quantity = [30, 5, 24, 23, 50, 1] -> rows 1, 3, 5 pass; price*discount
    # summed over them = 100*1 + 300*3 + 500*5 = 3500.
    qty = np.array([30, 5, 24, 23, 50, 1], np.int32)
    price = np.array([0, 100, 0, 300, 0, 500], np.int64)
    disc = np.array([9, 1, 9, 3, 9, 5], np.int64)
    ids, s = oracle.filter_rows([qty, price, disc], [(0, "lt", 24)], [("col", 1), ("col", 2), "mul"])
    assert ids.tolist() == [1, 3, 5]
    assert s == 3500


@pytest.mark.parametrize("op", list(NP_OPS))
@pytest.mark.parametrize("dtype", [np.int32, np.int64, np.uint8])
def test_each_operator_at_boundaries(op, dtype):
    rng = np.random.default_rng(7)
    info = np.iinfo(dtype)
    x = rng.integers(max(info.min, -50), min(info.max, 50) + 1, size=1000).astype(dtype)
    lo, hi = (10, 20) if dtype != np.uint8 else (10, 20)
    # plant exact boundary values so off-by-one mistakes change the result
    x[:6] = np.array([lo - 1, lo, lo + 1, hi - 1, hi, hi + 1]).astype(dtype)
    preds = [(0, op, lo, hi)]
    ids, _ = oracle.filter_rows([x], preds)
    assert np.array_equal(ids, np.flatnonzero(np_mask([x], preds)))


def test_conjunction_and_sum_vs_numpy():
    t = datagen.fact_table(20000, seed=11)
    cols = [t["date"], t["discount"], t["quantity"], t["price"]]
    preds = [(0, "ge", 731), (0, "lt", 1096), (1, "between", 5, 7), (2, "lt", 24)]
    ids, s = oracle.filter_rows(cols, preds, [("col", 3), ("col", 1), "mul"])
    m = np_mask(cols, preds)
    assert np.array_equal(ids, np.flatnonzero(m))
    assert s == int((t["price"] * t["discount"])[m].sum())


def test_expression_operand_order_and_ops():
    a = np.array([7, -3, 100, 0], np.int64)
    b = np.array([2, 5, -4, 9], np.int32)
    fact = [a, b]
    for toks, ref in [
        ([("col", 0), ("col", 1), "sub"], a - b),
        ([("col", 1), ("col", 0), "sub"], b - a),
        ([("const", 100), ("col", 1), "sub", ("col", 0), "mul"], (100 - b) * a),
        ([("col", 0), ("const", 3), "add", ("col", 1), "mul"], (a + 3) * b),
    ]:
        _, s = oracle.filter_rows(fact, [], toks)
        assert s == int(ref.sum())


def test_sum_is_additive_over_row_splits():
    t = datagen.fact_table(5000, seed=3)
    cols = [t["quantity"], t["price"], t["discount"]]
    preds = [(0, "lt", 24)]
    ex = [("col", 1), ("const", 100), ("col", 2), "sub", "mul"]
    _, whole = oracle.filter_rows(cols, preds, ex)
    parts = 0
    for lo, hi in [(0, 1), (1, 1777), (1777, 4096), (4096, 5000)]:
        _, s = oracle.filter_rows([c[lo:hi] for c in cols], preds, ex)
        parts += s
    assert parts == whole


def test_edge_cases():
    e = np.zeros(0, np.int32)
    ids, s = oracle.filter_rows([e], [(0, "lt", 5)], [("col", 0)])
    assert len(ids) == 0 and s == 0
    x = np.array([np.iinfo(np.int32).min, -1, 0, np.iinfo(np.int32).max], np.int32)
    assert oracle.filter_rows([x], [(0, "ge", np.iinfo(np.int32).min)])[0].tolist() == [0, 1, 2, 3]
    assert oracle.filter_rows([x], [(0, "gt", np.iinfo(np.int32).max)])[0].tolist() == []
    assert oracle.filter_rows([x], [(0, "lt", 0)])[0].tolist() == [0, 1]
    u = np.array([0, 255, 128], np.uint8)  # unsigned widening, not sign extension
    assert oracle.filter_rows([u], [(0, "gt", 127)])[0].tolist() == [1, 2]


def test_overflow_is_reported():
    big = np.array([np.iinfo(np.int64).max, 1], np.int64)
    with pytest.raises(oracle.OracleError) as ei:
        oracle.filter_rows([big], [], [("col", 0)])
    assert ei.value.status == oracle.ERR_OVERFLOW
    with pytest.raises(oracle.OracleError):
        oracle.filter_rows([big], [], [("col", 0), ("const", 2), "mul"])


def test_selectivity_matches_closed_form():
    # 731 <= date < 1096, 5 <= discount <= 7, quantity < 24 over independent
    # uniform columns: p = (365/2557) * (3/11) * (23/50).
    n = 400_000
    t = datagen.fact_table(n, seed=datagen.DEFAULT_SEED + 1)
    cols = [t["date"], t["discount"], t["quantity"]]
    preds = [(0, "ge", 731), (0, "lt", 1096), (1, "between", 5, 7), (2, "lt", 24)]
    ids, _ = oracle.filter_rows(cols, preds)
    p = (365 / 2557) * (3 / 11) * (23 / 50)
    assert abs(len(ids) - n * p) < 5 * math.sqrt(n * p * (1 - p))
    # date <= 2450 passes 2451/2557 of rows
    ids2, _ = oracle.filter_rows([t["date"]], [(0, "le", 2450)])
    p2 = 2451 / 2557
    assert abs(len(ids2) - n * p2) < 5 * math.sqrt(n * p2 * (1 - p2))


def test_invalid_plans_rejected():
    x = np.arange(4, dtype=np.int32)
    with pytest.raises(oracle.OracleError):
        oracle.filter_rows([x], [(3, "lt", 1)])
    with pytest.raises(oracle.OracleError):
        oracle.filter_rows([x], [], [("col", 5)])
    with pytest.raises(oracle.OracleError):
        oracle.filter_rows([x], [], [("col", 0), "add"])


@pytest.mark.parametrize("n,threads", [(0, 4), (1, 8), (7, 16), (1000, 3), (250_001, 16), (250_001, 1)])
def test_row_range_threads_give_the_single_thread_result(n, threads):
    """The all-core timing variant (row ranges on threads, joined in order) equals one call."""
    t = datagen.fact_table(n, seed=n + threads, cols=["date", "discount", "quantity", "price"])
    cols = [t[c] for c in ("date", "discount", "quantity", "price")]
    preds = [(0, "ge", 731), (0, "lt", 1096), (1, "between", 5, 7), (2, "lt", 24)]
    expr = [("col", 3), ("col", 1), "mul"]
    ids1, s1 = oracle.filter_rows(cols, preds, expr)
    idsn, sn = oracle.filter_rows(cols, preds, expr, threads=threads)
    assert np.array_equal(ids1, idsn) and s1 == sn
    # ranges that each keep every row: ids are 0..n-1 in order
    ids, s = oracle.filter_rows(cols, [], expr, threads=threads)
    assert np.array_equal(ids, np.arange(n)) and s == int((t["price"] * t["discount"]).sum())


def test_row_range_threads_reject_grouped_plans():
    with pytest.raises(ValueError):
        oracle.run_plan([np.zeros(4, np.int32)], group_cols=[0], aggs=[("count", None)], threads=4)
