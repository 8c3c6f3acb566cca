"""Shared scans (tqp_filter_shared): many filter queries in one pass over a
table, each compared with the oracle's filter of that query alone (count of
passing rows and SUM of its expression, exact)."""
import numpy as np
import pytest

import datagen
import oracle

pytestmark = pytest.mark.gpu

FCOLS = ["date", "discount", "quantity", "price", "flag", "status", "key"]
I64_MIN, I64_MAX = -(1 << 63), (1 << 63) - 1
REVENUE = [("col", 3), ("col", 1), "mul"]                               # price * discount
NET = [("col", 3), ("const", 100), ("col", 1), "sub", "mul"]            # price * (100 - discount)


def _table(n, seed):
    t = datagen.fact_table(n, seed=seed)
    return [t[c] for c in FCOLS]


def q6_queries(k, seed, expr=REVENUE):
    """k queries shaped like the paper's filter query: a 365-day window, a
    discount band of three values, a quantity cutoff (seeded)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(k):
        d0 = int(rng.integers(0, 2557 - 365))
        disc = int(rng.integers(1, 9))
        qty = int(rng.integers(2, 51))
        out.append(([(0, "ge", d0), (0, "lt", d0 + 365), (1, "between", disc - 1, disc + 1), (2, "lt", qty)], expr))
    return out


def run_shared(ctx, cols, queries):
    import torch
    import paper_2203_01877_gb300 as tqp
    from tests.gpu_util import up
    T = tqp.TableRef([up(c) for c in cols])
    outs = []
    for preds, ex in queries:
        cnt = torch.full((1,), -7, dtype=torch.int64, device="cuda")
        s = torch.full((1,), -7, dtype=torch.int64, device="cuda") if ex is not None else None
        outs.append((preds, ex, cnt, s))
    launch_of = tqp.tqp_filter_shared(ctx, T, outs)
    assert ctx.status() == 0
    got = [(int(c.item()), None if s is None else int(s.item())) for _, _, c, s in outs]
    return got, launch_of


def check(cols, queries, got):
    for i, (preds, ex) in enumerate(queries):
        ids, want_sum = oracle.filter_rows(cols, preds, ex)
        assert got[i][0] == len(ids), (i, preds)
        if ex is not None:
            assert got[i][1] == want_sum, (i, preds, ex)


@pytest.fixture(scope="module")
def ctx():
    import paper_2203_01877_gb300 as tqp
    c = tqp.Context(0, 256 << 20)
    yield c
    c.close()


def test_32_q6_queries_one_launch(ctx):
    cols = _table(3_000_017, 101)
    qs = q6_queries(32, 7)
    got, launch_of = run_shared(ctx, cols, qs)
    assert launch_of == [0] * 32
    check(cols, qs, got)


def test_more_than_32_queries_split(ctx):
    cols = _table(1_000_003, 102)
    qs = q6_queries(40, 8)
    got, launch_of = run_shared(ctx, cols, qs)
    assert launch_of == [0] * 32 + [1] * 8
    check(cols, qs, got)


def test_expressions_counts_and_packing(ctx):
    """Two distinct expressions per launch; a third starts another launch;
    count-only queries join any launch; an expression without the closed
    product form runs alone, and so do the queries of a launch of fewer than
    three."""
    cols = _table(777_777, 103)
    sq = [("col", 3), ("col", 1), "add", ("col", 2), ("col", 0), "add", "mul"]  # (price+discount)*(qty+date)
    base = q6_queries(9, 9)
    qty = [("col", 2)]
    qs = [base[0], (base[1][0], NET), (base[2][0], qty), (base[3][0], None), (base[4][0], sq),
          (base[5][0], REVENUE), ([], [("col", 6), ("const", 3), "mul"]), ([], None), (base[6][0], qty),
          (base[7][0], [("col", 5), ("col", 6), "mul"])]
    got, launch_of = run_shared(ctx, cols, qs)
    assert launch_of[0] == launch_of[1] == launch_of[3] == launch_of[5] == launch_of[7] == 0
    assert launch_of[2] == launch_of[6] == launch_of[8] == 1
    assert launch_of[4] == -1 and launch_of[9] == -1  # not closed; a launch of one
    check(cols, qs, got)


@pytest.mark.parametrize("n", [0, 1, 100, 1023, 1024, 9_000 + 37, 262_144 + 5])
def test_ragged_and_empty_tables(ctx, n):
    cols = _table(n, 104)
    qs = q6_queries(12, 10) + [([(4, "eq", 1)], REVENUE), ([(5, "ne", 0), (6, "lt", 5000)], [("col", 2)])]
    got, _ = run_shared(ctx, cols, qs)
    check(cols, qs, got)


def test_searched_tables_wide_ranges_and_edge_values(ctx):
    """Ranges too wide for a direct table (price and key), NE, never-true and
    always-true conditions, int64 extremes, and queries with no predicate."""
    cols = _table(2_000_003, 105)
    rng = np.random.default_rng(11)
    qs = []
    for _ in range(20):
        a, b = sorted(int(x) for x in rng.integers(100, 10_000_000, 2))
        qs.append(([(3, "between", a, b), (6, "ge", int(rng.integers(0, 90_000)))], REVENUE))
    qs += [
        ([(3, "lt", I64_MIN)], REVENUE),               # never true
        ([(3, "ge", I64_MIN), (3, "le", I64_MAX)], REVENUE),  # always true
        ([(1, "ne", 5), (1, "ne", 6), (4, "ne", 2)], NET),
        ([(0, "gt", I64_MAX)], None),                  # never true
        ([(0, "le", -5)], None),                       # below every date
        ([(2, "eq", 50), (0, "eq", 2556)], REVENUE),
        ([], REVENUE),
        ([(3, "between", 5_000_000, 4_000_000)], None),  # empty range
    ]
    got, launch_of = run_shared(ctx, cols, qs)
    assert set(launch_of) == {0}
    check(cols, qs, got)


def test_column_union_over_eight_splits(ctx):
    """A query set reading ten distinct columns needs two launches (eight
    staged columns each)."""
    n = 500_009
    base = _table(n, 106)
    rng = np.random.default_rng(12)
    extra = [rng.integers(0, 1000, n).astype(np.int32) for _ in range(3)]
    cols = base + extra  # columns 7, 8, 9
    qs = [([(c, "lt", 500)], [("col", 3)]) for c in (7, 8, 9)]
    qs += [([(0, "lt", 1000), (2, "lt", 25)], REVENUE), ([(4, "eq", 0), (5, "eq", 1)], [("col", 6)])]
    qs += [([(4, "eq", 2), (5, "eq", 0)], [("col", 6)]), ([(4, "ne", 1)], [("col", 6)])]
    got, launch_of = run_shared(ctx, cols, qs)
    assert launch_of[:4] == [0] * 4 and launch_of[4:] == [1] * 3
    check(cols, qs, got)


def test_same_results_as_single_query_filter(ctx):
    """Identical outputs to tqp_filter on every query (same table, same context)."""
    import torch
    import paper_2203_01877_gb300 as tqp
    from tests.gpu_util import up
    cols = _table(1_500_001, 107)
    qs = q6_queries(16, 13, NET)
    got, _ = run_shared(ctx, cols, qs)
    T = tqp.TableRef([up(c) for c in cols])
    for i, (preds, ex) in enumerate(qs):
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        s = torch.zeros(1, dtype=torch.int64, device="cuda")
        tqp.tqp_filter(ctx, T, preds, ex, s, None, 0, cnt)
        assert (int(cnt.item()), int(s.item())) == got[i]


def test_numeric_in_lists_share_the_scan(ctx):
    """IN lists on numeric columns (dense, sparse, empty, duplicated, outside
    the column type's range, int64 extremes) pack with range queries (two sum
    expressions: one launch)."""
    cols = _table(1_200_007, 109)
    rng = np.random.default_rng(14)
    qs = []
    for k in range(12):
        d0 = int(rng.integers(0, 2000))
        disc = sorted(int(x) for x in rng.choice(11, 3, replace=False))
        qty = [int(x) for x in rng.integers(1, 51, 6)]
        qs.append(([(0, "ge", d0), (0, "lt", d0 + 365), (1, "in", disc), (2, "in", qty)], REVENUE))
    qs += [
        ([(6, "in", [int(x) for x in rng.integers(0, 100_000, 200)])], REVENUE),   # sparse: a searched table
        ([(2, "in", list(range(10, 30)) + [12, 12, 29])], None),                   # dense, with repeats
        ([(1, "in", [])], REVENUE),                                               # never true
        ([(2, "in", [-(1 << 40), 1 << 40, 7])], [("col", 2)]),                     # outside int32, and 7
        ([(3, "in", [I64_MIN, I64_MAX, int(cols[3][5]), int(cols[3][99])])], REVENUE),
        ([(4, "in", [0, 2]), (5, "ne", 1), (0, "in", [0, 1, 2556])], None),
    ]
    got, launch_of = run_shared(ctx, cols, qs)
    assert set(launch_of) == {0}
    check(cols, qs, got)


def test_invalid_arguments_launch_nothing(ctx):
    import torch
    import paper_2203_01877_gb300 as tqp
    from tests.gpu_util import up
    cols = _table(10_000, 108)
    T = tqp.TableRef([up(c) for c in cols])
    cnt = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    s = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    for bad in ([([(99, "lt", 3)], REVENUE, cnt, s)],               # column out of range
                [([(0, "lt", 3)], REVENUE, None, s)],               # no count
                [([(0, "lt", 3)], REVENUE, cnt, None)],             # sum without output
                [([(0, "lt", 3)], None, cnt, s)],                   # output without sum
                [([(0, "lt", 3)], [("col", 42)], cnt, s)]):         # expression column out of range
        with pytest.raises(tqp.TqpError) as e:
            tqp.tqp_filter_shared(ctx, T, [([(0, "lt", 5)], None, cnt, None)] + bad)
        assert e.value.status == tqp.ERR_INVALID_ARG
    # a bad query after shareable ones: found before the shared launch
    ok = [([(0, "lt", 100 * k)], REVENUE, cnt, s) for k in range(1, 5)]
    for bad, status in (([(1, "like", "1%")], tqp.ERR_INVALID_ARG),            # LIKE on a number
                        ([(2, "in", list(range(4000)))], tqp.ERR_UNSUPPORTED)):  # more than the set budget
        with pytest.raises(tqp.TqpError) as e:
            tqp.tqp_filter_shared(ctx, T, ok + [(bad, None, cnt, None)])
        assert e.value.status == status, bad
    torch.cuda.synchronize()
    assert int(cnt.item()) == -7 and int(s.item()) == -7
