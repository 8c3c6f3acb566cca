"""GPU parity: tqp_filter (predicates + stream compaction + projection-sum)
against the CPU oracle, element by element (bit-exact: integer work)."""
import numpy as np
import pytest

import datagen
import oracle

pytestmark = pytest.mark.gpu

Q6_PREDS = [(0, "ge", 731), (0, "lt", 1096), (1, "between", 5, 7), (2, "lt", 24)]
Q6_EXPR = [("col", 3), ("col", 1), "mul"]


@pytest.fixture(scope="module")
def ctx():
    import paper_2203_01877_gb300 as tqp
    c = tqp.Context(0, 256 << 20)
    yield c
    c.close()


def q6_cols(n, seed):
    t = datagen.fact_table(n, seed=seed)
    return [t["date"], t["discount"], t["quantity"], t["price"]]


def check(ctx, cols, preds, expr, **kw):
    from tests.gpu_util import gpu_filter
    ids, k, s, st = gpu_filter(ctx, cols, preds, expr, **kw)
    want_ids, want_sum = oracle.filter_rows(cols, preds, expr)
    assert st == 0
    assert k == len(want_ids)
    assert np.array_equal(ids, want_ids)
    if expr is not None:
        assert s == want_sum
    return k


@pytest.mark.parametrize("n", [1, 15, 16, 17, 1000, 1023, 1024, 1025, 4096, 4111, 70001, 1_000_003])
def test_q6_shape_sizes(ctx, n):
    check(ctx, q6_cols(n, 100 + n), Q6_PREDS, Q6_EXPR)


def test_empty_table(ctx):
    from tests.gpu_util import gpu_filter
    cols = [np.zeros(0, np.int32), np.zeros(0, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int64)]
    ids, k, s, st = gpu_filter(ctx, cols, Q6_PREDS, Q6_EXPR)
    assert st == 0 and k == 0 and s == 0


def test_all_pass_and_none_pass(ctx):
    cols = q6_cols(300_001, 5)
    assert check(ctx, cols, [(0, "ge", 0)], Q6_EXPR) == 300_001
    assert check(ctx, cols, [(0, "lt", 0)], Q6_EXPR) == 0
    assert check(ctx, cols, [], Q6_EXPR) == 300_001          # no predicate: every row, summed columns staged
    assert check(ctx, cols, [(0, "gt", 5), (0, "lt", 3)], None) == 0  # contradictory range


@pytest.mark.parametrize("op", ["lt", "le", "gt", "ge", "eq", "ne", "between"])
@pytest.mark.parametrize("dtype", [np.int32, np.int64, np.uint8])
def test_each_operator_and_dtype(ctx, op, dtype):
    rng = np.random.default_rng(3)
    n = 50_017
    info = np.iinfo(dtype)
    x = rng.integers(max(info.min, -100), min(info.max, 100) + 1, size=n).astype(dtype)
    y = rng.integers(-1000, 1000, size=n).astype(np.int64)
    check(ctx, [x, y], [(0, op, 10, 60)], [("col", 1), ("col", 0), "sub"])


def test_extreme_values(ctx):
    i32 = np.iinfo(np.int32)
    x = np.array([i32.min, -1, 0, 1, i32.max] * 1000, np.int32)
    check(ctx, [x], [(0, "ge", i32.min)], None)
    check(ctx, [x], [(0, "le", i32.max), (0, "ne", 0)], None)
    check(ctx, [x], [(0, "gt", i32.max)], None)
    i64 = np.iinfo(np.int64)
    z = np.array([i64.min, -5, 0, 5, i64.max] * 999, np.int64)
    check(ctx, [z], [(0, "lt", i64.min)], None)
    check(ctx, [z], [(0, "gt", i64.max)], None)
    check(ctx, [z], [(0, "between", i64.min, i64.max)], None)
    check(ctx, [z], [(0, "ne", i64.max), (0, "ne", i64.min)], None)


def test_multi_expression_forms(ctx):
    cols = q6_cols(123_457, 8)
    for ex in ([("col", 3)],
               [("col", 3), ("const", 100), ("col", 1), "sub", "mul"],
               [("const", 3), ("col", 2), ("col", 0), "add", "mul", ("col", 1), "sub"],
               [("col", 0), ("col", 1), ("col", 2), ("col", 3), "add", "add", "add"]):
        check(ctx, cols, Q6_PREDS, ex)


def test_count_only_and_capacity(ctx):
    import paper_2203_01877_gb300 as tqp
    from tests.gpu_util import gpu_filter
    cols = q6_cols(400_000, 9)
    want_ids, want_sum = oracle.filter_rows(cols, Q6_PREDS, Q6_EXPR)
    ids, k, s, st = gpu_filter(ctx, cols, Q6_PREDS, Q6_EXPR, want_ids=False)
    assert st == 0 and k == len(want_ids) and s == want_sum
    cap = len(want_ids) // 2
    ids, k, s, st = gpu_filter(ctx, cols, Q6_PREDS, Q6_EXPR, capacity=cap)
    assert st == tqp.ERR_CAPACITY
    assert k == len(want_ids) and s == want_sum
    assert np.array_equal(ids, want_ids[:cap])
    # the context is usable again after the check cleared the latch
    check(ctx, cols, Q6_PREDS, Q6_EXPR)


def test_deterministic_repeat(ctx):
    from tests.gpu_util import gpu_filter
    cols = q6_cols(2_000_000, 21)
    a = gpu_filter(ctx, cols, Q6_PREDS, Q6_EXPR)
    b = gpu_filter(ctx, cols, Q6_PREDS, Q6_EXPR)
    assert np.array_equal(a[0], b[0]) and a[1:] == b[1:]


def test_invalid_arguments_rejected(ctx):
    import torch
    import paper_2203_01877_gb300 as tqp
    from tests.gpu_util import up
    x = up(np.arange(100, dtype=np.int32))
    t = tqp.TableRef([x])
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda:0")
    with pytest.raises(tqp.TqpError) as e:
        tqp.tqp_filter(ctx, t, [(3, "lt", 1)], d_count=cnt)
    assert e.value.status == tqp.ERR_INVALID_ARG
    with pytest.raises(tqp.TqpError):
        tqp.tqp_filter(ctx, t, [(0, "lt", 1)], d_count=None)
    mis = torch.zeros(101, dtype=torch.int32, device="cuda:0")[1:]  # 4-byte offset: not 16-byte aligned
    with pytest.raises(tqp.TqpError) as e:
        tqp.tqp_filter(ctx, tqp.TableRef([mis]), [(0, "lt", 1)], d_count=cnt)
    assert e.value.status == tqp.ERR_INVALID_ARG


def test_full_size_filter_project_reduce(ctx):
    """60M rows, the benchmark's launch configuration, compared in full."""
    import paper_2203_01877_gb300 as tqp
    n = 60_000_000
    cols = q6_cols(n, datagen.DEFAULT_SEED + 1)
    big = tqp.Context(0, 64 << 20)
    try:
        k = check(big, cols, Q6_PREDS, Q6_EXPR)
    finally:
        big.close()
    assert 1_000_000 < k < 1_150_000


def test_filter_host_projected_column(ctx):
    """A projected column in pinned host memory (read in place at passing rows
    only) gives the same row ids, count and sum as the device-resident table."""
    import torch
    import paper_2203_01877_gb300 as tqp
    t = datagen.fact_table(2_000_003, seed=31, cols=["date", "discount", "quantity", "price"])
    dev = [torch.from_numpy(t[c]).cuda() for c in ("date", "discount", "quantity", "price")]
    preds = [(0, "ge", 731), (0, "lt", 1096), (1, "between", 5, 7), (2, "lt", 24)]
    expr = [("col", 3), ("col", 1), "mul"]
    outs = []
    for host_price in (False, True):
        cols = list(dev)
        if host_price:
            cols[3] = torch.from_numpy(t["price"]).pin_memory()
        T = tqp.TableRef(cols, host_ok=True)
        ids = torch.full((len(t["date"]),), -1, dtype=torch.int32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        s = torch.zeros(1, dtype=torch.int64, device="cuda")
        tqp.tqp_filter(ctx, T, preds, expr, s, ids, len(t["date"]), cnt)
        assert ctx.status() == 0
        k = int(cnt.item())
        outs.append((k, int(s.item()), ids[:k].cpu()))
    assert outs[0][0] == outs[1][0] and outs[0][1] == outs[1][1] and torch.equal(outs[0][2], outs[1][2])


def test_filter_host_staged_column_rejected(ctx):
    """Host memory where the scan stages the column (a predicate column, or any
    column of another operator) is refused on the host, before any launch."""
    import torch
    import paper_2203_01877_gb300 as tqp
    t = datagen.fact_table(10_000, seed=32, cols=["date", "price"])
    hd = torch.from_numpy(t["date"]).pin_memory()
    dp = torch.from_numpy(t["price"]).cuda()
    T = tqp.TableRef([hd, dp], host_ok=True)
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(tqp.TqpError) as e:
        tqp.tqp_filter(ctx, T, [(0, "lt", 100)], None, None, None, 0, cnt)
    assert e.value.status == tqp.ERR_INVALID_ARG
    keys = torch.zeros(64, dtype=torch.int64, device="cuda")
    iv = torch.zeros(64, dtype=torch.int64, device="cuda")
    ng = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(tqp.TqpError) as e:
        tqp.tqp_groupby_agg(ctx, T, [], [0], [("count", None)], keys, iv, None, 64, ng)
    assert e.value.status == tqp.ERR_INVALID_ARG


def test_filter_pageable_projected_column_rejected(ctx):
    """A projected column in pageable host memory (a raw pointer the GPU
    cannot address, passed straight through the C ABI) is refused before any
    launch, by tqp_filter and by tqp_filter_noalloc; the same call with the
    column pinned runs."""
    import torch
    import paper_2203_01877_gb300 as tqp
    n = 100_000
    t = datagen.fact_table(n, seed=33, cols=["date", "price"])
    d_date = torch.from_numpy(t["date"]).cuda()
    pinned = torch.from_numpy(t["price"]).pin_memory()
    raw = np.empty(n + 2, np.int64)  # pageable; pick a 16-byte aligned start
    off = (-raw.ctypes.data % 16) // 8
    pageable = raw[off:off + n]
    pageable[:] = t["price"]
    T = tqp.TableRef([d_date, pinned], host_ok=True)
    T.carr[1].data = pageable.ctypes.data
    cnt = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    s = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    expr = [("col", 1)]
    with pytest.raises(tqp.TqpError) as e:
        tqp.tqp_filter(ctx, T, [(0, "lt", 100)], expr, s, None, 0, cnt)
    assert e.value.status == tqp.ERR_INVALID_ARG and "page-locked" in str(e.value)
    with pytest.raises(tqp.TqpError) as e:
        tqp.tqp_filter_noalloc(0, T, [(0, "lt", 100)], expr, s, None, 0, cnt)
    assert e.value.status == tqp.ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert int(cnt.item()) == -7 and int(s.item()) == -7  # nothing ran
    T.carr[1].data = pinned.data_ptr()
    tqp.tqp_filter(ctx, T, [(0, "lt", 100)], expr, s, None, 0, cnt)
    assert ctx.status() == 0
    want_ids, want_sum = oracle.filter_rows([t["date"], t["price"]], [(0, "lt", 100)], expr)
    assert int(cnt.item()) == len(want_ids) and int(s.item()) == want_sum


@pytest.mark.parametrize("extra", [1, 3])
@pytest.mark.parametrize("shape", [(1024, 2, 1), (1024, 3, 2), (2048, 2, 1)])
def test_ragged_last_tile_under_forced_shapes(ctx, extra, shape):
    """A last tile of one to three rows stages no bytes (its staged columns are read row by row), while its
    pipeline stage was already used earlier in the same chunk: the scan must neither stall nor report a wait
    that ran out, and must give the oracle's result."""
    from tests.gpu_util import gpu_filter
    n = shape[0] * 600 + extra
    cols = q6_cols(n, 4000 + extra)
    try:
        ctx.set_tuning(*shape)
        ids, k, s, st = gpu_filter(ctx, cols, Q6_PREDS, Q6_EXPR)
    finally:
        ctx.set_tuning(0, 0, 0)
    want_ids, want_sum = oracle.filter_rows(cols, Q6_PREDS, Q6_EXPR)
    assert st == 0 and k == len(want_ids) and s == want_sum
    assert np.array_equal(ids, want_ids)


@pytest.mark.parametrize("n", [1, 3, 128, 1023, 4099, 1_000_003])
@pytest.mark.parametrize("case", ["q6", "u8_i64", "six_conditions", "ne_and_extremes"])
def test_direct_filter_variant(ctx, n, case):
    """The direct form of the filter (variant 1: predicate columns read with plain vector loads, no staging)
    gives the oracle's row ids, count and sum; with more than four conditions it falls back to the staged
    scan."""
    from tests.gpu_util import gpu_filter
    rng = np.random.default_rng(n + len(case))
    if case == "q6":
        cols, preds, expr = q6_cols(n, 77), Q6_PREDS, Q6_EXPR
    elif case == "u8_i64":
        t = datagen.fact_table(n, seed=78)
        cols = [t["flag"], t["price"], t["status"]]
        preds, expr = [(0, "eq", 1), (1, "ge", 5_000_000), (2, "ne", 0)], [("col", 1)]
    elif case == "six_conditions":  # three ranges, a fourth column and two NE tests: six conditions
        cols = q6_cols(n, 79)
        preds, expr = Q6_PREDS + [(3, "gt", 1000), (1, "ne", 6), (2, "ne", 10)], Q6_EXPR
    else:
        x = rng.integers(np.iinfo(np.int64).min, np.iinfo(np.int64).max, n, dtype=np.int64)
        x[::7] = np.iinfo(np.int64).max
        y = rng.integers(-2**31, 2**31 - 1, n).astype(np.int32)
        cols, preds, expr = [x, y], [(0, "ne", np.iinfo(np.int64).max), (1, "le", 0)], [("col", 1)]
    try:
        ctx.set_variant(1)
        ids, k, s, st = gpu_filter(ctx, cols, preds, expr)
    finally:
        ctx.set_variant(-1)
    want_ids, want_sum = oracle.filter_rows(cols, preds, expr)
    assert st == 0 and k == len(want_ids) and s == want_sum
    assert np.array_equal(ids, want_ids)
