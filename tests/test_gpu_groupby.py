"""GPU parity: tqp_groupby_agg against the CPU oracle (bit-exact: integer sums,
one IEEE division per AVG compared by bit pattern)."""
import numpy as np
import pytest

import datagen
import oracle

pytestmark = pytest.mark.gpu

Q1_AGGS = [("sum", [("col", 3)]), ("sum", [("col", 4)]),
           ("sum", [("col", 4), ("const", 100), ("col", 5), "sub", "mul"]),
           ("count", None), ("avg", [("col", 4)])]


@pytest.fixture(scope="module")
def ctx():
    import paper_2203_01877_gb300 as tqp
    c = tqp.Context(0, 512 << 20)
    yield c
    c.close()


def q1_cols(n, seed):
    t = datagen.fact_table(n, seed=seed)
    return [t["date"], t["flag"], t["status"], t["quantity"], t["price"], t["discount"]]


def gpu_groupby(ctx, cols, preds, group_cols, aggs, capacity=4096):
    import torch
    import paper_2203_01877_gb300 as tqp
    from tests.gpu_util import up
    table = tqp.TableRef([up(c) for c in cols])
    ngc, na = len(group_cols), len(aggs)
    keys = torch.zeros(max(capacity * ngc, 1), dtype=torch.int64, device="cuda:0")
    iv = torch.zeros(max(capacity * na, 1), dtype=torch.int64, device="cuda:0")
    fv = torch.zeros(max(capacity * na, 1), dtype=torch.float64, device="cuda:0")
    ng = torch.full((1,), -7, dtype=torch.int64, device="cuda:0")
    tqp.tqp_groupby_agg(ctx, table, preds, group_cols, aggs, keys, iv, fv, capacity, ng)
    st = ctx.status()
    G = int(ng.item())
    if G < 0:
        return st, G, None, None, None
    return (st, G, keys[:G * ngc].reshape(G, ngc).cpu().numpy(), iv[:G * na].reshape(G, na).cpu().numpy(),
            fv[:G * na].reshape(G, na).cpu().numpy())


def check(ctx, cols, preds, group_cols, aggs, capacity=4096):
    st, G, k, iv, fv = gpu_groupby(ctx, cols, preds, group_cols, aggs, capacity)
    wk, wiv, wfv = oracle.groupby(cols, preds, group_cols, aggs)
    assert st == 0
    assert G == len(wiv)
    assert np.array_equal(k, wk)
    assert np.array_equal(iv, wiv)
    assert np.array_equal(fv.view(np.int64), wfv.view(np.int64))  # AVG bit patterns (NaN included)
    return G


@pytest.mark.parametrize("n", [1, 100, 1023, 1024, 4097, 100_003, 1_000_000])
def test_q1_shape(ctx, n):
    g = check(ctx, q1_cols(n, 40 + n), [(0, "le", 2450)], [1, 2], Q1_AGGS)
    if n >= 100_000:
        assert g == 6


def test_ungrouped_and_empty(ctx):
    cols = q1_cols(50_000, 3)
    check(ctx, cols, [(0, "le", 2450)], [], Q1_AGGS)
    check(ctx, cols, [(0, "gt", 99999)], [], Q1_AGGS)          # no row passes: one row, COUNT 0, AVG NaN
    check(ctx, cols, [(0, "gt", 99999)], [1, 2], Q1_AGGS)      # no groups at all
    empty = [c[:0] for c in cols]
    check(ctx, empty, [], [1], [("count", None)])


@pytest.mark.parametrize("ngroups", [7, 300, 2000, 50_000])
def test_many_groups_int32_key(ctx, ngroups):
    rng = np.random.default_rng(ngroups)
    n = 400_000
    lo = -(ngroups // 2)
    key = rng.integers(lo, lo + ngroups, n).astype(np.int32)  # exactly `ngroups` distinct keys
    val = rng.integers(-10**9, 10**9, n).astype(np.int64)
    check(ctx, [key, val], [], [0], [("sum", [("col", 1)]), ("count", None), ("avg", [("col", 1)])],
          capacity=ngroups)


def test_int64_and_mixed_keys(ctx):
    rng = np.random.default_rng(5)
    n = 300_000
    a = (rng.integers(-3, 3, n) * (2**28)).astype(np.int32)
    b = rng.integers(0, 256, n).astype(np.uint8)
    c = rng.integers(-100, 100, n).astype(np.int64)
    d = rng.integers(-3, 3, n).astype(np.int64) * (2**40)
    check(ctx, [a, b, c], [(2, "ne", 0)], [0, 1], [("sum", [("col", 2)]), ("count", None)], capacity=2048)
    check(ctx, [b, a, b, c], [], [0, 1, 2], [("count", None)], capacity=2048)        # 48-bit packed key
    check(ctx, [d, c], [(1, "gt", 0)], [0], [("sum", [("col", 1)])], capacity=64)   # one 64-bit key
    import paper_2203_01877_gb300 as tqp
    with pytest.raises(tqp.TqpError) as e:                                          # 72 bits: rejected
        gpu_groupby(ctx, [d, b], [], [0, 1], [("count", None)])
    assert e.value.status == tqp.ERR_UNSUPPORTED
    # a 64-bit key that packs to all ones: int64 max
    z = np.array([np.iinfo(np.int64).max, 0, np.iinfo(np.int64).min, np.iinfo(np.int64).max] * 1000, np.int64)
    check(ctx, [z], [], [0], [("count", None), ("sum", [("col", 0), ("const", 0), "mul"])], capacity=16)


def test_heavy_skew(ctx):
    rng = np.random.default_rng(8)
    n = 500_000
    key = np.where(rng.random(n) < 0.9, 42, rng.integers(0, 5000, n)).astype(np.int32)
    val = rng.integers(0, 1000, n).astype(np.int64)
    check(ctx, [key, val], [], [0], [("sum", [("col", 1)]), ("count", None)], capacity=8192)


def test_capacity_exceeded(ctx):
    import paper_2203_01877_gb300 as tqp
    key = np.arange(10_000, dtype=np.int32)
    st, G, *_ = gpu_groupby(ctx, [key], [], [0], [("count", None)], capacity=100)
    assert st == tqp.ERR_CAPACITY and G == -1
    check(ctx, [key], [], [0], [("count", None)], capacity=10_000)


def test_full_size_q1(ctx):
    """The 1M-row six-group configuration in the benchmark's launch shape."""
    g = check(ctx, q1_cols(1_000_000, datagen.DEFAULT_SEED), [(0, "le", 2450)], [1, 2], Q1_AGGS, capacity=64)
    assert g == 6


# ---- few groups (at most 64): the unstaged vector-load kernel ----------------------


@pytest.mark.parametrize("n", [1, 3, 100, 1023, 1025, 4097, 100_003])
def test_few_groups_q1_ragged(ctx, n):
    """Row counts that leave a ragged last quad of rows and partial warps."""
    g = check(ctx, q1_cols(n, 70 + n), [(0, "le", 2450)], [1, 2], Q1_AGGS, capacity=64)
    if n >= 100_000:
        assert g == 6


@pytest.mark.parametrize("ngroups", [9, 33, 64])
def test_few_groups_list_overflow(ctx, ngroups):
    """More distinct keys per warp step than the warp's key list holds: the
    list is flushed and restarted, and rows that still do not fit go to the
    global table one by one."""
    rng = np.random.default_rng(100 + ngroups)
    n = 300_001
    key = rng.integers(0, ngroups, n).astype(np.int32) * 7 - 100
    flag = rng.integers(0, 3, n).astype(np.uint8)
    val = rng.integers(-10**12, 10**12, n).astype(np.int64)
    check(ctx, [key, flag, val], [(1, "ne", 1)], [0], [("sum", [("col", 2)]), ("count", None),
                                                       ("avg", [("col", 2)])], capacity=64)


def test_few_groups_all_conditions_and_keys(ctx):
    """Four conditions (i64, i32, u8), a three-column packed key (u8, i32, u8)
    and three distinct closed-form sums."""
    t = datagen.fact_table(200_000, seed=77)
    cols = [t["date"], t["flag"], t["status"], t["quantity"], t["price"], t["discount"]]
    preds = [(0, "ge", 100), (3, "lt", 45), (5, "between", 1, 9), (1, "ne", 2)]
    aggs = [("sum", [("col", 4), ("col", 5), "mul"]), ("sum", [("col", 3), ("const", 3), "add"]),
            ("count", None), ("sum", [("const", 50), ("col", 3), "sub"])]
    k = (t["quantity"] % 4).astype(np.int32)
    check(ctx, cols + [k], preds, [1, 6, 2], aggs, capacity=64)


def test_few_groups_ungrouped_and_64bit_key(ctx):
    cols = q1_cols(77_777, 5)
    check(ctx, cols, [(0, "le", 2450)], [], Q1_AGGS, capacity=64)
    check(ctx, cols, [(0, "gt", 99999)], [], Q1_AGGS, capacity=64)   # no row passes: one row, COUNT 0, AVG NaN
    d = (np.arange(77_777) % 5).astype(np.int64) * (2**45) - 2**62
    check(ctx, [d, cols[4]], [], [0], [("sum", [("col", 1)]), ("count", None)], capacity=8)


def test_few_groups_capacity_exceeded(ctx):
    import paper_2203_01877_gb300 as tqp
    key = (np.arange(200_000) % 100).astype(np.int32)
    st, G, *_ = gpu_groupby(ctx, [key], [], [0], [("count", None)], capacity=64)
    assert st == tqp.ERR_CAPACITY and G == -1


@pytest.mark.parametrize("case", ["i32_i32_negative", "i64_negative", "u8_eight", "nine_values", "single_value"])
def test_few_groups_dense_ids(ctx, case):
    """Key columns whose ranges multiply to at most eight slots take mixed-radix
    slot ids (keys rebuilt from the slot index at the flush); nine values do not."""
    rng = np.random.default_rng(hash(case) % 2**32)
    n = 123_457
    val = rng.integers(-10**12, 10**12, n).astype(np.int64)
    if case == "i32_i32_negative":
        a = (rng.integers(0, 2, n) - 2**31).astype(np.int32)
        b = rng.integers(-5, -2, n).astype(np.int32)
        cols, gc = [a, b, val], [0, 1]
    elif case == "i64_negative":
        a = (rng.integers(0, 7, n) - 2**62).astype(np.int64)
        cols, gc = [a, val], [0]
    elif case == "u8_eight":
        a = rng.integers(248, 256, n).astype(np.uint8)
        cols, gc = [a, val], [0]
    elif case == "nine_values":
        a = rng.integers(-4, 5, n).astype(np.int32)
        cols, gc = [a, val], [0]
    else:
        a = np.full(n, 2**31 - 1, dtype=np.int32)
        cols, gc = [a, val], [0]
    vc = len(cols) - 1
    check(ctx, cols, [(vc, "gt", -10**11)], gc, [("sum", [("col", vc)]), ("count", None), ("avg", [("col", vc)])],
          capacity=16)


# ---- MIN / MAX (few groups: the direct kernel) -----------------------------------


def test_min_max_dense_groups(ctx):
    """MIN/MAX next to COUNT on the six-group shape (dense slot ids), with an
    expression argument."""
    cols = q1_cols(300_007, 91)
    aggs = [("min", [("col", 4)]), ("max", [("col", 4)]), ("count", None),
            ("max", [("col", 3), ("col", 5), "mul"])]
    check(ctx, cols, [(0, "le", 2450)], [1, 2], aggs, capacity=64)


def test_min_max_sparse_keys_and_extremes(ctx):
    """Keys too sparse for dense ids (warp key lists, flushed when full) and
    int64 extremes, whose order-preserving codes are the zero start."""
    rng = np.random.default_rng(93)
    n = 250_001
    kk = (rng.integers(0, 20, n) * 3 - 7).astype(np.int32)
    v = rng.integers(-10**18, 10**18, n).astype(np.int64)
    v[::997] = np.iinfo(np.int64).min
    v[5::991] = np.iinfo(np.int64).max
    check(ctx, [kk, v], [], [0], [("min", [("col", 1)]), ("max", [("col", 1)]), ("count", None)], capacity=32)


def test_min_max_with_sum_avg_and_ungrouped(ctx):
    """MIN and SUM of the same expression are separate accumulators (AVG shares
    the SUM); the ungrouped form over rows and over no rows (0, NaN flag)."""
    cols = q1_cols(120_001, 95)
    aggs = [("sum", [("col", 4)]), ("min", [("col", 4)]), ("avg", [("col", 4)]), ("max", [("col", 0)])]
    check(ctx, cols, [(0, "le", 2450)], [1], aggs, capacity=8)
    check(ctx, cols, [(0, "le", 2450)], [], aggs, capacity=1)
    check(ctx, cols, [(0, "gt", 99_999)], [], aggs, capacity=1)


def test_min_max_many_groups_and_wide_shapes(ctx):
    """MIN/MAX beyond the direct kernel's shapes (more than 64 groups, more than four predicates or three
    accumulators) run through the sort-based aggregation on the default path: the oracle's groups."""
    rng = np.random.default_rng(97)
    n = 300_007
    g = rng.integers(0, 20_000, n).astype(np.int32)
    v = rng.integers(-10**15, 10**15, n).astype(np.int64)
    w = rng.integers(-5, 5, n).astype(np.int32)
    check(ctx, [g, v, w], [], [0], [("min", [("col", 1)]), ("max", [("col", 1)]), ("count", None)],
          capacity=32_768)
    cols = q1_cols(100_003, 98)  # a few groups, but five predicates and four accumulators besides COUNT
    preds = [(0, "le", 2450), (3, "ge", 2), (4, "ne", 500), (5, "ne", 3), (5, "ne", 4)]
    aggs = [("min", [("col", 4)]), ("max", [("col", 3)]), ("sum", [("col", 4)]), ("max", [("col", 5)]),
            ("count", None)]
    check(ctx, cols, preds, [1, 2], aggs, capacity=64)


@pytest.mark.parametrize("case", ["q1", "many_groups", "int64_keys", "three_keys", "min_max", "none_pass"])
def test_sort_based_aggregation(ctx, case):
    """The sort-based group-by (variant 1: rows sorted by packed group key, runs of equal keys aggregated, paper
    Section 5.4 Algorithm 3) gives the oracle's groups, keys ascending, element by element."""
    rng = np.random.default_rng(len(case))
    n = 400_003
    if case == "q1":
        cols, preds, gc, aggs = q1_cols(n, 5), [(0, "le", 2450)], [1, 2], Q1_AGGS
    elif case == "many_groups":
        g = rng.integers(0, 60_000, n).astype(np.int32)
        v = rng.integers(-10**9, 10**9, n).astype(np.int64)
        cols, preds, gc, aggs = [g, v], [(1, "gt", -9 * 10**8)], [0], [("sum", [("col", 1)]), ("count", None),
                                                                        ("avg", [("col", 1)])]
    elif case == "int64_keys":
        k = rng.choice(np.array([np.iinfo(np.int64).min, -5, 0, 3, 2**40, np.iinfo(np.int64).max]), n)
        v = rng.integers(0, 1000, n).astype(np.int64)
        cols, preds, gc, aggs = [k.astype(np.int64), v], [], [0], [("sum", [("col", 1)]), ("count", None)]
    elif case == "three_keys":
        a = rng.integers(-3, 3, n).astype(np.int32)
        b = rng.integers(0, 4, n).astype(np.uint8)
        c = rng.integers(0, 5, n).astype(np.uint8)  # (the key tuple: 32 + 8 + 8 bits)
        v = rng.integers(0, 100, n).astype(np.int64)
        cols, preds, gc, aggs = [a, b, c, v], [(3, "ne", 50)], [0, 1, 2], [("sum", [("col", 3)]), ("count", None)]
    elif case == "min_max":
        g = rng.integers(0, 5_000, n).astype(np.int32)
        v = rng.integers(-10**12, 10**12, n).astype(np.int64)
        cols, preds, gc, aggs = [g, v], [], [0], [("min", [("col", 1)]), ("max", [("col", 1)]), ("count", None)]
    else:
        cols, preds, gc, aggs = q1_cols(n, 6), [(0, "gt", 99_999)], [1, 2], Q1_AGGS
    try:
        ctx.set_variant(1)
        check(ctx, cols, preds, gc, aggs, capacity=65_536)
    finally:
        ctx.set_variant(-1)


def test_sort_based_aggregation_capacity(ctx):
    """More groups than the bound: TQP_ERR_CAPACITY and a group count of -1, as the hash aggregation reports."""
    import paper_2203_01877_gb300 as tqp
    g = np.arange(10_000, dtype=np.int32)
    try:
        ctx.set_variant(1)
        st, G, _, _, _ = gpu_groupby(ctx, [g], [], [0], [("count", None)], capacity=1000)
    finally:
        ctx.set_variant(-1)
    assert st == tqp.ERR_CAPACITY and G == -1
