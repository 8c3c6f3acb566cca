"""GPU parity: tqp_run_plan / tqp_run_plans against the oracle's plan evaluator
(bit-exact; group order by key, top-k order by aggregate then key)."""
import numpy as np
import pytest

import datagen
import oracle
from tests.plan_util import compare, gpu_plan

pytestmark = pytest.mark.gpu

Q1_AGGS = [("sum", [("col", 3)]), ("sum", [("col", 4)]),
           ("sum", [("col", 4), ("const", 100), ("col", 5), "sub", "mul"]),
           ("count", None), ("avg", [("col", 4)])]


@pytest.fixture(scope="module")
def ctx():
    import paper_2203_01877_gb300 as tqp
    c = tqp.Context(0, 2 << 30)
    yield c
    c.close()


def run_both(ctx, **spec):
    got = gpu_plan(ctx, **spec)
    ospec = dict(spec)
    ospec.pop("capacity_groups", None)
    ospec.pop("max_groups", None)
    want = oracle.run_plan(want_pairs=False, cap_groups=None, **ospec)
    compare(got, want, spec)
    return got


def q1(n, seed):
    t = datagen.fact_table(n, seed=seed)
    return [t["date"], t["flag"], t["status"], t["quantity"], t["price"], t["discount"]]


def join_case(nb, ng, n, seed):
    dim = datagen.dim_table(nb, ng, seed=seed)
    pr = datagen.probe_table(n, nb, seed=seed)
    return [pr["fk"], pr["value"]], [dim["key"], dim["payload"]]


def test_q1_plan(ctx):
    run_both(ctx, fact=q1(300_000, 1), preds=[(0, "le", 2450)], group_cols=[1, 2], aggs=Q1_AGGS,
             capacity_groups=64)


def test_q6_plan(ctx):
    t = datagen.fact_table(500_000, seed=2)
    fact = [t["date"], t["discount"], t["quantity"], t["price"]]
    run_both(ctx, fact=fact, preds=[(0, "ge", 731), (0, "lt", 1096), (1, "between", 5, 7), (2, "lt", 24)],
             sum_expr=[("col", 3), ("col", 1), "mul"], want_row_ids=True)


def test_scan_plan_topk(ctx):
    rng = np.random.default_rng(3)
    g = rng.integers(0, 5000, 400_000).astype(np.int32)
    v = rng.integers(0, 50, 400_000).astype(np.int64)
    run_both(ctx, fact=[g, v], group_cols=[0], aggs=[("sum", [("col", 1)]), ("count", None)], topk=100,
             topk_agg=0, max_groups=8192)


@pytest.mark.parametrize("dist", ["ties", "signed_wide", "few_groups", "near_ties", "all_equal_sum"])
def test_topk_rank_distributions(ctx, dist):
    """Top-k over rank distributions that take each route of the selection:
    decided by the first (log-scale) pass, by later passes, and by ties that
    leave more candidates than one block sorts."""
    rng = np.random.default_rng(11)
    n = 300_000
    if dist == "ties":            # every group has 4 rows: top-k by COUNT is all ties
        g = np.repeat(np.arange(n // 4, dtype=np.int32), 4)
        v = rng.integers(-5, 5, n).astype(np.int64)
        agg, k = 1, 1000
    elif dist == "signed_wide":   # sums of both signs over 15 decades
        g = rng.integers(0, 40_000, n).astype(np.int32)
        v = (np.sign(rng.standard_normal(n)) * 10.0 ** rng.uniform(0, 15, n)).astype(np.int64)
        agg, k = 0, 500
    elif dist == "few_groups":    # fewer groups than k
        g = rng.integers(0, 37, n).astype(np.int32)
        v = rng.integers(-1000, 1000, n).astype(np.int64)
        agg, k = 0, 100
    elif dist == "near_ties":     # large sums within a narrow band: decided in a late pass
        g = rng.integers(0, 60_000, n).astype(np.int32)
        v = (10**12 + rng.integers(0, 4, n)).astype(np.int64)
        agg, k = 0, 300
    else:                         # every group the same sum: the tie order (key) decides
        g = np.repeat(rng.permutation(n // 3).astype(np.int32), 3)
        v = np.full(n, -7, dtype=np.int64)
        agg, k = 0, 64
    run_both(ctx, fact=[g, v], group_cols=[0], aggs=[("sum", [("col", 1)]), ("count", None)], topk=k,
             topk_agg=agg, max_groups=200_000)


@pytest.mark.parametrize("k", [1, 4, 6, 10])
def test_few_groups_topk(ctx, k):
    """Top-k over a few-groups aggregate: the direct kernel fills the table and
    leaves it to the selection (k above the number of groups included)."""
    run_both(ctx, fact=q1(200_001, 60 + k), preds=[(0, "le", 2450)], group_cols=[1, 2], aggs=Q1_AGGS, topk=k,
             topk_agg=1, max_groups=16, capacity_groups=k)


def test_scan_plan_min_max(ctx):
    run_both(ctx, fact=q1(150_001, 71), preds=[(0, "le", 2450)], group_cols=[1, 2],
             aggs=[("min", [("col", 3)]), ("max", [("col", 4)]), ("count", None)], capacity_groups=64)


@pytest.mark.parametrize("rows", [20_000, 1_300_000])
def test_min_max_in_joined_plans_and_topk(ctx, rows):
    """MIN/MAX with a join (each joined row's value into its dimension group's code by atomic maximum),
    with duplicate build keys and misses, and as the top-k order (ranked by the decoded value): the oracle's
    results, element by element."""
    rng = np.random.default_rng(rows)
    fact, dim = join_case(2_000, 50, rows, 73)
    dup = [np.concatenate([dim[0], dim[0][:300]]), np.concatenate([dim[1], rng.integers(0, 50, 300).astype(np.int32)])]
    fk = fact[0].copy()
    fk[::17] = 99_999  # misses
    aggs = [("max", [("col", 1)]), ("min", [("col", 1), ("const", -3), "mul"]), ("count", None),
            ("sum", [("col", 1)])]
    for d in (dim, dup):
        run_both(ctx, fact=[fk, fact[1]], dim=d, fact_fk=0, dim_key=0, group_cols=[3], aggs=aggs,
                 capacity_groups=64)
        for agg in (0, 1):
            run_both(ctx, fact=[fk, fact[1]], dim=d, fact_fk=0, dim_key=0, group_cols=[3], aggs=aggs, topk=5,
                     topk_agg=agg, capacity_groups=5)
    # without a join: top-k by MIN (the direct kernel) and by MAX over many groups (the sort-based path)
    run_both(ctx, fact=q1(5_000, 74), group_cols=[1], aggs=[("min", [("col", 4)])], topk=2, topk_agg=0,
             max_groups=8, capacity_groups=2)
    g = rng.integers(0, 5_000, 50_000).astype(np.int32)
    v = rng.integers(-10**12, 10**12, 50_000).astype(np.int64)
    run_both(ctx, fact=[g, v], group_cols=[0], aggs=[("max", [("col", 1)]), ("count", None)], topk=25,
             topk_agg=0, max_groups=8192, capacity_groups=25)


@pytest.mark.parametrize("topk", [0, 1, 100, 1000])
def test_join_group_topk(ctx, topk):
    fact, dim = join_case(30_000, 3_000, 1_200_000, 7)
    run_both(ctx, fact=fact, dim=dim, fact_fk=0, dim_key=0, group_cols=[3],
             aggs=[("sum", [("col", 1)]), ("count", None)], topk=topk, topk_agg=0,
             capacity_groups=(topk or 3000))


def test_join_with_filter_sum_ids_and_avg(ctx):
    fact, dim = join_case(20_000, 500, 800_000, 9)
    run_both(ctx, fact=fact, dim=dim, fact_fk=0, dim_key=0, preds=[(1, "lt", 5_000_000)], group_cols=[3],
             aggs=[("avg", [("col", 1)]), ("count", None), ("sum", [("col", 1), ("const", 3), "mul"])],
             sum_expr=[("col", 1)], want_row_ids=True, capacity_groups=500)


def test_join_duplicates_and_misses(ctx):
    rng = np.random.default_rng(11)
    dk = rng.integers(0, 2000, 6000).astype(np.int32)     # duplicate dimension keys
    dp = rng.integers(-50, 50, 6000).astype(np.int32)
    fk = rng.integers(-100, 2100, 300_000).astype(np.int32)  # some miss
    fv = rng.integers(-1000, 1000, 300_000).astype(np.int64)
    run_both(ctx, fact=[fk, fv], dim=[dk, dp], fact_fk=0, dim_key=0, group_cols=[3],
             aggs=[("sum", [("col", 1)]), ("count", None)], sum_expr=[("col", 1)], capacity_groups=200)
    run_both(ctx, fact=[fk, fv], dim=[dk, dp], fact_fk=0, dim_key=0, group_cols=[],
             aggs=[("sum", [("col", 1)]), ("count", None)], capacity_groups=1)


def test_unsupported_join_shapes(ctx):
    import paper_2203_01877_gb300 as tqp
    fact, dim = join_case(1000, 10, 5000, 1)
    with pytest.raises(tqp.TqpError) as e:
        gpu_plan(ctx, fact=fact, dim=dim, group_cols=[0], aggs=[("count", None)])  # fact column as group key
    assert e.value.status == tqp.ERR_UNSUPPORTED


def test_run_plans_matches_run_plan(ctx):
    import paper_2203_01877_gb300 as tqp
    from tests.plan_util import gpu_plan_collect, gpu_plan_prepare
    fact, dim = join_case(10_000, 1_000, 200_000, 5)
    specs = [
        dict(fact=q1(100_000, 4), preds=[(0, "le", 2450)], group_cols=[1, 2], aggs=Q1_AGGS, capacity_groups=64),
        dict(fact=fact, dim=dim, fact_fk=0, dim_key=0, group_cols=[3],
             aggs=[("sum", [("col", 1)]), ("count", None)], topk=100, topk_agg=0),
        dict(fact=q1(70_000, 6), preds=[(0, "lt", 400)], sum_expr=[("col", 4)], want_row_ids=True),
    ]
    prepared = [gpu_plan_prepare(**s) for s in specs]
    tqp.tqp_run_plans(ctx, [p[0] for p in prepared], [p[1] for p in prepared])
    assert ctx.status() == 0
    for s, (plan, res, bufs, keep, shape) in zip(specs, prepared):
        batched = gpu_plan_collect(bufs, shape)
        batched["status"] = 0
        alone = gpu_plan(ctx, **s)
        for k in alone:
            if isinstance(alone[k], np.ndarray):
                assert np.array_equal(alone[k].view(np.int64) if alone[k].dtype == np.float64 else alone[k],
                                      batched[k].view(np.int64) if batched[k].dtype == np.float64 else batched[k])
            else:
                assert alone[k] == batched[k]


def test_full_size_join_group_topk(ctx):
    """Build 1.5M unique keys, probe 60M Zipf(0.5) foreign keys, 150K groups, top-100."""
    nb, ng, n = 1_500_000, 150_000, 60_000_000
    dim = datagen.dim_table(nb, ng, seed=datagen.DEFAULT_SEED + 2)
    pr = datagen.probe_table(n, nb, seed=datagen.DEFAULT_SEED + 2)
    got = run_both(ctx, fact=[pr["fk"], pr["value"]], dim=[dim["key"], dim["payload"]], fact_fk=0, dim_key=0,
                   group_cols=[3], aggs=[("sum", [("col", 1)]), ("count", None)], topk=100, topk_agg=0)
    assert got["num_pairs"] == n and got["total_groups"] == ng


HASHED_AGGS = [("sum", [("col", 1)]), ("count", None)]


def test_full_size_hashed_join_group_topk(ctx):
    """Sparse build keys force the hashed join table: build 1.5M unique int32 keys scattered over [0, 2^31),
    probe 60M Zipf(0.5) foreign keys, 150K groups.  The full group table (keys ascending) and the top-100,
    each element by element against the oracle."""
    from tests.plan_util import hashed_join_inputs
    dim, pr = hashed_join_inputs()
    n = len(pr["fk"])
    spec = dict(fact=[pr["fk"], pr["value"]], dim=[dim["key"], dim["payload"]], fact_fk=0, dim_key=0,
                group_cols=[3], aggs=HASHED_AGGS)
    got = gpu_plan(ctx, capacity_groups=150_000, **spec)
    full = oracle.run_plan(want_pairs=False, cap_groups=None, want_row_ids=False, **spec)
    compare(got, full, spec)
    assert full["num_pairs"] == n and full["total_groups"] == 150_000 and full["num_groups"] == 150_000
    assert int(full["ivals"][:, 1].sum()) == n and int(full["ivals"][:, 0].sum()) == int(pr["value"].sum())
    # top-100: the oracle ranks the groups whose SUM reaches the 100th largest SUM of its own full table
    # (every group that can be in the top 100, ties included); restricting the dimension to their rows
    # leaves those groups' aggregates unchanged and lets the oracle run in seconds
    got = gpu_plan(ctx, topk=100, topk_agg=0, **spec)
    sums = full["ivals"][:, 0]
    cut = np.partition(sums, len(sums) - 100)[len(sums) - 100]
    cand = full["keys"][sums >= cut, 0]
    keep = np.isin(dim["payload"], cand)
    want = oracle.run_plan(fact=spec["fact"], dim=[dim["key"][keep], dim["payload"][keep]], fact_fk=0, dim_key=0,
                           group_cols=[3], aggs=HASHED_AGGS, topk=100, topk_agg=0, want_pairs=False,
                           cap_groups=None, want_row_ids=False)
    assert got["status"] == 0 and got["num_groups"] == want["num_groups"] == 100
    assert got["total_groups"] == 150_000
    assert np.array_equal(got["keys"], want["keys"]) and np.array_equal(got["ivals"], want["ivals"])


def test_hashed_join_duplicate_build_keys(ctx):
    """Ten build rows per sparse key (150K keys, each row its own payload group): every probe row joins ten
    build rows, so each adds to up to ten groups; the full table and the top-100 against the oracle."""
    from tests.plan_util import hashed_join_inputs
    dim, pr = hashed_join_inputs(n_probe=2_000_000, dup=10, seed=77)
    n = len(pr["fk"])
    spec = dict(fact=[pr["fk"], pr["value"]], dim=[dim["key"], dim["payload"]], fact_fk=0, dim_key=0,
                group_cols=[3], aggs=HASHED_AGGS)
    got = run_both(ctx, capacity_groups=150_000, **spec)
    assert got["num_pairs"] == 10 * n
    run_both(ctx, topk=100, topk_agg=0, **spec)


def _variant_case(name):
    """Grouped join plans of >= 2^20 fact rows (the size from which the radix-partitioned aggregation is the
    default), with misses, predicates, two sums, duplicate build keys, sparse keys and top-k."""
    rng = np.random.default_rng(len(name))
    n = 1_300_003
    if name == "sparse_keys_topk":
        dim = datagen.dim_table(60_000, 4_000, seed=11, sparse=True)
        pr = datagen.probe_table(n, 60_000, seed=11, sparse=True)
        fk = pr["fk"].copy()
        fk[::13] = 12345  # (not a sparse key: misses)
        return dict(fact=[fk, pr["value"]], dim=[dim["key"], dim["payload"]], fact_fk=0, dim_key=0,
                    group_cols=[3], aggs=[("sum", [("col", 1)]), ("count", None)], topk=50, topk_agg=0)
    if name == "duplicate_keys":
        dim = datagen.dim_table(90_000, 2_500, seed=12, dup=3)  # 30K keys, three build rows each
        pr = datagen.probe_table(n, 31_000, seed=12)  # keys 30000.. miss
        return dict(fact=[pr["fk"], pr["value"]], dim=[dim["key"], dim["payload"]], fact_fk=0, dim_key=0,
                    group_cols=[3], aggs=[("sum", [("col", 1)]), ("count", None)], capacity_groups=4096)
    dim = datagen.dim_table(50_000, 5_000, seed=13)
    pr = datagen.probe_table(n, 55_000, seed=13)  # keys 50000.. miss
    qty = rng.integers(1, 51, n).astype(np.int32)
    fact = [pr["fk"], pr["value"], qty]
    d = [dim["key"], dim["payload"]]
    if name == "count_only":
        return dict(fact=fact, dim=d, fact_fk=0, dim_key=0, group_cols=[4], aggs=[("count", None)],
                    capacity_groups=8192)
    # predicates, an ungrouped sum and two sums besides the count (AVG shares SUM(value))
    return dict(fact=fact, dim=d, fact_fk=0, dim_key=0, preds=[(2, "lt", 30), (1, "ge", 200_000)],
                group_cols=[4], aggs=[("sum", [("col", 1)]), ("sum", [("col", 1), ("const", 100), ("col", 2),
                                                                       "sub", "mul"]),
                                      ("count", None), ("avg", [("col", 1)])],
                sum_expr=[("col", 1), ("col", 2), "mul"], capacity_groups=8192)


@pytest.mark.parametrize("name", ["preds_sums", "count_only", "duplicate_keys", "sparse_keys_topk"])
def test_join_plan_variants(ctx, name):
    """Both aggregation algorithms of a grouped join plan -- radix-partitioned (0) and the fused probe (1) --
    give the oracle's result, element by element."""
    spec = _variant_case(name)
    ospec = {k: v for k, v in spec.items() if k not in ("capacity_groups",)}
    want = oracle.run_plan(want_pairs=False, cap_groups=None, want_row_ids=False, **ospec)
    try:
        for variant in (0, 1):
            ctx.set_variant(variant)
            got = gpu_plan(ctx, **spec)
            compare(got, want, spec)
    finally:
        ctx.set_variant(-1)


def _semi_case(kind, n, seed, prepared=False):
    rng = np.random.default_rng(seed)
    dk = rng.permutation(60_000)[:20_000].astype(np.int32)  # keys 0..59999, a third present
    dim = [np.concatenate([dk, dk[:500]]), rng.integers(0, 9, len(dk) + 500).astype(np.int32)]  # some duplicates
    fk = rng.integers(0, 60_000, n).astype(np.int32)
    g = rng.integers(0, 40, n).astype(np.int32)
    v = rng.integers(100, 10_000_000, n).astype(np.int64)
    q = rng.integers(1, 51, n).astype(np.int32)
    return dict(fact=[fk, g, v, q], dim=dim, fact_fk=0, dim_key=0, join_kind=kind, preds=[(3, "lt", 40)],
                group_cols=[1], aggs=[("sum", [("col", 2)]), ("count", None), ("avg", [("col", 2)]),
                                      ("sum", [("col", 2), ("col", 3), "mul"])],
                sum_expr=[("col", 2)], want_row_ids=True, capacity_groups=64)


@pytest.mark.parametrize("kind", ["semi", "anti"])
@pytest.mark.parametrize("n", [1, 5_003, 700_001])
def test_semi_anti_plans(ctx, kind, n):
    """Left semi / anti join plans: each passing fact row once if it has / has no equal dim key, grouped by a
    fact column; counts, row ids (before the join), the ungrouped sum and every group against the oracle."""
    spec = _semi_case(kind, n, n)
    run_both(ctx, **spec)
    spec = dict(spec, want_row_ids=False, group_cols=[], aggs=[("count", None)], capacity_groups=1)
    run_both(ctx, **spec)


@pytest.mark.parametrize("kind", ["semi", "anti"])
def test_semi_anti_topk_and_batched(ctx, kind):
    """Top-k over a semi / anti join plan, alone and inside a batch of mixed plans (which runs it on the
    single-plan path): both equal the oracle."""
    import paper_2203_01877_gb300 as tqp
    from tests.plan_util import gpu_plan_prepare, gpu_plan_collect
    spec = dict(_semi_case(kind, 300_007, 9), topk=7, topk_agg=0, capacity_groups=7, max_groups=64,
                want_row_ids=False)
    run_both(ctx, **spec)
    inner = dict(spec, join_kind="inner", group_cols=[5], aggs=[("sum", [("col", 2)]), ("count", None)],
                 sum_expr=None, topk=0, capacity_groups=64, max_groups=0)
    specs = [spec, inner, dict(spec, join_kind="anti" if kind == "semi" else "semi")]
    prepared = [gpu_plan_prepare(**s) for s in specs]
    tqp.tqp_run_plans(ctx, [x[0] for x in prepared], [x[1] for x in prepared])
    st = ctx.status()
    for s, x in zip(specs, prepared):
        got = gpu_plan_collect(x[2], x[4])
        got["status"] = st
        o = {k: v for k, v in s.items() if k not in ("capacity_groups", "max_groups")}
        want = oracle.run_plan(want_pairs=False, cap_groups=None, **o)
        compare(got, want, s)


def test_semi_anti_plan_rules(ctx):
    import paper_2203_01877_gb300 as tqp
    from tests.plan_util import gpu_plan_prepare
    spec = _semi_case("semi", 1000, 3)
    plan, res, bufs, keep, shape = gpu_plan_prepare(**dict(spec, group_cols=[5]))  # a dim column
    with pytest.raises(tqp.TqpError) as e:
        tqp.tqp_run_plan(ctx, plan, res)
    assert e.value.status == tqp.ERR_INVALID_ARG
    plan, res, bufs, keep, shape = gpu_plan_prepare(**dict(spec, join_kind="left_outer"))
    with pytest.raises(tqp.TqpError) as e:
        tqp.tqp_run_plan(ctx, plan, res)
    assert e.value.status == tqp.ERR_UNSUPPORTED
