"""GPU parity: batched execution (tqp_run_plans and tqp_batch_create / _run)
against the oracle's plan evaluator and against tqp_run_plan alone, bit-exact,
over a mix of plan shapes and table sizes: empty, one row, ragged tails,
several chunks, and a plan the batch hands to the single-plan path."""
import numpy as np
import pytest

import datagen
import oracle
from tests.plan_util import compare, gpu_plan, gpu_plan_collect, gpu_plan_prepare

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


def q1(n, seed):
    t = datagen.fact_table(n, seed=seed)
    return [t["date"], t["flag"], t["status"], t["quantity"], t["price"], t["discount"]]


def join_case(nb, ng, n, seed):
    dim = datagen.dim_table(nb, ng, seed=seed)
    pr = datagen.probe_table(n, nb, seed=seed)
    return [pr["fk"], pr["value"]], [dim["key"], dim["payload"]]


def oracle_of(spec):
    ospec = dict(spec)
    ospec.pop("capacity_groups", None)
    ospec.pop("max_groups", None)
    return oracle.run_plan(want_pairs=False, cap_groups=None, **ospec)


def mixed_specs():
    fact, dim = join_case(10_000, 1_000, 200_000, 5)
    f2, d2 = join_case(3_000, 40, 77_777, 6)
    rng = np.random.default_rng(21)
    g = rng.integers(0, 20_000, 150_001).astype(np.int32)
    v = rng.integers(-100, 100, 150_001).astype(np.int64)
    empty_q1 = [c[:0] for c in q1(10, 7)]
    kk = (rng.integers(0, 20, 123_457) * 3 - 7).astype(np.int32)
    fl = rng.integers(0, 3, 123_457).astype(np.uint8)
    v2 = rng.integers(-10**9, 10**9, 123_457).astype(np.int64)
    return [
        # filter: count only; count + sum + row ids
        dict(fact=q1(100_003, 1), preds=[(0, "le", 2450)]),
        dict(fact=q1(70_000, 6), preds=[(0, "lt", 400)], sum_expr=[("col", 4)], want_row_ids=True),
        # group-by into a small table; group-by with top-k
        dict(fact=q1(100_000, 4), preds=[(0, "le", 2450)], group_cols=[1, 2], aggs=Q1_AGGS, capacity_groups=64),
        dict(fact=[g, v], group_cols=[0], aggs=[("sum", [("col", 1)]), ("count", None)], topk=10, topk_agg=0,
             max_groups=32768),
        # few groups with keys too sparse for dense slot ids (warp key lists, flushed when full)
        dict(fact=[kk, fl, v2], preds=[(1, "ne", 1)], group_cols=[0],
             aggs=[("sum", [("col", 2)]), ("count", None), ("avg", [("col", 2)])], capacity_groups=32),
        # few groups with top-k (the direct kernel, then the selection)
        dict(fact=q1(80_000, 9), preds=[(0, "le", 2450)], group_cols=[1, 2], aggs=Q1_AGGS, topk=3, topk_agg=2,
             max_groups=16, capacity_groups=3),
        # a large group table without top-k: the single-plan path, inside the batch
        dict(fact=[g, v], group_cols=[0], aggs=[("count", None)], capacity_groups=20_000),
        # joins: grouped top-k; filtered, averaged, with sum and row ids; ungrouped sum
        dict(fact=fact, dim=dim, fact_fk=0, dim_key=0, group_cols=[3],
             aggs=[("sum", [("col", 1)]), ("count", None)], topk=100, topk_agg=0),
        dict(fact=f2, dim=d2, fact_fk=0, dim_key=0, preds=[(1, "lt", 5_000_000)], group_cols=[3],
             aggs=[("avg", [("col", 1)]), ("count", None)], sum_expr=[("col", 1)], want_row_ids=True,
             capacity_groups=40),
        dict(fact=f2, dim=d2, fact_fk=0, dim_key=0, sum_expr=[("col", 1)]),
        # empty and one-row tables
        dict(fact=empty_q1, preds=[(0, "le", 2450)], sum_expr=[("col", 4)], want_row_ids=True),
        dict(fact=empty_q1, group_cols=[1], aggs=[("count", None)], capacity_groups=8),
        dict(fact=[c[:1] for c in q1(10, 8)], aggs=[("sum", [("col", 3)]), ("count", None)], capacity_groups=1),
        dict(fact=[c[:0] for c in f2], dim=d2, fact_fk=0, dim_key=0, group_cols=[3], aggs=[("count", None)],
             sum_expr=[("col", 1)], capacity_groups=40),
        dict(fact=f2, dim=[c[:0] for c in d2], fact_fk=0, dim_key=0, group_cols=[3], aggs=[("count", None)],
             sum_expr=[("col", 1)], capacity_groups=40),
    ]


def clobber(bufs):
    for k, t in bufs.items():
        if t is not None:
            t.fill_(-7)


def test_run_plans_mixed(ctx):
    import paper_2203_01877_gb300 as tqp
    specs = mixed_specs()
    prepared = [gpu_plan_prepare(**s) for s in specs]
    tqp.tqp_run_plans(ctx, [p[0] for p in prepared], [p[1] for p in prepared])
    assert ctx.status() == 0
    for s, (plan, res, bufs, keep, shape) in zip(specs, prepared):
        got = gpu_plan_collect(bufs, shape)
        got["status"] = 0
        compare(got, oracle_of(s), s)


def test_batch_replays_and_interleaves(ctx):
    """A captured batch replays to the same bytes, also after single-plan calls
    have reused the arena's per-call scratch in between."""
    import paper_2203_01877_gb300 as tqp
    specs = mixed_specs()
    prepared = [gpu_plan_prepare(**s) for s in specs]
    batch = tqp.tqp_batch_create(ctx, [p[0] for p in prepared], [p[1] for p in prepared])
    try:
        wants = [oracle_of(s) for s in specs]
        for rep in range(3):
            for p in prepared:
                clobber(p[2])
            tqp.tqp_batch_run(batch)
            assert ctx.status() == 0
            for s, w, (plan, res, bufs, keep, shape) in zip(specs, wants, prepared):
                got = gpu_plan_collect(bufs, shape)
                got["status"] = 0
                compare(got, w, s)
            # single-plan calls between replays
            compare(gpu_plan(ctx, **specs[rep]), wants[rep], specs[rep])
    finally:
        tqp.tqp_batch_destroy(batch)


def random_spec(rng, i):
    n = int(np.exp(rng.uniform(np.log(1), np.log(300_000))))
    kind = i % 4
    seed = 1000 + i
    if kind == 0:
        return dict(fact=q1(n, seed), preds=[(0, "lt", int(rng.integers(1, 2500)))], sum_expr=[("col", 4)],
                    want_row_ids=bool(i % 8 == 0))
    if kind == 1:
        return dict(fact=q1(n, seed), preds=[(0, "le", int(rng.integers(1, 2500)))], group_cols=[1, 2],
                    aggs=Q1_AGGS, capacity_groups=64)
    nb = int(rng.integers(1, 5000))
    fact, dim = join_case(nb, max(1, nb // 10), n, seed)
    if kind == 2:
        return dict(fact=fact, dim=dim, fact_fk=0, dim_key=0, group_cols=[3],
                    aggs=[("sum", [("col", 1)]), ("count", None)], topk=int(rng.integers(1, 50)), topk_agg=0)
    return dict(fact=fact, dim=dim, fact_fk=0, dim_key=0, preds=[(1, "lt", int(rng.integers(0, 1 << 24)))],
                sum_expr=[("col", 1)])


def test_many_small_plans(ctx):
    """96 plans, log-uniform sizes from 1 row to 300K rows, four shapes."""
    import paper_2203_01877_gb300 as tqp
    rng = np.random.default_rng(2203)
    specs = [random_spec(rng, i) for i in range(96)]
    prepared = [gpu_plan_prepare(**s) for s in specs]
    tqp.tqp_run_plans(ctx, [p[0] for p in prepared], [p[1] for p in prepared])
    assert ctx.status() == 0
    for s, (plan, res, bufs, keep, shape) in zip(specs, prepared):
        got = gpu_plan_collect(bufs, shape)
        got["status"] = 0
        compare(got, oracle_of(s), s)


def test_batch_regions_are_released(ctx):
    import paper_2203_01877_gb300 as tqp
    specs = mixed_specs()[:4]
    prepared = [gpu_plan_prepare(**s) for s in specs]
    plans, results = [p[0] for p in prepared], [p[1] for p in prepared]
    for _ in range(3):   # create / destroy cycles must not leak the long-lived region
        a = tqp.tqp_batch_create(ctx, plans, results)
        b = tqp.tqp_batch_create(ctx, plans, results)
        tqp.tqp_batch_run(a)
        tqp.tqp_batch_run(b)
        tqp.tqp_batch_destroy(a)   # out of order
        tqp.tqp_batch_destroy(b)
    assert ctx.status() == 0
    compare(gpu_plan(ctx, **specs[2]), oracle_of(specs[2]), specs[2])


def shared_table_specs():
    """Plans over two uploaded tables: filter-only plans (count, count + sum,
    four expression shapes) that the batch packs into shared scans, grouped
    plans whose passing-row counts join the packs, and plans with row ids that
    keep their own scan."""
    rng = np.random.default_rng(31)
    big, small = q1(2_000_003, 41), q1(333_333, 42)
    exprs = [[("col", 4)], [("col", 4), ("col", 5), "mul"],
             [("col", 4), ("const", 100), ("col", 5), "sub", "mul"], [("col", 3), ("const", 7), "add"]]
    specs = []
    for i in range(44):
        d0 = int(rng.integers(0, 2200))
        preds = [(0, "ge", d0), (0, "lt", d0 + int(rng.integers(1, 400))), (1, "ne", int(rng.integers(0, 3))),
                 (3, "le", int(rng.integers(1, 51)))]
        fact = big if i % 4 else small
        if i % 11 == 5:
            specs.append(dict(fact=fact, preds=preds, group_cols=[1, 2], aggs=Q1_AGGS, capacity_groups=64))
        elif i % 13 == 7:
            specs.append(dict(fact=fact, preds=preds, sum_expr=exprs[i % 4], want_row_ids=True))
        elif i % 5 == 0:
            specs.append(dict(fact=fact, preds=preds))
        else:
            specs.append(dict(fact=fact, preds=preds, sum_expr=exprs[(i // 3) % 4]))
    return specs, big, small


def test_filter_plans_share_scans(ctx):
    """Filter-only plans over one table run as shared scans inside the batch;
    every output equals the oracle's for the plan alone (one-shot and replayed)."""
    import paper_2203_01877_gb300 as tqp
    from tests.gpu_util import up
    specs, big, small = shared_table_specs()
    refs = {id(big): tqp.TableRef([up(c) for c in big]), id(small): tqp.TableRef([up(c) for c in small])}
    prepared = [gpu_plan_prepare(fact_ref=refs[id(s["fact"])], **s) for s in specs]
    wants = [oracle_of(s) for s in specs]
    tqp.tqp_run_plans(ctx, [p[0] for p in prepared], [p[1] for p in prepared])
    assert ctx.status() == 0
    for s, w, (plan, res, bufs, keep, shape) in zip(specs, wants, prepared):
        got = gpu_plan_collect(bufs, shape)
        got["status"] = 0
        compare(got, w, s)
    batch = tqp.tqp_batch_create(ctx, [p[0] for p in prepared], [p[1] for p in prepared])
    try:
        for _ in range(2):
            for p in prepared:
                clobber(p[2])
            tqp.tqp_batch_run(batch)
            assert ctx.status() == 0
            for s, w, (plan, res, bufs, keep, shape) in zip(specs, wants, prepared):
                got = gpu_plan_collect(bufs, shape)
                got["status"] = 0
                compare(got, w, s)
    finally:
        tqp.tqp_batch_destroy(batch)
