"""GPU parity of joined plans over a prepared (resident) dimension table
(tqp_dim_prepare): against the oracle, and identical to the same plans that
build their own hash table, alone and batched.  Covers direct-mapped (dense
keys) and hashed (sparse keys) tables, duplicate dimension keys, an empty
dimension, ungrouped aggregates and the mismatch errors."""
import numpy as np
import pytest

import datagen
import oracle
from tests.plan_util import compare, gpu_plan_collect, gpu_plan_prepare

pytestmark = pytest.mark.gpu

AGGS = [("sum", [("col", 1)]), ("count", None)]


@pytest.fixture(scope="module")
def ctx():
    import paper_2203_01877_gb300 as tqp
    c = tqp.Context(0, 2 << 30)
    yield c
    c.close()


def oracle_of(spec):
    ospec = {k: v for k, v in spec.items() if k not in ("capacity_groups", "max_groups", "dim_ref", "prepared")}
    return oracle.run_plan(want_pairs=False, cap_groups=None, **ospec)


def run(ctx, spec):
    import paper_2203_01877_gb300 as tqp
    plan, res, bufs, keep, shape = gpu_plan_prepare(**spec)
    tqp.tqp_run_plan(ctx, plan, res)
    got = gpu_plan_collect(bufs, shape)
    got["status"] = ctx.status()
    return got


def dim_ref(dim):
    import paper_2203_01877_gb300 as tqp
    from tests.gpu_util import up
    return tqp.TableRef([up(c) for c in dim])


def case(kind, seed):
    rng = np.random.default_rng(seed)
    if kind == "dense":
        nb = 20_000
        d = datagen.dim_table(nb, 700, seed=seed)
        dim = [d["key"], d["payload"]]
        fk = datagen.probe_table(400_003, nb, seed=seed)["fk"]
    elif kind == "sparse":
        nb = 9_000
        dk = (rng.permutation(nb).astype(np.int64) * 7_919_993 - 1_000_000_000).astype(np.int32)
        dim = [dk, rng.integers(0, 300, nb).astype(np.int32)]
        fk = dk[rng.integers(0, nb, 300_001)]
        fk[::11] = 5  # misses (unless 5 is a key)
    else:  # duplicate keys: chains
        dk = rng.integers(0, 3_000, 8_000).astype(np.int32)
        dim = [dk, rng.integers(-20, 20, 8_000).astype(np.int32)]
        fk = rng.integers(-50, 3_050, 250_001).astype(np.int32)
    value = rng.integers(-1_000_000, 1_000_000, len(fk)).astype(np.int64)
    return [fk, value], dim


@pytest.mark.parametrize("kind", ["dense", "sparse", "dup"])
@pytest.mark.parametrize("topk", [0, 25])
def test_prepared_matches_oracle_and_own_build(ctx, kind, topk):
    import paper_2203_01877_gb300 as tqp
    fact, dim = case(kind, 3 if topk else 4)
    D = dim_ref(dim)
    pdim = tqp.tqp_dim_prepare(ctx, D, 0, [1])
    try:
        spec = dict(fact=fact, dim=dim, fact_fk=0, dim_key=0, group_cols=[3], aggs=AGGS, topk=topk, topk_agg=0,
                    preds=[(1, "gt", -900_000)], sum_expr=[("col", 1), ("const", 3), "mul"],
                    capacity_groups=topk or 1024)
        want = oracle_of(spec)
        got_p = run(ctx, dict(spec, dim_ref=D, prepared=pdim))
        got_b = run(ctx, dict(spec, dim_ref=D))
        compare(got_p, want, spec)
        compare(got_b, want, spec)
        assert pdim.groups == len(np.unique(dim[1]))
    finally:
        tqp.tqp_dim_destroy(pdim)


def test_prepared_batched_mix(ctx):
    import paper_2203_01877_gb300 as tqp
    fact, dim = case("dense", 7)
    D = dim_ref(dim)
    pdim = tqp.tqp_dim_prepare(ctx, D, 0, [1])
    try:
        specs = []
        for i in range(12):
            sl = slice(i * 30_000, i * 30_000 + 17_001 + 1_000 * i)
            f = [fact[0][sl], fact[1][sl]]
            specs.append(dict(fact=f, dim=dim, fact_fk=0, dim_key=0, group_cols=[3], aggs=AGGS,
                              topk=(10 if i % 2 else 0), topk_agg=0, capacity_groups=1024, dim_ref=D,
                              prepared=(pdim if i % 3 else None)))
        prepared = [gpu_plan_prepare(**s) for s in specs]
        tqp.tqp_run_plans(ctx, [p[0] for p in prepared], [p[1] for p in prepared])
        assert ctx.status() == 0
        for s, (plan, res, bufs, keep, shape) in zip(specs, prepared):
            got = gpu_plan_collect(bufs, shape)
            got["status"] = 0
            compare(got, oracle_of(s), s)
        batch = tqp.tqp_batch_create(ctx, [p[0] for p in prepared], [p[1] for p in prepared])
        try:
            for p in prepared:
                for t in p[2].values():
                    if t is not None:
                        t.fill_(-7)
            tqp.tqp_batch_run(batch)
            assert ctx.status() == 0
            for s, (plan, res, bufs, keep, shape) in zip(specs, prepared):
                got = gpu_plan_collect(bufs, shape)
                got["status"] = 0
                compare(got, oracle_of(s), s)
        finally:
            tqp.tqp_batch_destroy(batch)
    finally:
        tqp.tqp_dim_destroy(pdim)


def test_prepared_ungrouped_and_empty(ctx):
    import paper_2203_01877_gb300 as tqp
    fact, dim = case("dense", 9)
    D = dim_ref(dim)
    p0 = tqp.tqp_dim_prepare(ctx, D, 0, [])
    try:
        assert p0.groups == 1
        spec = dict(fact=fact, dim=dim, fact_fk=0, dim_key=0, aggs=AGGS, capacity_groups=1)
        compare(run(ctx, dict(spec, dim_ref=D, prepared=p0)), oracle_of(spec), spec)
    finally:
        tqp.tqp_dim_destroy(p0)
    empty = [dim[0][:0], dim[1][:0]]
    E = dim_ref(empty)
    pe = tqp.tqp_dim_prepare(ctx, E, 0, [1])
    try:
        assert pe.groups == 0
        spec = dict(fact=fact, dim=empty, fact_fk=0, dim_key=0, group_cols=[3], aggs=AGGS, sum_expr=[("col", 1)],
                    capacity_groups=8)
        compare(run(ctx, dict(spec, dim_ref=E, prepared=pe)), oracle_of(spec), spec)
    finally:
        tqp.tqp_dim_destroy(pe)


def test_prepared_mismatch_errors(ctx):
    import paper_2203_01877_gb300 as tqp
    fact, dim = case("dense", 11)
    D = dim_ref(dim)
    pdim = tqp.tqp_dim_prepare(ctx, D, 0, [1])
    try:
        other = dim_ref(dim)  # same values, another table: not the prepared one
        for spec in (dict(fact=fact, dim=dim, fact_fk=0, dim_key=0, group_cols=[2], aggs=AGGS, dim_ref=D),
                     dict(fact=fact, dim=dim, fact_fk=0, dim_key=0, group_cols=[3], aggs=AGGS, dim_ref=other)):
            with pytest.raises(tqp.TqpError) as e:
                run(ctx, dict(spec, prepared=pdim, capacity_groups=1024))
            assert e.value.status == tqp.ERR_INVALID_ARG
    finally:
        tqp.tqp_dim_destroy(pdim)
