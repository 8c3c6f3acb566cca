"""GPU: the autotuner.  With autotuning on, operator results are byte-identical
to the built-in launch shapes (filter, group-by, hash join with pairs, joined
plan, batch); choices are recorded per shape class and survive a JSON save /
load round trip."""
import json

import numpy as np
import pytest

import datagen
import oracle
from tests.plan_util import compare, gpu_plan_collect, gpu_plan_prepare

pytestmark = pytest.mark.gpu


def run_ops(ctx, tqp, torch, cols_q6, q1, join_case):
    out = {}
    T6 = tqp.TableRef(cols_q6)
    n = cols_q6[0].numel()
    ids = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    s = torch.zeros(1, dtype=torch.int64, device="cuda")
    tqp.tqp_filter(ctx, T6, [(0, "ge", 731), (0, "lt", 1096), (1, "between", 5, 7), (2, "lt", 24)],
                   [("col", 3), ("col", 1), "mul"], s, ids, n, cnt)
    k = int(cnt.item())
    out["filter"] = (k, int(s.item()), ids[:k].cpu().numpy())
    T1 = tqp.TableRef(q1)
    keys = torch.zeros(128, dtype=torch.int64, device="cuda")
    iv = torch.zeros(320, dtype=torch.int64, device="cuda")
    fv = torch.zeros(320, dtype=torch.float64, device="cuda")
    ng = torch.zeros(1, dtype=torch.int64, device="cuda")
    aggs = [("sum", [("col", 3)]), ("sum", [("col", 4)]),
            ("sum", [("col", 4), ("const", 100), ("col", 5), "sub", "mul"]), ("count", None), ("avg", [("col", 4)])]
    tqp.tqp_groupby_agg(ctx, T1, [(0, "le", 2450)], [1, 2], aggs, keys, iv, fv, 64, ng)
    g = int(ng.item())
    out["groupby"] = (g, keys[:2 * g].cpu().numpy(), iv[:5 * g].cpu().numpy(), fv[:5 * g].cpu().numpy().view(np.int64))
    fact, dim = join_case
    spec = dict(fact=fact, dim=dim, fact_fk=0, dim_key=0, group_cols=[3], aggs=[("sum", [("col", 1)]), ("count", None)],
                topk=50, topk_agg=0, capacity_groups=50)
    plan, res, bufs, keep, shape = gpu_plan_prepare(**spec)
    tqp.tqp_run_plan(ctx, plan, res)
    got = gpu_plan_collect(bufs, shape)
    out["plan"] = (got["num_groups"], got["total_groups"], got["keys"], got["ivals"])
    ctx.check()
    return out, spec, got


def same(a, b):
    for k in a:
        for x, y in zip(a[k], b[k]):
            assert np.array_equal(np.asarray(x), np.asarray(y)), k


def test_autotuned_results_equal_builtin(tmp_path):
    import torch
    import paper_2203_01877_gb300 as tqp
    t = datagen.fact_table(3_000_017, seed=41)
    cols_q6 = [torch.from_numpy(t[c]).cuda() for c in ("date", "discount", "quantity", "price")]
    q1 = [torch.from_numpy(t[c]).cuda() for c in ("date", "flag", "status", "quantity", "price", "discount")]
    d = datagen.dim_table(40_000, 2_000, seed=42)
    pr = datagen.probe_table(1_500_000, 40_000, seed=42)
    join_case = ([pr["fk"], pr["value"]], [d["key"], d["payload"]])
    base_ctx = tqp.Context(0, 1 << 30)
    base, spec, got = run_ops(base_ctx, tqp, torch, cols_q6, q1, join_case)
    want = oracle.run_plan(want_pairs=False, cap_groups=None,
                           **{k: v for k, v in spec.items() if k != "capacity_groups"})
    got["status"] = 0
    compare(got, want, spec)
    base_ctx.close()

    ctx = tqp.Context(0, 1 << 30)
    ctx.set_autotune(True)
    tuned, _, _ = run_ops(ctx, tqp, torch, cols_q6, q1, join_case)
    same(base, tuned)
    assert ctx.tuned_count >= 3
    again, _, _ = run_ops(ctx, tqp, torch, cols_q6, q1, join_case)  # cached choices
    same(base, again)
    path = str(tmp_path / "tuning.json")
    ctx.save_tuning(path)
    doc = json.load(open(path))
    assert len(doc["entries"]) == ctx.tuned_count
    assert all(e["tile_rows"] % 1024 == 0 and 2 <= e["stages"] <= 4 for e in doc["entries"])
    ctx.close()
    ctx2 = tqp.Context(0, 1 << 30)
    ctx2.load_tuning(path)
    assert ctx2.tuned_count == len(doc["entries"])
    loaded, _, _ = run_ops(ctx2, tqp, torch, cols_q6, q1, join_case)
    same(base, loaded)
    ctx2.close()


def test_autotuned_batch_matches_oracle():
    import torch
    import paper_2203_01877_gb300 as tqp
    specs = []
    for i in range(9):
        t = datagen.fact_table(200_000 + 77_777 * i, seed=60 + i)
        if i % 3 == 0:
            specs.append(dict(fact=[t[c] for c in ("date", "flag", "status", "quantity", "price", "discount")],
                              preds=[(0, "le", 2450)], group_cols=[1, 2],
                              aggs=[("sum", [("col", 4)]), ("count", None)], capacity_groups=64))
        elif i % 3 == 1:
            specs.append(dict(fact=[t[c] for c in ("date", "discount", "quantity", "price")],
                              preds=[(0, "ge", 731), (0, "lt", 1096), (1, "between", 5, 7), (2, "lt", 24)],
                              sum_expr=[("col", 3), ("col", 1), "mul"], want_row_ids=True))
        else:
            d = datagen.dim_table(5_000, 500, seed=70 + i)
            pr = datagen.probe_table(len(t["date"]), 5_000, seed=70 + i)
            specs.append(dict(fact=[pr["fk"], pr["value"]], dim=[d["key"], d["payload"]], fact_fk=0, dim_key=0,
                              group_cols=[3], aggs=[("sum", [("col", 1)]), ("count", None)], topk=10, topk_agg=0))
    ctx = tqp.Context(0, 2 << 30)
    ctx.set_autotune(True)
    prepared = [gpu_plan_prepare(**s) for s in specs]
    batch = tqp.tqp_batch_create(ctx, [p[0] for p in prepared], [p[1] for p in prepared])
    try:
        for p in prepared:
            for v in p[2].values():
                if v is not None:
                    v.fill_(-7)
        tqp.tqp_batch_run(batch)
        assert ctx.status() == 0
        for s, (plan, res, bufs, keep, shape) in zip(specs, prepared):
            got = gpu_plan_collect(bufs, shape)
            got["status"] = 0
            want = oracle.run_plan(want_pairs=False, cap_groups=None,
                                   **{k: v for k, v in s.items() if k != "capacity_groups"})
            compare(got, want, s)
    finally:
        tqp.tqp_batch_destroy(batch)
        ctx.close()
