"""GPU: the serving loop (tqp_server_*).  Mixed queries over seeded row ranges
of a resident fact table and a prepared dimension arrive with seeded random
gaps; every result must equal the same plan run alone (byte for byte), a
sample also equals the oracle, one-at-a-time mode gives the same, the
budget admission splits batches, and a plan that alone does not fit its slot
runs in scratch taken from the device's free memory."""
import time

import numpy as np
import pytest

import datagen
import oracle
from tests.plan_util import compare

pytestmark = pytest.mark.gpu

Q1_AGGS = [("sum", [("col", 3)]), ("sum", [("col", 4)]),
           ("sum", [("col", 4), ("const", 100), ("col", 5), "sub", "mul"]), ("count", None), ("avg", [("col", 4)])]
FACT_COLS = ("date", "flag", "status", "quantity", "price", "discount", "key")
N_FACT = 6_000_000
N_DIM = 200_000


@pytest.fixture(scope="module")
def world():
    import torch
    import paper_2203_01877_gb300 as tqp
    ft = datagen.fact_table(N_FACT, seed=datagen.DEFAULT_SEED + 40, cols=FACT_COLS)
    host = {k: ft[k] for k in FACT_COLS}
    dev = {k: torch.from_numpy(v).cuda() for k, v in host.items()}
    d = datagen.dim_table(N_DIM, 5_000, seed=datagen.DEFAULT_SEED + 41)
    dim_host = [d["key"], d["payload"]]
    dim_dev = tqp.TableRef([torch.from_numpy(c).cuda() for c in dim_host])
    return host, dev, dim_host, dim_dev


def make_query(tqp, torch, world, kind, r0, n, prepared):
    """One query over rows [r0, r0 + n): plan, result, buffers (the layout of
    plan_util.gpu_plan_prepare), its table refs, the oracle spec and the shape."""
    host, dev, dim_host, dim_dev = world
    if kind == 0:      # q1 shape over the range
        names, dim = ("date", "flag", "status", "quantity", "price", "discount"), None
        spec = dict(preds=[(0, "le", 2450)], group_cols=[1, 2], aggs=Q1_AGGS, capacity_groups=64)
    elif kind == 1:    # q6 shape with row ids
        names, dim = ("date", "discount", "quantity", "price"), None
        spec = dict(preds=[(0, "ge", 731), (0, "lt", 1096), (1, "between", 5, 7), (2, "lt", 24)],
                    sum_expr=[("col", 3), ("col", 1), "mul"], want_row_ids=True)
    else:              # join on key with the (prepared) dimension, group by payload, top-20
        names, dim = ("key", "price"), dim_host
        spec = dict(preds=[(1, "lt", 5_000_000)], fact_fk=0, dim_key=0, group_cols=[3],
                    aggs=[("sum", [("col", 1)]), ("count", None)], topk=20, topk_agg=0, capacity_groups=20)
    T = tqp.TableRef([dev[c][r0:r0 + n] for c in names])
    ngc, na = len(spec.get("group_cols", ())), len(spec.get("aggs", ()))
    capg = spec.get("capacity_groups", 64)
    z = lambda m, dt=torch.int64: torch.full((max(m, 1),), -7, dtype=dt, device="cuda")  # noqa: E731
    ids = bool(spec.get("want_row_ids"))
    bufs = {"row_ids": z(n, torch.int32) if ids else None, "num_rows": z(1),
            "sum": z(1) if spec.get("sum_expr") is not None else None, "keys": z(capg * ngc), "ivals": z(capg * na),
            "fvals": z(capg * na, torch.float64), "num_groups": z(1), "total_groups": z(1), "num_joined": z(1)}
    plan = tqp.make_plan(T, spec["preds"], dim_dev if dim is not None else None, spec.get("fact_fk", 0),
                         spec.get("dim_key", 0), spec.get("group_cols", ()), spec.get("aggs", ()),
                         spec.get("sum_expr"), spec.get("topk", 0), spec.get("topk_agg", 0), emit_row_ids=ids,
                         prepared=prepared if dim is not None else None)
    res = tqp.make_result(bufs["row_ids"], n if ids else 0, bufs["num_rows"], bufs["sum"], bufs["keys"],
                          bufs["ivals"], bufs["fvals"], capg, bufs["num_groups"], bufs["total_groups"],
                          bufs["num_joined"])
    ospec = dict(spec, fact=[host[c][r0:r0 + n] for c in names], dim=dim)
    shape = (ngc, na, ids, spec.get("sum_expr") is not None, ngc + na > 0)
    return plan, res, bufs, T, ospec, shape


def outputs(torch, bufs):
    """Every written output as one int64 host tensor (row ids up to the count)."""
    torch.cuda.synchronize()
    parts = []
    for k in sorted(bufs):
        t = bufs[k]
        if t is None:
            continue
        if k == "row_ids":
            t = t[:max(int(bufs["num_rows"].item()), 0)]
        parts.append(t.view(torch.int64) if t.dtype == torch.float64 else t.to(torch.int64))
    return torch.cat([t.flatten() for t in parts]).cpu()


def queries(rng, count, max_rows):
    qs = []
    for i in range(count):
        n = int(np.exp(rng.uniform(np.log(10_000), np.log(max_rows))))
        r0 = int(rng.integers(0, (N_FACT - n) // 16)) * 16
        qs.append((i % 3, r0, n))
    return qs


def run_server(tqp, torch, world, qs, prepared, max_batch, max_inflight, budget, gaps):
    ctx = tqp.Context(0, budget + (64 << 20))
    srv = tqp.Server(ctx, max_batch=max_batch, max_inflight=max_inflight, budget_bytes=budget)
    made = [make_query(tqp, torch, world, k, r0, n, prepared) for (k, r0, n) in qs]
    done = {}
    try:
        for i, (plan, res, bufs, T, spec, shape) in enumerate(made):
            srv.submit(plan, res, i)
            if gaps is not None and gaps[i] > 0:
                time.sleep(gaps[i])
            for c in srv.poll():
                done[c[0]] = c
        srv.drain(120.0)
        for c in srv.poll():
            done[c[0]] = c
    finally:
        srv.close()
        ctx.close()
    return made, done


def test_server_mix_equals_alone(world):
    import torch
    import paper_2203_01877_gb300 as tqp
    rng = np.random.default_rng(5)
    qs = queries(rng, 150, 400_000)
    gaps = rng.exponential(2e-4, len(qs))
    gaps[:50] = 0  # a burst first: batches must form
    pctx = tqp.Context(0, 512 << 20)
    pdim = tqp.tqp_dim_prepare(pctx, world[3], 0, [1])
    try:
        made, done = run_server(tqp, torch, world, qs, pdim, 32, 3, 1 << 30, gaps)
        assert sorted(done) == list(range(len(qs)))
        assert all(c[1] == 0 for c in done.values())
        assert max(c[2] for c in done.values()) > 1  # batching happened
        got = [outputs(torch, m[2]) for m in made]
        # the same plans alone, on a separate context
        actx = tqp.Context(0, 1 << 30)
        try:
            for i, (k, r0, n) in enumerate(qs):
                plan, res, bufs, T, spec, shape = make_query(tqp, torch, world, k, r0, n, pdim)
                tqp.tqp_run_plan(actx, plan, res)
                assert actx.status() == 0
                assert torch.equal(outputs(torch, bufs), got[i]), f"query {i} differs alone vs in the mix"
        finally:
            actx.close()
        # a sample against the oracle
        from tests.plan_util import gpu_plan_collect
        for i in range(0, len(qs), 19):
            plan, res, bufs, T, ospec, shape = made[i]
            got_i = gpu_plan_collect(bufs, shape)
            got_i["status"] = 0
            want = oracle.run_plan(want_pairs=False, cap_groups=None,
                                   **{k: v for k, v in ospec.items() if k != "capacity_groups"})
            compare(got_i, want, ospec)
    finally:
        tqp.tqp_dim_destroy(pdim)
        pctx.close()


def test_server_one_at_a_time_and_admission(world):
    import torch
    import paper_2203_01877_gb300 as tqp
    rng = np.random.default_rng(9)
    qs = queries(rng, 40, 300_000)
    made1, done1 = run_server(tqp, torch, world, qs, None, 1, 1, 256 << 20, None)
    assert all(c[1] == 0 and c[2] == 1 for c in done1.values())
    got1 = [outputs(torch, m[2]) for m in made1]
    # a tight budget: a slot holds about two joins (each builds ~18 MB of
    # tables), so larger batches get split to fit
    made2, done2 = run_server(tqp, torch, world, qs, None, 64, 2, 96 << 20, None)
    assert all(c[1] == 0 for c in done2.values()), sorted((k, c[1]) for k, c in done2.items() if c[1])
    assert max(c[2] for c in done2.values()) > 1
    for i in range(len(qs)):
        assert torch.equal(outputs(torch, made2[i][2]), got1[i])
    # a plan that alone exceeds its slot's share runs in scratch taken from free HBM (admission by free
    # device memory); its result is the oracle's, and the others still run in the slots
    big = [(2, 0, 100_000)] + [q for q in qs if q[0] != 2][:5]  # a join builds a ~4 MB table
    made3, done3 = run_server(tqp, torch, world, big, None, 8, 2, 2 << 20, None)
    assert all(done3[i][1] == 0 for i in range(len(big))), sorted((k, c[1]) for k, c in done3.items())
    from tests.plan_util import gpu_plan_collect
    plan, res, bufs, T, ospec, shape = made3[0]
    got0 = gpu_plan_collect(bufs, shape)
    got0["status"] = 0
    want0 = oracle.run_plan(want_pairs=False, cap_groups=None,
                            **{k: v for k, v in ospec.items() if k != "capacity_groups"})
    compare(got0, want0, ospec)
