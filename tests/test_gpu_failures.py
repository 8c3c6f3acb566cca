"""Failure paths, made on purpose without faulting the GPU.

* A bounded device wait that runs out: the context's wait limit is set to a
  couple of polls, so the scan engine's stage waits and the pair-output
  join's look-back give up almost at once.  The kernels then skip their
  work, stay inside their buffers and latch TQP_ERR_TIMEOUT, which
  tqp_ctx_check returns; the context stays usable, and with the default
  limit restored the same call gives the oracle's result.
* Scratch exhaustion on the host: every operator called on a context whose
  arena is too small returns TQP_ERR_OUT_OF_MEMORY before writing any output,
  leaves no long-lived region behind, and the same context then runs a call
  that fits.
"""
import numpy as np
import pytest

import datagen
import oracle

pytestmark = pytest.mark.gpu

DEFAULT_WAIT = 1 << 22
Q6_PREDS = [(0, "ge", 731), (0, "lt", 1096), (1, "between", 5, 7), (2, "lt", 24)]
Q6_EXPR = [("col", 3), ("col", 1), "mul"]


def _join_inputs():
    rng = np.random.default_rng(5)
    nb, npr = 50_000, 3_000_000
    bk = rng.permutation(10 * nb)[:nb].astype(np.int32)      # sparse keys: a hashed table
    pk = rng.integers(0, 10 * nb, npr).astype(np.int32)
    return bk, pk


def _join(ctx, bk, pk, cap):
    import torch
    import paper_2203_01877_gb300 as tqp
    from tests.gpu_util import up
    ob = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    op = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    cnt = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    tqp.tqp_hash_join(ctx, tqp.TableRef([up(bk)]), 0, tqp.TableRef([up(pk)]), 0, ob, op, cap, cnt)
    st = ctx.status()
    return st, int(cnt.item()), ob, op


def test_expired_wait_in_join_reports_timeout():
    import paper_2203_01877_gb300 as tqp
    bk, pk = _join_inputs()
    wb, wp = oracle.join_pairs(bk, pk)
    cap = len(wb) + 16
    ctx = tqp.Context(0, 512 << 20)
    try:
        ctx.set_tuning(1024, 2, 1)  # many small tiles and chunks: waits and look-backs on every CTA
        ctx.set_wait_limit(2)
        for _ in range(2):
            st, k, _, _ = _join(ctx, bk, pk, cap)
            assert st == tqp.ERR_TIMEOUT
        ctx.set_wait_limit(DEFAULT_WAIT)
        st, k, ob, op = _join(ctx, bk, pk, cap)
        assert st == 0 and k == len(wb)
        assert np.array_equal(ob[:k].cpu().numpy(), wb) and np.array_equal(op[:k].cpu().numpy(), wp)
    finally:
        ctx.close()


def test_expired_wait_in_filter_and_plan_reports_timeout():
    import torch
    import paper_2203_01877_gb300 as tqp
    from tests.gpu_util import gpu_filter
    from tests.plan_util import gpu_plan, compare
    n = 2_000_003
    t = datagen.fact_table(n, seed=41, cols=["date", "discount", "quantity", "price"])
    cols = [t[c] for c in ("date", "discount", "quantity", "price")]
    dim = datagen.dim_table(20_000, 2_000, seed=41)
    pr = datagen.probe_table(n, 20_000, seed=41)
    spec = dict(fact=[pr["fk"], pr["value"]], dim=[dim["key"], dim["payload"]], fact_fk=0, dim_key=0,
                group_cols=[3], aggs=[("sum", [("col", 1)]), ("count", None)], capacity_groups=4096)
    ctx = tqp.Context(0, 512 << 20)
    try:
        ctx.set_tuning(1024, 2, 1)
        ctx.set_wait_limit(2)
        # variant 0 of the filter and variant 1 of the joined plan (the fused probe) run through the staged
        # scan engine and its waits
        ctx.set_variant(0)
        _, _, _, st = gpu_filter(ctx, cols, Q6_PREDS, Q6_EXPR)
        assert st == tqp.ERR_TIMEOUT
        ctx.set_variant(1)
        assert gpu_plan(ctx, **spec)["status"] == tqp.ERR_TIMEOUT
        ctx.set_wait_limit(DEFAULT_WAIT)
        ctx.set_variant(0)
        ids, k, s, st = gpu_filter(ctx, cols, Q6_PREDS, Q6_EXPR)
        want_ids, want_sum = oracle.filter_rows(cols, Q6_PREDS, Q6_EXPR)
        assert st == 0 and k == len(want_ids) and s == want_sum and np.array_equal(ids, want_ids)
        ctx.set_variant(1)
        got = gpu_plan(ctx, **spec)
        want = oracle.run_plan(want_pairs=False, cap_groups=4096, **{k: v for k, v in spec.items()
                                                                      if k != "capacity_groups"})
        compare(got, want, spec)
    finally:
        ctx.close()
    torch.cuda.synchronize()


def test_arena_exhaustion_every_operator():
    import torch
    import paper_2203_01877_gb300 as tqp
    from tests.gpu_util import up
    ctx = tqp.Context(0, 256 << 10)  # 256 KB of scratch: a 4M-row selection mask alone needs 512 KB
    n = 4_000_000
    t = datagen.fact_table(n, seed=42)
    F = tqp.TableRef([up(t[c]) for c in ("date", "flag", "status", "quantity", "price", "discount", "key")])
    dim = datagen.dim_table(500_000, 5_000, seed=42)
    D = tqp.TableRef([up(dim["key"]), up(dim["payload"])])
    z = lambda m, dt=torch.int64: torch.full((m,), -7, dtype=dt, device="cuda")  # noqa: E731
    ids, cnt, s = z(n, torch.int32), z(1), z(1)

    def oom(fn):
        with pytest.raises(tqp.TqpError) as e:
            fn()
        assert e.value.status == tqp.ERR_OUT_OF_MEMORY, str(e.value)
        assert "need at least" in str(e.value)

    try:
        for _ in range(2):  # twice: a failed call leaves nothing behind
            oom(lambda: tqp.tqp_filter(ctx, F, [(0, "lt", 1000)], [("col", 4)], s, ids, n, cnt))
            keys, iv, ng = z(1 << 16), z(1 << 16), z(1)
            oom(lambda: tqp.tqp_groupby_agg(ctx, F, [], [6], [("count", None)], keys, iv, None, 1 << 16, ng))
            ob, op = z(n, torch.int32), z(n, torch.int32)
            oom(lambda: tqp.tqp_hash_join(ctx, D, 0, F, 6, ob, op, n, cnt))
            plan = tqp.make_plan(F, (), D, 6, 0, [8], [("count", None)], None, 10, 0)
            rk, riv, rng_, rtot, rj = z(10), z(10), z(1), z(1), z(1)
            res = tqp.make_result(None, 0, None, None, rk, riv, None, 10, rng_, rtot, rj)
            oom(lambda: tqp.tqp_run_plan(ctx, plan, res))
            oom(lambda: tqp.tqp_dim_prepare(ctx, D, 0, [1], max_groups=5_000))
            oom(lambda: tqp.tqp_batch_create(ctx, [plan], [res]))
            torch.cuda.synchronize()
            for x in (ids, cnt, s, keys, iv, ng, ob, op, rk, riv, rng_, rtot, rj):
                assert bool((x == -7).all())  # no output was written
        assert ctx.status() == 0
        # the same context still runs a call that fits its scratch
        small = datagen.fact_table(100_000, seed=43, cols=["date", "discount", "quantity", "price"])
        cols = [small[c] for c in ("date", "discount", "quantity", "price")]
        T = tqp.TableRef([up(c) for c in cols])
        ids2, cnt2, s2 = z(100_000, torch.int32), z(1), z(1)  # (a 16 KB selection mask)
        tqp.tqp_filter(ctx, T, Q6_PREDS, Q6_EXPR, s2, ids2, 100_000, cnt2)
        assert ctx.status() == 0
        want_ids, want_sum = oracle.filter_rows(cols, Q6_PREDS, Q6_EXPR)
        k = int(cnt2.item())
        assert k == len(want_ids) and int(s2.item()) == want_sum
        assert np.array_equal(ids2[:k].cpu().numpy(), want_ids)
        # and long-lived regions that fit: the failed ones released theirs
        sd = datagen.dim_table(2_000, 200, seed=44)
        SD = tqp.TableRef([up(sd["key"]), up(sd["payload"])])
        for _ in range(3):
            pd = tqp.tqp_dim_prepare(ctx, SD, 0, [1], max_groups=200)
            assert pd.groups == 200
            tqp.tqp_dim_destroy(pd)
    finally:
        ctx.close()
