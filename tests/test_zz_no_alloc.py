"""tqp_filter_noalloc -- the filter for callers that cannot allocate device
memory -- must give exactly what tqp_filter gives.

It is called through the C ABI twice in a row on the same inputs (the shared
scratch array keeps the previous call's contents, so the second call checks
that everything that must start at zero is cleared), and each result is
compared element by element with tqp_filter's and with the CPU oracle's.
This file is collected last so a run that stops at the first failure has run
every other test first; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

import datagen
import oracle

pytestmark = pytest.mark.gpu

PREDS = [(0, "ge", 731), (0, "lt", 1096), (1, "between", 5, 7), (2, "lt", 24)]
EXPR = [("col", 3), ("col", 1), "mul"]


def _run_both(n, seed):
    import torch
    import paper_2203_01877_gb300 as tqp
    t = datagen.fact_table(n, seed=seed)
    o_ids, o_sum = oracle.filter_rows([t[k] for k in ("date", "discount", "quantity", "price")], PREDS, EXPR)
    cols = [torch.from_numpy(t[k]).cuda() for k in ("date", "discount", "quantity", "price")]
    table = tqp.TableRef(cols)
    ctx = tqp.Context(0, 64 << 20)
    ref_ids = torch.zeros(max(n, 1), dtype=torch.int32, device="cuda")
    ref_cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    ref_sum = torch.zeros(1, dtype=torch.int64, device="cuda")
    tqp.tqp_filter(ctx, table, PREDS, EXPR, ref_sum, ref_ids, n, ref_cnt)
    ctx.check()
    k = int(ref_cnt.item())
    want_ids = ref_ids[:k].cpu().numpy()
    want_sum = int(ref_sum.item())
    ctx.close()
    assert k == len(o_ids) and want_sum == o_sum
    assert np.array_equal(want_ids, o_ids)

    for _ in range(2):  # two calls in a row share the scratch array
        ids = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
        cnt = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        s = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        tqp.tqp_filter_noalloc(0, table, PREDS, EXPR, s, ids, n, cnt, status)
        torch.cuda.synchronize()
        assert int(status.item()) == tqp.OK
        assert int(cnt.item()) == k
        assert int(s.item()) == want_sum
        assert np.array_equal(ids[:k].cpu().numpy(), want_ids)


@pytest.mark.parametrize("n", [1, 4097, 1_000_003, 1 << 24])
def test_noalloc_matches_tqp_filter(n):
    _run_both(n, seed=900 + n)


def test_noalloc_rejects_oversized_tables():
    import torch
    import paper_2203_01877_gb300 as tqp
    n = (1 << 24) + 1
    col = torch.zeros(n, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(tqp.TqpError) as e:
        tqp.tqp_filter_noalloc(0, tqp.TableRef([col]), [(0, "lt", 1)], d_count=cnt)
    assert e.value.status == tqp.ERR_INVALID_ARG
    assert "at most" in str(e.value)


def test_noalloc_capacity_exceeded():
    """More passing rows than `capacity`: the status word says so, the count
    stays exact and the first `capacity` ids are the oracle's."""
    import torch
    import paper_2203_01877_gb300 as tqp
    n = 200_003
    t = datagen.fact_table(n, seed=917)
    host = [t[k] for k in ("date", "discount", "quantity", "price")]
    o_ids, o_sum = oracle.filter_rows(host, PREDS, EXPR)
    cap = len(o_ids) // 3
    table = tqp.TableRef([torch.from_numpy(a).cuda() for a in host])
    for _ in range(2):
        ids = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
        cnt = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        s = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        tqp.tqp_filter_noalloc(0, table, PREDS, EXPR, s, ids, cap, cnt, status)
        torch.cuda.synchronize()
        assert int(status.item()) == tqp.ERR_CAPACITY
        assert int(cnt.item()) == len(o_ids)
        assert int(s.item()) == o_sum
        assert np.array_equal(ids.cpu().numpy(), o_ids[:cap])
