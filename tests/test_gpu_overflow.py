"""Past the no-overflow precondition: the GPU's int64 sums and products wrap
modulo 2^64 (two's complement), which this test pins against Python's exact
integers reduced the same way (the oracle reports such inputs as overflow)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

M = 1 << 64


def wrap(x: int) -> int:
    x %= M
    return x - M if x >= (1 << 63) else x


def test_filter_sum_and_products_wrap():
    import torch
    import paper_2203_01877_gb300 as tqp
    from tests.gpu_util import up
    rng = np.random.default_rng(7)
    n = 500_003
    a = rng.integers(1 << 60, (1 << 62), n, dtype=np.int64)       # the sum of these passes 2^63 many times
    b = rng.integers(-(1 << 40), 1 << 40, n, dtype=np.int64)      # products of two such pass 2^63
    k = rng.integers(0, 10, n).astype(np.int32)
    T = tqp.TableRef([up(a), up(b), up(k)])
    ctx = tqp.Context(0, 64 << 20)
    try:
        for expr, terms in (([("col", 0)], lambda m: a[m].tolist()),
                            ([("col", 1), ("col", 1), "mul"], lambda m: [x * x for x in b[m].tolist()]),
                            ([("col", 0), ("col", 1), "mul"], lambda m: [x * y for x, y in zip(a[m].tolist(), b[m].tolist())])):
            s = torch.zeros(1, dtype=torch.int64, device="cuda")
            cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
            tqp.tqp_filter(ctx, T, [(2, "lt", 7)], expr, s, None, 0, cnt)
            assert ctx.status() == 0
            m = k < 7
            assert int(cnt.item()) == int(m.sum())
            assert int(s.item()) == wrap(sum(terms(m))), expr
    finally:
        ctx.close()


def test_groupby_sums_wrap():
    import torch
    import paper_2203_01877_gb300 as tqp
    from tests.gpu_util import up
    rng = np.random.default_rng(8)
    n = 400_009
    g = rng.integers(0, 5, n).astype(np.int32)
    v = rng.integers(1 << 61, (1 << 62), n, dtype=np.int64)
    T = tqp.TableRef([up(g), up(v)])
    ctx = tqp.Context(0, 64 << 20)
    try:
        keys = torch.zeros(8, dtype=torch.int64, device="cuda")
        iv = torch.zeros(16, dtype=torch.int64, device="cuda")
        ng = torch.zeros(1, dtype=torch.int64, device="cuda")
        tqp.tqp_groupby_agg(ctx, T, [], [0], [("sum", [("col", 1)]), ("count", None)], keys, iv, None, 8, ng)
        assert ctx.status() == 0
        G = int(ng.item())
        assert G == 5
        got = iv[:2 * G].cpu().numpy().reshape(G, 2)
        for i, key in enumerate(keys[:G].cpu().numpy()):
            sel = g == key
            assert got[i, 1] == int(sel.sum())
            assert int(got[i, 0]) == wrap(sum(v[sel].tolist()))
    finally:
        ctx.close()
