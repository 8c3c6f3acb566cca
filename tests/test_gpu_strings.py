"""GPU parity: string columns with IN / LIKE / NOT LIKE and numeric IN, through
tqp_filter, tqp_groupby_agg, tqp_run_plan (with a join), tqp_filter_shared and
a batch, against the oracle (row ids and sums exact)."""
import numpy as np
import pytest

import datagen
import oracle
from tests.plan_util import compare, gpu_plan

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2203_01877_gb300 as tqp
    c = tqp.Context(0, 512 << 20)
    yield c
    c.close()


def table(n, seed, width=datagen.STR_WIDTH):
    t = datagen.fact_table(n, seed=seed, cols=["date", "quantity", "price", "flag"])
    s = datagen.string_column(n, seed=seed, width=width)
    return [s, t["date"], t["quantity"], t["price"], t["flag"]]


def vocab_words(seed, k, start=0):
    return [w.decode() for w in datagen.string_vocab(seed)[start:start + k]]


def run_filter(ctx, cols, preds, expr):
    import torch
    import paper_2203_01877_gb300 as tqp
    from tests.gpu_util import up
    T = tqp.TableRef([up(c) for c in cols])
    n = len(cols[0])
    ids = torch.zeros(max(n, 1), dtype=torch.int32, device="cuda")
    cnt = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    s = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    tqp.tqp_filter(ctx, T, preds, expr, s, ids, n, cnt)
    assert ctx.status() == 0
    k = int(cnt.item())
    return ids[:k].cpu().numpy(), int(s.item())


def cases(seed):
    w = vocab_words(seed, 6)
    return [
        [(0, "like", f"%{w[0][:2]}%")],
        [(0, "like", f"{w[1]}%"), (2, "lt", 30)],
        [(0, "not_like", f"%{w[2][-2:]}"), (1, "between", 500, 1500)],
        [(0, "like", f"_{w[3][1:3]}%_")],
        [(0, "in", [w[0], w[1], f"{w[2]} {w[3]}", "nope"])],
        [(0, "like", "%"), (4, "in", [0, 2])],
        [(0, "like", "")],
        [(0, "like", "%a%e%"), (0, "not_like", "%z%"), (3, "in", list(range(100, 200000, 97)))],
        [(2, "in", [1, 5, 9, 50]), (0, "like", "%_ _%")],
    ]


@pytest.mark.parametrize("n", [1, 31, 32, 33, 1000, 100_003, 2_000_000])
def test_filter_string_predicates(ctx, n):
    cols = table(n, 300 + n % 97)
    expr = [("col", 3), ("col", 2), "mul"]
    for preds in cases(300 + n % 97):
        want_ids, want_sum = oracle.filter_rows(cols, preds, expr)
        ids, s = run_filter(ctx, cols, preds, expr)
        assert np.array_equal(ids, want_ids), preds
        assert s == want_sum, preds


@pytest.mark.parametrize("width", [1, 5, 255])
def test_widths_and_full_width_strings(ctx, width):
    n = 70_001
    cols = table(n, 31, width=width)  # width 1 and 5 cut most rows: no padding byte left
    w = vocab_words(31, 3)
    for preds in ([(0, "like", w[0][:min(width, 2)] + "%")], [(0, "like", "_" * width)],
                  [(0, "in", [w[0][:width], w[1][:width]])], [(0, "not_like", "%" + w[2][-1:])],
                  [(0, "like", "%" * 3)]):
        want_ids, want_sum = oracle.filter_rows(cols, preds, [("col", 3)])
        ids, s = run_filter(ctx, cols, preds, [("col", 3)])
        assert np.array_equal(ids, want_ids) and s == want_sum, (width, preds)


def test_groupby_with_like(ctx):
    import torch
    import paper_2203_01877_gb300 as tqp
    from tests.gpu_util import up
    n = 1_000_003
    cols = table(n, 41)
    w = vocab_words(41, 2)
    preds = [(0, "like", f"%{w[0][:2]}%"), (1, "lt", 2000)]
    aggs = [("sum", [("col", 3)]), ("count", None), ("min", [("col", 2)])]
    T = tqp.TableRef([up(c) for c in cols])
    keys = torch.zeros(64, dtype=torch.int64, device="cuda")
    iv = torch.zeros(64 * 3, dtype=torch.int64, device="cuda")
    fv = torch.zeros(64 * 3, dtype=torch.float64, device="cuda")
    ng = torch.zeros(1, dtype=torch.int64, device="cuda")
    tqp.tqp_groupby_agg(ctx, T, preds, [4], aggs, keys, iv, fv, 64, ng)
    assert ctx.status() == 0
    G = int(ng.item())
    wk, wi, _ = oracle.groupby(cols, preds, [4], aggs)
    assert G == len(wk)
    assert np.array_equal(keys[:G].cpu().numpy(), wk[:, 0]) and np.array_equal(iv[:G * 3].cpu().numpy().reshape(G, 3), wi)


def test_join_plan_with_string_predicate(ctx):
    """The pass column is appended to the fact table: dimension columns move up by one."""
    n = 600_007
    pr = datagen.probe_table(n, 20_000, seed=42)
    dim = datagen.dim_table(20_000, 500, seed=42)
    s = datagen.string_column(n, seed=42)
    w = vocab_words(42, 2)
    spec = dict(fact=[pr["fk"], pr["value"], s], dim=[dim["key"], dim["payload"]], fact_fk=0, dim_key=0,
                preds=[(2, "not_like", f"%{w[0][1:3]}%"), (1, "ge", 1000)], group_cols=[4],
                aggs=[("sum", [("col", 1)]), ("count", None)], sum_expr=[("col", 1)], capacity_groups=1024)
    got = gpu_plan(ctx, **spec)
    want = oracle.run_plan(want_pairs=False, cap_groups=1024,
                           **{k: v for k, v in spec.items() if k != "capacity_groups"})
    compare(got, want, spec)


def test_shared_and_batch_paths(ctx):
    import torch
    import paper_2203_01877_gb300 as tqp
    from tests.gpu_util import up
    from tests.plan_util import gpu_plan_collect, gpu_plan_prepare
    n = 300_001
    cols = table(n, 51)
    T = tqp.TableRef([up(c) for c in cols])
    qs = []
    for preds in cases(51) + [[(1, "lt", d)] for d in (500, 900, 1300, 1700)]:
        cnt = torch.full((1,), -7, dtype=torch.int64, device="cuda")
        sm = torch.full((1,), -7, dtype=torch.int64, device="cuda")
        qs.append((preds, [("col", 3)], cnt, sm))
    launch_of = tqp.tqp_filter_shared(ctx, T, qs)
    assert ctx.status() == 0
    for (preds, ex, cnt, sm), lo in zip(qs, launch_of):
        ids, want_sum = oracle.filter_rows(cols, preds, ex)
        assert int(cnt.item()) == len(ids) and int(sm.item()) == want_sum, preds
        assert (lo == -1) == any(p[0] == 0 for p in preds)  # the string column: a scan of its own
    specs = [dict(fact=cols, preds=p, sum_expr=[("col", 3)], want_row_ids=True) for p in cases(51)[:4]]
    specs.append(dict(fact=cols, preds=cases(51)[1], group_cols=[4], aggs=[("count", None)], capacity_groups=8))
    prepared = [gpu_plan_prepare(fact_ref=T, **s_) for s_ in specs]
    tqp.tqp_run_plans(ctx, [p[0] for p in prepared], [p[1] for p in prepared])
    assert ctx.status() == 0
    for s_, (plan, res, bufs, keep, shape) in zip(specs, prepared):
        got = gpu_plan_collect(bufs, shape)
        got["status"] = 0
        want = oracle.run_plan(want_pairs=False, cap_groups=None,
                               **{k: v for k, v in s_.items() if k != "capacity_groups"})
        compare(got, want, s_)


def test_invalid_string_uses(ctx):
    import torch
    import paper_2203_01877_gb300 as tqp
    from tests.gpu_util import up
    n = 1000
    cols = table(n, 61)
    T = tqp.TableRef([up(c) for c in cols])
    cnt = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    s = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    bad = [
        ([(0, "eq", 5)], None, tqp.ERR_INVALID_ARG),             # a comparison on a string column
        ([(1, "like", "1%")], None, tqp.ERR_INVALID_ARG),        # LIKE on a number
        ([(1, "lt", 5)], [("col", 0)], tqp.ERR_INVALID_ARG),     # a string in the sum
        ([(0, "like", "x" * 256)], None, tqp.ERR_INVALID_ARG),   # pattern too long
        ([(1, "in", list(range(4000)))], None, tqp.ERR_UNSUPPORTED),  # more than the set budget
    ]
    for preds, ex, status in bad:
        with pytest.raises(tqp.TqpError) as e:
            tqp.tqp_filter(ctx, T, preds, ex, s if ex else None, None, 0, cnt)
        assert e.value.status == status, preds
    with pytest.raises(tqp.TqpError) as e:
        tqp.tqp_filter_noalloc(0, T, [(0, "like", "a%")], None, None, None, 0, cnt)
    assert e.value.status == tqp.ERR_UNSUPPORTED
    keys = torch.zeros(64, dtype=torch.int64, device="cuda")
    ng = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(tqp.TqpError) as e:  # a string group key
        tqp.tqp_groupby_agg(ctx, T, [], [0], [("count", None)], keys, keys, None, 64, ng)
    assert e.value.status == tqp.ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert int(cnt.item()) == -7


@pytest.mark.parametrize("width,seglen", [(8, 0), (64, 40)])
def test_like_random_patterns(ctx, width, seglen):
    """Random strings and patterns over 'ab%_' (the segment program), and patterns with a 40-byte
    segment (the greedy matcher), against the oracle."""
    rng = np.random.default_rng(width)
    n = 20_000
    alpha = np.frombuffer(b"ab%_", np.uint8)
    vals = [bytes(alpha[rng.integers(0, 4, int(rng.integers(0, width + 1)))]) for _ in range(n)]
    if seglen:
        vals = [b"a" * seglen + v[: width - seglen] if i % 3 == 0 else v for i, v in enumerate(vals)]
    s = oracle.pad_strings(vals, width)
    v = rng.integers(0, 1000, n).astype(np.int64)
    cols = [s, v]
    for _ in range(25):
        m = int(rng.integers(0, 7))
        pat = bytes(alpha[rng.integers(0, 4, m)])
        if seglen:
            pat = b"%" + b"a" * seglen + pat
        for op in ("like", "not_like"):
            preds = [(0, op, pat)]
            want_ids, want_sum = oracle.filter_rows(cols, preds, [("col", 1)])
            ids, sm = run_filter(ctx, cols, preds, [("col", 1)])
            assert np.array_equal(ids, want_ids) and sm == want_sum, (op, pat)
