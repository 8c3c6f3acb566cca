"""GPU parity of aggregate expressions against the oracle: every closed form
the scan bodies evaluate from the staged tile (constant, x, x + k, k - x,
a * x + b, x * y, x * (k - y), scaled products), the shapes that fall back to
the postfix interpreter (sums of two columns, triple products), and both
aggregation modes of the group-by body (lane tables: at most three sums and
eight keys; warp cache: more sums or more keys).  Tables span several tiles
and end in a ragged tail, so both the full-tile fast path and the general
path run."""
import numpy as np
import pytest

import oracle
from tests.plan_util import compare, gpu_plan

pytestmark = pytest.mark.gpu

CLOSED = [
    [("col", 1)],
    [("col", 1), ("const", 7), "add"],
    [("const", 100), ("col", 2), "sub"],
    [("col", 1), ("const", 3), "mul"],
    [("col", 1), ("const", 3), "mul", ("const", -5), "add"],
    [("const", 9)],
    [("col", 1), ("col", 2), "mul"],
    [("col", 1), ("const", 100), ("col", 2), "sub", "mul"],
    [("col", 2), ("const", 2), "mul", ("col", 1), "mul"],
    [("col", 1), ("col", 2), "mul", ("const", 3), "mul"],
    [("col", 1), ("col", 1), "mul"],
    [("const", 0), ("col", 1), "mul"],
    [("const", 4), ("col", 3), "add", ("col", 2), "mul"],
]
INTERPRETED = [
    [("col", 1), ("col", 2), "add"],
    [("col", 1), ("col", 2), "mul", ("col", 3), "mul"],
    [("col", 1), ("col", 2), "sub", ("col", 3), "add"],
]


@pytest.fixture(scope="module")
def ctx():
    import paper_2203_01877_gb300 as tqp
    c = tqp.Context(0, 1 << 30)
    yield c
    c.close()


def table(n, ngroups, seed):
    rng = np.random.default_rng(seed)
    g = rng.integers(0, ngroups, n).astype(np.int32)
    x = rng.integers(-1_000_000, 1_000_000, n).astype(np.int64)
    y = rng.integers(-50, 50, n).astype(np.int32)
    z = rng.integers(0, 255, n).astype(np.uint8)
    return [g, x, y, z]


def run(ctx, **spec):
    got = gpu_plan(ctx, **spec)
    ospec = dict(spec)
    ospec.pop("capacity_groups", None)
    want = oracle.run_plan(want_pairs=False, cap_groups=None, **ospec)
    compare(got, want, spec)


@pytest.mark.parametrize("ngroups", [6, 40])
@pytest.mark.parametrize("chunk", range(0, len(CLOSED), 3))
def test_groupby_closed_forms(ctx, ngroups, chunk):
    """Three sums + COUNT: the lane tables with 6 keys, the warp cache with 40."""
    exprs = CLOSED[chunk:chunk + 3]
    aggs = [("sum", e) for e in exprs] + [("count", None)]
    run(ctx, fact=table(300_007, ngroups, 5 + chunk), preds=[(2, "ge", -40)], group_cols=[0], aggs=aggs,
        capacity_groups=64)


@pytest.mark.parametrize("exprs", [CLOSED[6:10], INTERPRETED, CLOSED[:2] + INTERPRETED[:1] + CLOSED[7:8]])
def test_groupby_four_sums_and_interpreter(ctx, exprs):
    aggs = [("sum", e) for e in exprs] + [("count", None), ("avg", exprs[0])]
    run(ctx, fact=table(200_003, 7, 11), preds=[(3, "lt", 200)], group_cols=[0, 3], aggs=aggs,
        capacity_groups=4096)


@pytest.mark.parametrize("sum_expr", [CLOSED[1], CLOSED[7], CLOSED[9], INTERPRETED[0]])
def test_joined_plan_closed_forms(ctx, sum_expr):
    rng = np.random.default_rng(17)
    nb = 5000
    dk = rng.permutation(nb).astype(np.int32) + 1000      # dense keys: direct-mapped table
    dp = rng.integers(0, 300, nb).astype(np.int32)
    fact = table(250_001, 10, 19)
    fact[0] = rng.integers(900, 1000 + nb + 100, 250_001).astype(np.int32)  # some misses on both sides
    run(ctx, fact=fact, dim=[dk, dp], fact_fk=0, dim_key=0, group_cols=[5],
        aggs=[("sum", sum_expr), ("sum", CLOSED[2]), ("count", None)], sum_expr=sum_expr, capacity_groups=300)


def test_joined_plan_sparse_keys(ctx):
    """Build keys spread over a wide range: the hashed (not direct-mapped) table."""
    rng = np.random.default_rng(23)
    nb = 4000
    dk = (rng.permutation(nb).astype(np.int64) * 1_000_003 - 7_000_000).astype(np.int32)
    dp = rng.integers(0, 50, nb).astype(np.int32)
    fact = table(150_003, 10, 29)
    fact[0] = dk[rng.integers(0, nb, 150_003)]
    fact[0][::7] = 123  # misses
    run(ctx, fact=fact, dim=[dk, dp], fact_fk=0, dim_key=0, group_cols=[5],
        aggs=[("sum", CLOSED[7]), ("count", None)], sum_expr=CLOSED[4], capacity_groups=64)
