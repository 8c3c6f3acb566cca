"""GPU parity: the few-groups aggregate compiled at run time for each query's
shape (tqp_ctx_set_jit) against the oracle, bit-exact, on the dense-slot and
key-list paths, ragged tails, every factor kind and mixed column types; the
generic kernel gives the same results."""
import numpy as np
import pytest

import datagen
from tests.test_gpu_groupby import Q1_AGGS, check, gpu_groupby, q1_cols

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2203_01877_gb300 as tqp
    c = tqp.Context(0, 512 << 20)
    c.set_jit(2)  # every input, whatever its size
    yield c
    c.close()


def launches():
    import paper_2203_01877_gb300 as tqp
    return tqp.tqp_jit_stats()["launches"]


def run_cases():
    rng = np.random.default_rng(91)
    n = 1_000_003
    cases = [(q1_cols(n, 90), [(0, "le", 2450)], [1, 2], Q1_AGGS, 64)]            # dense slots, ragged tail
    t = datagen.fact_table(300_001, seed=92)
    cols = [t["date"], t["flag"], t["status"], t["quantity"], t["price"], t["discount"],
            (t["quantity"] % 4).astype(np.int32)]
    cases.append((cols, [(0, "ge", 100), (3, "lt", 45), (5, "between", 1, 9), (1, "ne", 2)], [1, 6, 2],
                  [("sum", [("col", 4), ("col", 5), "mul"]), ("sum", [("col", 3), ("const", 3), "add"]),
                   ("count", None), ("sum", [("const", 50), ("col", 3), "sub"])], 64))  # 24 groups: key list
    key = rng.integers(0, 33, 200_003).astype(np.int32) * 7 - 100
    flag = rng.integers(0, 3, 200_003).astype(np.uint8)
    val = rng.integers(-10**12, 10**12, 200_003).astype(np.int64)
    cases.append(([key, flag, val], [(1, "ne", 1)], [0],
                  [("sum", [("col", 2)]), ("count", None), ("avg", [("col", 2)])], 64))  # list overflow
    a = (rng.integers(0, 7, 150_001) - 2**62).astype(np.int64)
    v = rng.integers(-10**6, 10**6, 150_001).astype(np.int64)
    q = rng.integers(0, 256, 150_001).astype(np.uint8)
    cases.append(([a, v, q], [(1, "gt", -10**5), (2, "lt", 200)], [0],
                  [("sum", [("col", 1), ("const", 3), "mul", ("const", -7), "add"]),   # affine factor
                   ("sum", [("col", 1), ("col", 1), "mul"]),                           # one column twice
                   ("sum", [("col", 2), ("const", 9), "add", ("col", 1), "mul"])], 16))
    cases.append(([v, q], [], [], [("sum", [("col", 1)]), ("count", None)], 4))      # ungrouped, no condition
    return cases


def test_specialised_kernels_match_the_oracle(ctx):
    before = launches()
    cases = run_cases()
    for cols, preds, gc, aggs, cap in cases:
        check(ctx, cols, preds, gc, aggs, capacity=cap)
    assert launches() - before == len(cases)


def test_generic_and_specialised_agree(ctx):
    cols, preds, gc, aggs, cap = run_cases()[0]
    ctx.set_jit(0)
    try:
        before = launches()
        generic = gpu_groupby(ctx, cols, preds, gc, aggs, cap)
        assert launches() == before
    finally:
        ctx.set_jit(2)
    special = gpu_groupby(ctx, cols, preds, gc, aggs, cap)
    assert generic[:2] == special[:2]
    for x, y in zip(generic[2:], special[2:]):  # keys, integer values, AVG bit patterns
        assert np.array_equal(x.view(np.int64), y.view(np.int64))


def test_min_max_stays_generic(ctx):
    cols = q1_cols(100_003, 93)
    before = launches()
    check(ctx, cols, [(0, "le", 2450)], [1, 2], [("min", [("col", 4)]), ("max", [("col", 3)]), ("count", None)],
          capacity=64)
    assert launches() == before
