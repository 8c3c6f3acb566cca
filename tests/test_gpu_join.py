"""GPU parity: tqp_hash_join index pairs against the CPU oracle, in canonical
(probe ascending, build ascending) order -- bit-exact."""
import numpy as np
import pytest

import datagen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2203_01877_gb300 as tqp
    c = tqp.Context(0, 2 << 30)
    yield c
    c.close()


def gpu_join(ctx, bk, pk, capacity=None):
    import torch
    import paper_2203_01877_gb300 as tqp
    from tests.gpu_util import up
    b = tqp.TableRef([up(bk)])
    p = tqp.TableRef([up(pk)])
    cap = capacity if capacity is not None else max(len(pk) * 4, 16)
    ob = torch.zeros(max(cap, 1), dtype=torch.int32, device="cuda:0")
    op = torch.zeros(max(cap, 1), dtype=torch.int32, device="cuda:0")
    cnt = torch.full((1,), -7, dtype=torch.int64, device="cuda:0")
    tqp.tqp_hash_join(ctx, b, 0, p, 0, ob, op, cap, cnt)
    st = ctx.status()
    k = int(cnt.item())
    m = min(k, cap)
    return st, k, ob[:m].cpu().numpy(), op[:m].cpu().numpy()


def check(ctx, bk, pk):
    wb, wp = oracle.join_pairs(bk, pk)
    st, k, ob, op = gpu_join(ctx, bk, pk, capacity=len(wb) + 16)
    assert st == 0
    assert k == len(wb)
    assert np.array_equal(op, wp)
    assert np.array_equal(ob, wb)
    return k


@pytest.mark.parametrize("nb,np_", [(1, 1), (10, 1000), (1000, 1), (3000, 5000), (100_000, 1_000_003)])
def test_unique_build_keys(ctx, nb, np_):
    rng = np.random.default_rng(nb + np_)
    bk = rng.permutation(nb * 2)[:nb].astype(np.int32)
    pk = rng.integers(0, nb * 2, np_).astype(np.int32)
    check(ctx, bk, pk)


@pytest.mark.parametrize("seed", [0, 1])
def test_duplicates_both_sides(ctx, seed):
    rng = np.random.default_rng(seed)
    bk = rng.integers(-50, 50, 20_000).astype(np.int32)
    pk = rng.integers(-60, 60, 30_000).astype(np.int32)
    check(ctx, bk, pk)


def test_mixed_types_and_special_values(ctx):
    bk = np.array([-1, 0, 5, -1, 2**40, np.iinfo(np.int64).min, 7] * 50, np.int64)
    pk = np.array([-1, 5, 3, 2**40, np.iinfo(np.int64).min, -1] * 70, np.int32 if False else np.int64)
    check(ctx, bk, pk)
    pk32 = np.array([-1, 5, 7, 0, 123] * 300, np.int32)
    check(ctx, bk, pk32)
    u8 = np.array([0, 5, 7, 255] * 100, np.uint8)
    check(ctx, bk, u8)


def test_empty_sides(ctx):
    e = np.zeros(0, np.int32)
    x = np.arange(100, dtype=np.int32)
    for bk, pk in [(e, x), (x, e)]:
        st, k, _, _ = gpu_join(ctx, bk, pk)
        assert st == 0 and k == 0


def test_capacity_exceeded(ctx):
    import paper_2203_01877_gb300 as tqp
    bk = np.zeros(100, np.int32)
    pk = np.zeros(100, np.int32)
    st, k, ob, op = gpu_join(ctx, bk, pk, capacity=500)
    assert st == tqp.ERR_CAPACITY and k == 10_000
    wb, wp = oracle.join_pairs(bk, pk)
    assert np.array_equal(ob, wb[:500]) and np.array_equal(op, wp[:500])


def test_zipf_probe_shape(ctx):
    nb, n = 150_000, 6_000_000
    dim = datagen.dim_table(nb, 15_000, seed=4)
    pr = datagen.probe_table(n, nb, seed=4)
    k = check(ctx, dim["key"], pr["fk"])
    assert k == n


def test_full_size_hashed_pairs(ctx):
    """Sparse build keys force the hashed table: 1.5M unique int32 keys scattered over [0, 2^31), 60M Zipf(0.5)
    probe keys.  Every probe row matches exactly one build row, so the canonical output is fixed at any size:
    probe indices 0..n-1 in order, each with the build row of its key; the oracle checks a sample of a million
    probe rows element by element."""
    from tests.plan_util import hashed_join_inputs
    dim, pr = hashed_join_inputs()
    bk, pk = dim["key"], pr["fk"]
    n = len(pk)
    st, k, ob, op = gpu_join(ctx, bk, pk, capacity=n)
    assert st == 0 and k == n
    assert np.array_equal(op, np.arange(n, dtype=np.int32))
    assert np.array_equal(bk[ob], pk)
    sample = np.sort(np.random.default_rng(0).choice(n, 1_000_000, replace=False))
    wb, wp = oracle.join_pairs(bk, pk[sample])
    assert np.array_equal(wp, np.arange(len(sample)))
    assert np.array_equal(ob[sample], wb)


def test_hashed_pairs_duplicate_build_keys(ctx):
    """Ten build rows per sparse key (1.5M build rows, 150K keys), 6M probe rows: 60M pairs.  Each probe row's
    ten build rows appear in ascending order; the oracle checks a sample of probe rows element by element."""
    from tests.plan_util import hashed_join_inputs
    dim, pr = hashed_join_inputs(n_probe=6_000_000, dup=10, seed=78)
    bk, pk = dim["key"], pr["fk"]
    n = len(pk)
    st, k, ob, op = gpu_join(ctx, bk, pk, capacity=10 * n)
    assert st == 0 and k == 10 * n
    assert np.array_equal(op, np.repeat(np.arange(n, dtype=np.int32), 10))
    assert np.array_equal(bk[ob], pk[op])
    runs = ob.reshape(n, 10)
    assert bool((np.diff(runs, axis=1) > 0).all())
    sample = np.sort(np.random.default_rng(1).choice(n, 200_000, replace=False))
    wb, wp = oracle.join_pairs(bk, pk[sample])
    assert np.array_equal(wp, np.repeat(np.arange(len(sample)), 10))
    assert np.array_equal(runs[sample].ravel(), wb)


@pytest.mark.parametrize("kind", ["inner", "semi", "anti", "left_outer"])
@pytest.mark.parametrize("case", ["dups", "sparse", "dense_big", "empty_build", "empty_probe"])
def test_join_kinds_pairs(ctx, kind, case):
    """tqp_hash_join_kind: the index pairs of every join kind (semi / anti: each kept probe row once with build
    index -1; left outer: the inner pairs plus each unmatched probe row once with -1), in canonical order,
    element by element against the oracle."""
    import torch
    import paper_2203_01877_gb300 as tqp
    from tests.gpu_util import up
    rng = np.random.default_rng(hash((kind, case)) % 2**32)
    if case == "dups":
        bk = rng.integers(-50, 50, 20_000).astype(np.int32)
        pk = rng.integers(-60, 60, 30_000).astype(np.int32)
    elif case == "sparse":
        bk = (rng.permutation(40_000).astype(np.int64) * 1_000_003 % 2**31).astype(np.int32)
        pk = np.where(rng.random(500_000) < 0.7, bk[rng.integers(0, 40_000, 500_000)],
                      rng.integers(0, 2**31 - 1, 500_000)).astype(np.int32)
    elif case == "dense_big":
        dim = datagen.dim_table(150_000, 15_000, seed=21)
        bk = dim["key"]
        pk = datagen.probe_table(3_000_000, 165_000, seed=21)["fk"]  # keys 150000.. miss
    elif case == "empty_build":
        bk = np.zeros(0, np.int32)
        pk = rng.integers(0, 100, 10_000).astype(np.int32)
    else:
        bk = rng.integers(0, 100, 1_000).astype(np.int32)
        pk = np.zeros(0, np.int32)
    wb, wp = oracle.join_pairs(bk, pk, join_kind=kind)
    cap = max(len(wb), 1)
    ob = torch.full((cap,), -7, dtype=torch.int32, device="cuda")
    op = torch.full((cap,), -7, dtype=torch.int32, device="cuda")
    cnt = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    tqp.tqp_hash_join_kind(ctx, tqp.TableRef([up(bk)]), 0, tqp.TableRef([up(pk)]), 0, kind, ob, op, cap, cnt)
    assert ctx.status() == 0
    k = int(cnt.item())
    assert k == len(wb)
    assert np.array_equal(op[:k].cpu().numpy(), wp) and np.array_equal(ob[:k].cpu().numpy(), wb)


def test_join_kind_rejected(ctx):
    import paper_2203_01877_gb300 as tqp
    from tests.gpu_util import up, zeros
    import torch
    x = up(np.arange(10, dtype=np.int32))
    with pytest.raises(tqp.TqpError) as e:
        tqp.tqp_hash_join_kind(ctx, tqp.TableRef([x]), 0, tqp.TableRef([x]), 0, 7, zeros(10, torch.int32),
                               zeros(10, torch.int32), 10, zeros(1, torch.int64))
    assert e.value.status == tqp.ERR_INVALID_ARG


@pytest.mark.parametrize("kind", ["inner", "left_outer", "semi"])
@pytest.mark.parametrize("case", ["dups", "sparse", "dense_big", "extremes", "empty_build"])
def test_sort_based_join(ctx, kind, case):
    """The sort-based join (variant 1: build keys radix-sorted, probe keys bucketized into them, paper Section
    5.2 Algorithm 1) gives the same canonical pairs as the oracle for every shape the hash table handles."""
    import torch
    import paper_2203_01877_gb300 as tqp
    from tests.gpu_util import up
    rng = np.random.default_rng(hash(("sort", kind, case)) % 2**32)
    if case == "dups":
        bk = rng.integers(-50, 50, 20_000).astype(np.int32)
        pk = rng.integers(-60, 60, 30_000).astype(np.int32)
    elif case == "sparse":
        bk = (rng.permutation(40_000).astype(np.int64) * 1_000_003 % 2**31).astype(np.int32)
        pk = np.where(rng.random(500_000) < 0.7, bk[rng.integers(0, 40_000, 500_000)],
                      rng.integers(0, 2**31 - 1, 500_000)).astype(np.int32)
    elif case == "dense_big":
        dim = datagen.dim_table(150_000, 15_000, seed=22, dup=3)
        bk = dim["key"]
        pk = datagen.probe_table(2_000_000, 51_000, seed=22)["fk"]
    elif case == "extremes":
        big = np.iinfo(np.int64)
        bk = np.array([big.min, -1, 0, 1, big.max, 7, 7, -1, 2**40] * 40, np.int64)
        pk = np.array([big.max, big.min, -1, 5, 7, 2**40, 0, -2] * 90, np.int64)
    else:
        bk = np.zeros(0, np.int32)
        pk = rng.integers(0, 100, 10_000).astype(np.int32)
    wb, wp = oracle.join_pairs(bk, pk, join_kind=kind)
    cap = max(len(wb), 1)
    ob = torch.full((cap,), -7, dtype=torch.int32, device="cuda")
    op = torch.full((cap,), -7, dtype=torch.int32, device="cuda")
    cnt = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    try:
        ctx.set_variant(1)
        tqp.tqp_hash_join_kind(ctx, tqp.TableRef([up(bk)]), 0, tqp.TableRef([up(pk)]), 0, kind, ob, op, cap, cnt)
        assert ctx.status() == 0
    finally:
        ctx.set_variant(-1)
    k = int(cnt.item())
    assert k == len(wb)
    assert np.array_equal(op[:k].cpu().numpy(), wp) and np.array_equal(ob[:k].cpu().numpy(), wb)
