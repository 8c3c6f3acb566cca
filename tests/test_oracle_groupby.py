"""Pins for the oracle's group-by aggregation and top-k (CPU only).

Group-by follows Algorithm 3 (Section 5.4): sort rows by the group-key tuple,
cut the sorted list into runs of equal keys, evaluate SUM/COUNT/AVG per run,
keys ascending.  Pinned against numpy's ``unique(return_inverse)`` +
``add.at`` (library routines), against a second, independent restatement of
Algorithm 3's tensor steps in numpy, against hand-worked values and against
the invariants sum(COUNT) = surviving rows and sum over groups of SUM = the
ungrouped SUM.
"""
import struct

import numpy as np
import pytest

import datagen
import oracle


def np_groupby(keys_2d, vals, mask):
    k = keys_2d[mask]
    v = [x[mask] for x in vals]
    uniq, inv = np.unique(k, axis=0, return_inverse=True)
    inv = inv.reshape(-1)
    sums = []
    for x in v:
        s = np.zeros(len(uniq), np.int64)
        np.add.at(s, inv, x)
        sums.append(s)
    cnt = np.bincount(inv, minlength=len(uniq)).astype(np.int64)
    return uniq, sums, cnt


def alg3_numpy(key_cols, val):
    """Algorithm 3's steps with numpy tensors: concatenate group columns, sort
    (lexicographically), permute the data, unique-consecutive with inverse,
    then a scatter-add per aggregate."""
    grps = np.stack(key_cols, axis=1)
    order = np.lexsort(grps.T[::-1])
    grps = grps[order]
    data = val[order]
    change = np.ones(len(grps), bool)
    change[1:] = np.any(grps[1:] != grps[:-1], axis=1)
    inv = np.cumsum(change) - 1
    uniq = grps[change]
    sums = np.zeros(len(uniq), np.int64)
    np.add.at(sums, inv, data)
    return uniq, sums


def test_hand_worked_example():
    # keys (flag, status) and value; rows 0..7:
    #  (1,0):10  (0,1):5  (1,0):7  (0,0):1  (0,1):4  (2,1):100  (0,0):2  (1,1):3
    # groups ascending: (0,0)->1+2=3 n2; (0,1)->5+4=9 n2; (1,0)->10+7=17 n2;
    # (1,1)->3 n1; (2,1)->100 n1.  AVG(0,1) = 4.5.
    flag = np.array([1, 0, 1, 0, 0, 2, 0, 1], np.uint8)
    status = np.array([0, 1, 0, 0, 1, 1, 0, 1], np.uint8)
    val = np.array([10, 5, 7, 1, 4, 100, 2, 3], np.int64)
    keys, iv, fv = oracle.groupby([flag, status, val], [], [0, 1],
                                  [("sum", [("col", 2)]), ("count", None), ("avg", [("col", 2)])])
    assert keys.tolist() == [[0, 0], [0, 1], [1, 0], [1, 1], [2, 1]]
    assert iv[:, 0].tolist() == [3, 9, 17, 3, 100]
    assert iv[:, 1].tolist() == [2, 2, 2, 1, 1]
    assert fv[:, 2].tolist() == [1.5, 4.5, 8.5, 3.0, 100.0]


def test_q1_shape_vs_numpy_and_invariants():
    n = 50_000
    t = datagen.fact_table(n, seed=5)
    cols = [t["date"], t["flag"], t["status"], t["quantity"], t["price"], t["discount"]]
    preds = [(0, "le", 2450)]
    aggs = [("sum", [("col", 3)]), ("sum", [("col", 4)]),
            ("sum", [("col", 4), ("const", 100), ("col", 5), "sub", "mul"]),
            ("count", None), ("avg", [("col", 4)])]
    keys, iv, fv = oracle.groupby(cols, preds, [1, 2], aggs)
    m = t["date"] <= 2450
    k2 = np.stack([t["flag"].astype(np.int64), t["status"].astype(np.int64)], 1)
    disc_price = t["price"] * (100 - t["discount"])
    uniq, sums, cnt = np_groupby(k2, [t["quantity"].astype(np.int64), t["price"], disc_price], m)
    assert np.array_equal(keys, uniq)
    assert np.array_equal(iv[:, 0], sums[0])
    assert np.array_equal(iv[:, 1], sums[1])
    assert np.array_equal(iv[:, 2], sums[2])
    assert np.array_equal(iv[:, 3], cnt)
    # AVG is one IEEE division of the two exact integers: compare bit patterns
    for g in range(len(uniq)):
        want = float(sums[1][g]) / float(cnt[g])
        assert struct.pack("<d", fv[g, 4]) == struct.pack("<d", want)
    # invariants: counts add to the surviving rows; sums add to the ungrouped sum
    assert iv[:, 3].sum() == int(m.sum())
    _, s = oracle.filter_rows(cols, preds, [("col", 4)])
    assert iv[:, 1].sum() == s
    assert len(uniq) == 6


def test_alg3_second_restatement():
    rng = np.random.default_rng(1)
    n = 3000
    a = rng.integers(-5, 5, n).astype(np.int32)
    b = rng.integers(0, 3, n).astype(np.int64)
    v = rng.integers(-1000, 1000, n).astype(np.int64)
    keys, iv, _ = oracle.groupby([a, b, v], [], [0, 1], [("sum", [("col", 2)])])
    uniq, sums = alg3_numpy([a.astype(np.int64), b], v)
    assert np.array_equal(keys, uniq)
    assert np.array_equal(iv[:, 0], sums)


def test_signed_lexicographic_key_order():
    a = np.array([3, -1, 3, -1, 0, -7], np.int32)
    b = np.array([0, 5, -2, -9, 0, 1], np.int64)
    keys, iv, _ = oracle.groupby([a, b], [], [0, 1], [("count", None)])
    assert keys.tolist() == [[-7, 1], [-1, -9], [-1, 5], [0, 0], [3, -2], [3, 0]]


def test_ungrouped_aggregate_and_empty_input():
    x = np.array([4, 6, 8], np.int64)
    keys, iv, fv = oracle.groupby([x], [], [], [("sum", [("col", 0)]), ("count", None), ("avg", [("col", 0)])])
    assert keys.shape == (1, 0)
    assert iv.tolist() == [[18, 3, 18]] and fv[0, 2] == 6.0
    keys, iv, fv = oracle.groupby([x], [(0, "gt", 100)], [], [("sum", [("col", 0)]), ("count", None), ("avg", [("col", 0)])])
    assert iv.tolist() == [[0, 0, 0]] and np.isnan(fv[0, 2])
    keys, iv, fv = oracle.groupby([x], [(0, "gt", 100)], [0], [("count", None)])
    assert keys.shape == (0, 1)


def test_topk_vs_full_sort_with_ties():
    rng = np.random.default_rng(9)
    g = rng.integers(0, 500, 20000).astype(np.int32)
    v = rng.integers(0, 4, 20000).astype(np.int64)  # many equal sums -> ties broken by key
    keys_all, iv_all, _ = oracle.groupby([g, v], [], [0], [("sum", [("col", 1)]), ("count", None)])
    order = np.lexsort((keys_all[:, 0], -iv_all[:, 0]))
    for k in (1, 10, 100, 499, 500, 800):
        keys, iv, _ = oracle.groupby([g, v], [], [0], [("sum", [("col", 1)]), ("count", None)], topk=k, topk_agg=0)
        sel = order[:k]
        assert np.array_equal(keys[:, 0], keys_all[sel, 0])
        assert np.array_equal(iv, iv_all[sel])


def test_min_max_vs_numpy():
    """MIN and MAX per group against numpy's minimum.at / maximum.at over the
    same groups (np.unique with inverse), with a predicate, an expression
    argument, all-positive and all-negative columns (so a missing first-row
    initialisation shows), and int64 extremes."""
    rng = np.random.default_rng(12)
    n = 40_000
    k1 = rng.integers(-3, 4, n).astype(np.int32)
    k2 = rng.integers(0, 5, n).astype(np.uint8)
    v = rng.integers(-10**15, 10**15, n).astype(np.int64)
    pos = rng.integers(1, 1000, n).astype(np.int32)
    neg = -rng.integers(1, 1000, n).astype(np.int64)
    v[::997] = np.iinfo(np.int64).min
    v[5::991] = np.iinfo(np.int64).max
    cols = [k1, k2, v, pos, neg]
    aggs = [("min", [("col", 2)]), ("max", [("col", 2)]), ("min", [("col", 3)]), ("max", [("col", 4)]),
            ("min", [("col", 3), ("col", 4), "add"]), ("count", None)]
    keys, iv, fv = oracle.groupby(cols, [(3, "gt", 100)], [0, 1], aggs)
    mask = pos > 100
    kk = np.stack([k1.astype(np.int64), k2.astype(np.int64)], 1)[mask]
    uniq, inv = np.unique(kk, axis=0, return_inverse=True)
    inv = inv.reshape(-1)

    def red(x, fn):
        big = np.iinfo(np.int64).max if fn is np.minimum else np.iinfo(np.int64).min
        out = np.full(len(uniq), big, dtype=np.int64)
        fn.at(out, inv, x[mask].astype(np.int64))
        return out

    want = np.stack([red(v, np.minimum), red(v, np.maximum), red(pos, np.minimum), red(neg, np.maximum),
                     red(pos.astype(np.int64) + neg, np.minimum),
                     np.bincount(inv, minlength=len(uniq)).astype(np.int64)], 1)
    assert np.array_equal(keys, uniq)
    assert np.array_equal(iv, want)
    assert np.all(fv == 0.0)


def test_min_max_hand_worked_and_empty():
    """Three groups worked by hand; the ungrouped MIN/MAX over no rows is 0
    with NaN as its flag (like AVG), and over one row is that row."""
    g = np.array([2, 1, 2, 1, 3], np.int32)
    x = np.array([5, -7, -2, 9, 4], np.int64)
    keys, iv, fv = oracle.groupby([g, x], [], [0], [("min", [("col", 1)]), ("max", [("col", 1)])])
    assert keys.tolist() == [[1], [2], [3]]
    assert iv.tolist() == [[-7, 9], [-2, 5], [4, 4]]
    keys, iv, fv = oracle.groupby([g, x], [(1, "gt", 100)], [], [("min", [("col", 1)]), ("count", None)])
    assert iv.tolist() == [[0, 0]] and np.isnan(fv[0, 0])
    keys, iv, fv = oracle.groupby([g, x], [(1, "eq", -2)], [], [("max", [("col", 1)])])
    assert iv.tolist() == [[-2]] and fv[0, 0] == 0.0


def test_topk_by_max_with_ties():
    """Top-k ranks by the MAX aggregate descending, ties by key ascending."""
    g = np.array([4, 4, 1, 1, 3, 2, 2], np.int32)
    x = np.array([7, 3, 7, 1, 9, 7, -1], np.int64)
    keys, iv, fv = oracle.groupby([g, x], [], [0], [("max", [("col", 1)])], topk=3, topk_agg=0)
    assert keys.reshape(-1).tolist() == [3, 1, 2]
    assert iv.reshape(-1).tolist() == [9, 7, 7]
