"""Pins for the oracle's equi-join and join -> group-by -> top-k (CPU only).

The join's result is the multiset of index pairs with equal keys (Section 5.2:
late materialisation, the output is pairs of row indexes).  The oracle emits it
in (probe row, build row) ascending order.  Pinned against a nested loop on
tiny inputs, the cardinality identity |join| = sum_k mult_build(k) *
mult_probe(k), and against independent numpy restatements of the paper's two
join algorithms: the sort-based join (Algorithm 1) and the interleaved hash
join with collision rounds (Algorithm 2).
"""
import numpy as np
import pytest

import datagen
import oracle


def nested_loop(bk, pk):
    out = []
    for p in range(len(pk)):
        for b in range(len(bk)):
            if bk[b] == pk[p]:
                out.append((b, p))
    return out


def alg1_sort_join(left, right):
    """Algorithm 1: sort both key columns, histogram per key value, multiply the
    histograms, prefix sums, then expand each output offset into a (left,
    right) index pair via a binary search over the bucket prefix sums."""
    left = np.asarray(left, np.int64)
    right = np.asarray(right, np.int64)
    base = min(left.min(initial=0), right.min(initial=0))
    lsort_idx = np.argsort(left, kind="stable")
    rsort_idx = np.argsort(right, kind="stable")
    L = left[lsort_idx] - base
    R = right[rsort_idx] - base
    m = int(max(L.max(initial=0), R.max(initial=0))) + 1
    lh = np.bincount(L, minlength=m)
    rh = np.bincount(R, minlength=m)
    hm = lh * rh
    clh, crh, chm = np.cumsum(lh), np.cumsum(rh), np.cumsum(hm)
    out_size = int(chm[-1]) if m else 0
    off = np.arange(out_size)
    bucket = np.searchsorted(chm, off, side="right")
    off = off - (chm[bucket] - hm[bucket])
    li = lsort_idx[clh[bucket] - lh[bucket] + off // rh[bucket]]
    ri = rsort_idx[crh[bucket] - rh[bucket] + off % rh[bucket]]
    return li, ri


def alg2_hash_join(left, right, m):
    """Algorithm 2: hash = key mod m; as many build/probe rounds as the largest
    hash bucket; each round scatters left indexes into an (m+1)-slot table
    (slot m retires rows already scattered), probes with the right hashes and
    keeps candidate pairs whose keys are equal."""
    left = np.asarray(left, np.int64)
    right = np.asarray(right, np.int64)
    lidx = np.arange(len(left))
    ridx = np.arange(len(right))
    lh = np.remainder(left, m)
    rh = np.remainder(right, m)
    rounds = int(np.bincount(lh, minlength=m).max(initial=0))
    lo, ro = [], []
    for _ in range(rounds):
        table = np.full(m + 1, -1, np.int64)
        table[lh] = lidx  # one writer per slot wins, as scatter_ does
        table[m] = -1
        sct = table[table >= 0]
        lh[sct] = m
        cand = table[rh]
        valid = cand >= 0
        vl, vr = cand[valid], ridx[valid]
        match = left[vl] == right[vr]
        lo.append(vl[match])
        ro.append(vr[match])
    if not lo:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    return np.concatenate(lo), np.concatenate(ro)


def canon(b, p):
    b = np.asarray(b, np.int64)
    p = np.asarray(p, np.int64)
    o = np.lexsort((b, p))
    return b[o], p[o]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_nested_loop_tiny_with_duplicates(seed):
    rng = np.random.default_rng(seed)
    bk = rng.integers(-5, 15, 60).astype(np.int32)
    pk = rng.integers(-8, 20, 90).astype(np.int32)
    b, p = oracle.join_pairs(bk, pk)
    assert list(zip(b.tolist(), p.tolist())) == nested_loop(bk.tolist(), pk.tolist())


def test_hand_worked_example():
    # build keys [7, 3, 7, 9], probe keys [3, 7, 1, 7]:
    # probe 0 (3) -> build 1; probe 1 (7) -> builds 0, 2; probe 3 (7) -> 0, 2.
    b, p = oracle.join_pairs(np.array([7, 3, 7, 9], np.int32), np.array([3, 7, 1, 7], np.int32))
    assert b.tolist() == [1, 0, 2, 0, 2]
    assert p.tolist() == [0, 1, 1, 3, 3]


def test_cardinality_identity_and_paper_algorithms():
    rng = np.random.default_rng(4)
    bk = rng.integers(0, 400, 3000).astype(np.int32)
    pk = rng.integers(0, 500, 5000).astype(np.int32)
    b, p = oracle.join_pairs(bk, pk)
    vals, cb = np.unique(bk, return_counts=True)
    cp = np.bincount(pk, minlength=500)
    assert len(b) == int((cb * cp[vals]).sum())
    assert np.all(bk[b] == pk[p])
    ob, op = canon(b, p)
    l1, r1 = alg1_sort_join(bk, pk)
    assert np.array_equal(canon(l1, r1)[0], ob) and np.array_equal(canon(l1, r1)[1], op)
    l2, r2 = alg2_hash_join(bk, pk, 64)
    assert np.array_equal(canon(l2, r2)[0], ob) and np.array_equal(canon(l2, r2)[1], op)


def test_unique_build_keys_each_probe_matches_once():
    nb = 1500
    dim = datagen.dim_table(nb, 150, seed=3)
    pr = datagen.probe_table(20000, nb, seed=3)
    b, p = oracle.join_pairs(dim["key"], pr["fk"])
    assert np.array_equal(p, np.arange(20000))
    assert np.array_equal(b, pr["fk"])  # build key == build row index


def test_join_group_topk_invariants():
    nb, ng, n = 3000, 300, 40000
    dim = datagen.dim_table(nb, ng, seed=8)
    pr = datagen.probe_table(n, nb, seed=8)
    fact = [pr["fk"], pr["value"]]
    r = oracle.run_plan(fact, (), dim=[dim["key"], dim["payload"]], fact_fk=0, dim_key=0,
                        group_cols=[3], aggs=[("sum", [("col", 1)]), ("count", None)],
                        want_row_ids=False, cap_groups=ng)
    keys, iv = r["keys"][:, 0], r["ivals"]
    assert r["num_pairs"] == n
    assert iv[:, 1].sum() == n
    assert iv[:, 0].sum() == int(pr["value"].sum())
    # independent: gather the payload of each matched build row, numpy add.at
    g = dim["payload"][pr["fk"]].astype(np.int64)
    s = np.zeros(ng, np.int64)
    np.add.at(s, g, pr["value"])
    c = np.bincount(g, minlength=ng)
    present = np.flatnonzero(c)
    assert np.array_equal(keys, present)
    assert np.array_equal(iv[:, 0], s[present]) and np.array_equal(iv[:, 1], c[present])
    # top-100 by SUM desc, key asc == brute-force full sort
    rk = oracle.run_plan(fact, (), dim=[dim["key"], dim["payload"]], fact_fk=0, dim_key=0,
                         group_cols=[3], aggs=[("sum", [("col", 1)]), ("count", None)],
                         topk=100, topk_agg=0, want_row_ids=False)
    order = np.lexsort((present, -s[present]))[:100]
    assert np.array_equal(rk["keys"][:, 0], present[order])
    assert np.array_equal(rk["ivals"][:, 0], s[present][order])
    assert rk["total_groups"] == len(present)


def test_empty_sides():
    e = np.zeros(0, np.int32)
    x = np.array([1, 2], np.int32)
    for bk, pk in [(e, x), (x, e), (e, e)]:
        b, p = oracle.join_pairs(bk, pk)
        assert len(b) == 0 and len(p) == 0


def test_semi_anti_vs_nested_loop_and_numpy():
    """Left semi / anti join: each surviving fact row once when it has an
    equal-key dim row / has none, in ascending row order, dim row -1.  Pinned
    against a nested loop on a tiny case, numpy's isin on a larger one, the
    partition identity semi + anti = surviving rows, and semi = the distinct
    fact rows of the inner join."""
    fk = np.array([4, 1, 9, 4, 7, 1, 3], np.int32)
    val = np.array([10, 20, 30, 40, 50, 60, 70], np.int64)
    dk = np.array([1, 4, 4, 5], np.int32)
    want_semi = [f for f in range(len(fk)) if any(dk[d] == fk[f] for d in range(len(dk)))]
    want_anti = [f for f in range(len(fk)) if f not in want_semi]
    for kind, want in (("semi", want_semi), ("anti", want_anti)):
        r = oracle.run_plan([fk, val], (), dim=[dk], fact_fk=0, dim_key=0, want_row_ids=False, want_pairs=True,
                            join_kind=kind, sum_expr=[("col", 1)])
        assert r["pair_fact"].tolist() == want
        assert r["pair_dim"].tolist() == [-1] * len(want)
        assert r["sum"] == int(val[want].sum())

    rng = np.random.default_rng(41)
    n = 30_000
    fk = rng.integers(-50, 2_050, n).astype(np.int32)
    g = rng.integers(0, 7, n).astype(np.int32)
    v = rng.integers(-10**9, 10**9, n).astype(np.int64)
    dk = rng.integers(0, 2_000, 5_000).astype(np.int32)  # duplicates and gaps
    preds = [(2, "gt", -5 * 10**8)]
    surv = np.flatnonzero(v > -5 * 10**8)
    hit = np.isin(fk[surv], dk)
    inner = oracle.run_plan([fk, g, v], preds, dim=[dk], fact_fk=0, dim_key=0, want_row_ids=False,
                            want_pairs=True)
    got = {}
    for kind, rows in (("semi", surv[hit]), ("anti", surv[~hit])):
        r = oracle.run_plan([fk, g, v], preds, dim=[dk], fact_fk=0, dim_key=0, group_cols=[1],
                            aggs=[("sum", [("col", 2)]), ("count", None)], want_row_ids=False, want_pairs=True,
                            join_kind=kind)
        assert np.array_equal(r["pair_fact"], rows)
        u, inv = np.unique(g[rows], return_inverse=True)
        s = np.zeros(len(u), np.int64)
        np.add.at(s, inv.reshape(-1), v[rows])
        assert np.array_equal(r["keys"].reshape(-1), u)
        assert np.array_equal(r["ivals"][:, 0], s)
        assert np.array_equal(r["ivals"][:, 1], np.bincount(inv.reshape(-1)))
        got[kind] = r["pair_fact"]
    assert np.array_equal(np.sort(np.concatenate([got["semi"], got["anti"]])), surv)
    assert np.array_equal(got["semi"], np.unique(inner["pair_fact"]))


def test_semi_anti_reject_dim_columns():
    fk = np.array([1, 2], np.int32)
    dk = np.array([1], np.int32)
    dp = np.array([9], np.int32)
    with pytest.raises(oracle.OracleError):
        oracle.run_plan([fk], (), dim=[dk, dp], fact_fk=0, dim_key=0, group_cols=[2], aggs=[("count", None)],
                        join_kind="semi")


def test_left_outer_vs_nested_loop_and_identities():
    """Left outer join: the inner pairs, and each surviving fact row without an equal-key dim row once with dim
    row -1, in (fact row, dim row) order.  Pinned against a nested loop on a tiny case; on a larger one against
    the identities outer = inner + anti (as pair sets, in canonical order) and its grouped COUNT/SUM = inner's
    + anti's, group by group."""
    fk = np.array([4, 1, 9, 4, 7, 1, 3], np.int32)
    val = np.array([10, 20, 30, 40, 50, 60, 70], np.int64)
    dk = np.array([1, 4, 4, 5], np.int32)
    want = []
    for f in range(len(fk)):
        m = [d for d in range(len(dk)) if dk[d] == fk[f]]
        want += [(f, d) for d in m] if m else [(f, -1)]
    r = oracle.run_plan([fk, val], (), dim=[dk], fact_fk=0, dim_key=0, want_row_ids=False, want_pairs=True,
                        join_kind="left_outer", sum_expr=[("col", 1)])
    assert list(zip(r["pair_fact"].tolist(), r["pair_dim"].tolist())) == want
    assert r["num_pairs"] == len(want)
    assert r["sum"] == sum(int(val[f]) for f, _ in want)
    b, p = oracle.join_pairs(dk, fk, join_kind="left_outer")
    assert list(zip(p.tolist(), b.tolist())) == want

    rng = np.random.default_rng(43)
    n = 30_000
    fk = rng.integers(-50, 2_050, n).astype(np.int32)
    g = rng.integers(0, 7, n).astype(np.int32)
    v = rng.integers(-10**9, 10**9, n).astype(np.int64)
    dk = rng.integers(0, 2_000, 5_000).astype(np.int32)
    preds = [(2, "gt", -5 * 10**8)]
    aggs = [("sum", [("col", 2)]), ("count", None)]
    res = {}
    for kind in ("inner", "anti", "left_outer"):
        res[kind] = oracle.run_plan([fk, g, v], preds, dim=[dk], fact_fk=0, dim_key=0, group_cols=[1], aggs=aggs,
                                    want_row_ids=False, want_pairs=True, join_kind=kind)
    inner, anti, outer = res["inner"], res["anti"], res["left_outer"]
    assert outer["num_pairs"] == inner["num_pairs"] + anti["num_pairs"]
    pairs = np.concatenate([np.stack([inner["pair_fact"], inner["pair_dim"]], 1),
                            np.stack([anti["pair_fact"], anti["pair_dim"]], 1)])
    pairs = pairs[np.lexsort((pairs[:, 1], pairs[:, 0]))]
    assert np.array_equal(outer["pair_fact"], pairs[:, 0]) and np.array_equal(outer["pair_dim"], pairs[:, 1])
    # grouped: per fact group, outer = inner + anti
    def by_key(r):
        return {int(k): tuple(int(x) for x in iv) for k, iv in zip(r["keys"].reshape(-1), r["ivals"])}
    gi, ga, go = by_key(inner), by_key(anti), by_key(outer)
    for k in set(gi) | set(ga):
        a, b = gi.get(k, (0, 0)), ga.get(k, (0, 0))
        assert go[k] == (a[0] + b[0], a[1] + b[1])
    assert set(go) == set(gi) | set(ga)
