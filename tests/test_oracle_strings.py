"""Pins of the oracle's string columns, IN and LIKE (paper Section 4.1: a
string column is an (n x m) array of character codes right-padded with 0;
Section 5 lists IN and LIKE among the supported expressions).

LIKE is checked against Python's regular-expression engine (``%`` -> ``.*``,
``_`` -> ``.``, everything else literal, whole-string match) on random
strings and patterns and on hand-worked cases; IN against Python set
membership and ``numpy.isin``; a mixed plan against a row loop written here.
"""
import re

import numpy as np
import pytest

import oracle


def like_regex(pattern: bytes) -> re.Pattern:
    out = []
    for ch in pattern:
        c = bytes([ch])
        out.append(b".*" if c == b"%" else b"." if c == b"_" else re.escape(c))
    return re.compile(b"".join(out), re.DOTALL)


def strings_of(col: np.ndarray):
    return [bytes(r).split(b"\0", 1)[0] for r in col]


def rows(fact, preds):
    return oracle.run_plan(fact, preds, want_row_ids=True)["row_ids"]


def test_like_hand_worked():
    cases = [
        (b"", b"", True), (b"", b"%", True), (b"", b"%%", True), (b"", b"_", False),
        (b"abc", b"abc", True), (b"abc", b"ab", False), (b"abc", b"abcd", False),
        (b"abc", b"a%c", True), (b"abc", b"a_c", True), (b"ac", b"a_c", False), (b"ac", b"a%c", True),
        (b"aXbXc", b"%b%", True), (b"aXbXc", b"%b", False), (b"abab", b"%ab", True), (b"abab", b"ab%ab", True),
        (b"aaa", b"a%a%a", True), (b"aa", b"a%a%a", False), (b"a%b", b"a%b", True), (b"a_b", b"a_b", True),
        (b"xyz", b"___", True), (b"xyz", b"____", False), (b"xyz", b"%__", True), (b"xyz", b"%___%", True),
    ]
    width = 6
    col = oracle.pad_strings([c[0] for c in cases], width)
    for i, (s, pat, want) in enumerate(cases):
        got = rows([col], [(0, "like", pat)])
        assert (i in set(got.tolist())) == want, (s, pat)
        got_not = rows([col], [(0, "not_like", pat)])
        assert (i in set(got_not.tolist())) == (not want), (s, pat)
        assert (like_regex(pat).fullmatch(s) is not None) == want  # the reference itself, on the same cases


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_like_vs_regex_random(seed):
    rng = np.random.default_rng(seed)
    width = 7
    n = 600
    lens = rng.integers(0, width + 1, n)  # some strings fill the whole width (no padding byte)
    alpha = np.frombuffer(b"ab%_", np.uint8)
    vals = [bytes(alpha[rng.integers(0, 4, L)]) for L in lens]
    col = oracle.pad_strings(vals, width)
    for _ in range(40):
        m = int(rng.integers(0, 7))
        pat = bytes(np.frombuffer(b"ab%_", np.uint8)[rng.integers(0, 4, m)])
        rx = like_regex(pat)
        want = np.array([i for i, v in enumerate(vals) if rx.fullmatch(v)], dtype=np.int32)
        assert np.array_equal(rows([col], [(0, "like", pat)]), want), pat
        want_not = np.setdiff1d(np.arange(n, dtype=np.int32), want)
        assert np.array_equal(rows([col], [(0, "not_like", pat)]), want_not), pat


def test_in_strings_and_numbers():
    rng = np.random.default_rng(4)
    width = 5
    words = [b"red", b"green", b"blue", b"cyan", b"", b"ivory", b"red2"]
    pick = rng.integers(0, len(words), 2000)
    col = oracle.pad_strings([words[i] for i in pick], width)
    num = rng.integers(-50, 50, 2000).astype(np.int64)
    u8 = rng.integers(0, 256, 2000).astype(np.uint8)
    for sel in ([b"red", b"blue"], [b"", b"ivory"], [b"gre"], [b"red", b"red"], []):
        want = np.array([i for i, w in enumerate(pick) if words[w] in set(sel)], dtype=np.int32)
        assert np.array_equal(rows([col], [(0, "in", sel)]), want), sel
    for vals in ([0, 3, -7, 49], [-50], list(range(-60, 60, 7)), [], [5, 5, 5]):
        want = np.flatnonzero(np.isin(num, vals)).astype(np.int32)
        assert np.array_equal(rows([num], [(0, "in", vals)]), want), vals
    want = np.flatnonzero(np.isin(u8, [0, 255, 17])).astype(np.int32)
    assert np.array_equal(rows([u8], [(0, "in", [0, 255, 17])]), want)


def test_mixed_plan_vs_row_loop():
    rng = np.random.default_rng(5)
    n, width = 3000, 8
    alpha = np.frombuffer(b"abcde", np.uint8)
    vals = [bytes(alpha[rng.integers(0, 5, int(rng.integers(0, width + 1)))]) for _ in range(n)]
    s = oracle.pad_strings(vals, width)
    g = rng.integers(0, 4, n).astype(np.int32)
    x = rng.integers(0, 1000, n).astype(np.int64)
    preds = [(0, "like", "%ab%"), (0, "not_like", "e%"), (2, "lt", 700), (1, "in", [0, 2, 3])]
    r = oracle.run_plan([s, g, x], preds, group_cols=[1], aggs=[("sum", [("col", 2)]), ("count", None)],
                        sum_expr=[("col", 2)], want_row_ids=True)
    keep = [i for i in range(n) if b"ab" in vals[i] and not vals[i].startswith(b"e") and x[i] < 700 and g[i] in (0, 2, 3)]
    assert r["row_ids"].tolist() == keep
    assert r["sum"] == int(x[keep].sum())
    for key, (sm, cnt) in zip(r["keys"][:, 0], r["ivals"]):
        sel = [i for i in keep if g[i] == key]
        assert sm == int(x[sel].sum()) and cnt == len(sel)


def test_threads_give_the_same_rows():
    rng = np.random.default_rng(6)
    vals = [bytes(np.frombuffer(b"xyz", np.uint8)[rng.integers(0, 3, 4)]) for _ in range(50_001)]
    s = oracle.pad_strings(vals, 4)
    v = rng.integers(0, 100, 50_001).astype(np.int64)
    preds = [(0, "like", "%zz%"), (1, "ge", 10)]
    one = oracle.run_plan([s, v], preds, sum_expr=[("col", 1)], want_row_ids=True)
    many = oracle.run_plan([s, v], preds, sum_expr=[("col", 1)], want_row_ids=True, threads=4)
    assert np.array_equal(one["row_ids"], many["row_ids"]) and one["sum"] == many["sum"]


def test_string_columns_feed_set_predicates_only():
    s = oracle.pad_strings([b"a", b"b"], 2)
    v = np.arange(2, dtype=np.int64)
    bad = [
        dict(fact=[s, v], preds=[(0, "eq", 1)]),                                  # comparison on a string column
        dict(fact=[s, v], preds=[(1, "like", "a")]),                              # LIKE on a number
        dict(fact=[s, v], sum_expr=[("col", 0)]),                                 # string in an expression
        dict(fact=[s, v], group_cols=[0], aggs=[("count", None)]),                # string group key
        dict(fact=[v, s], dim=[v], fact_fk=1, dim_key=0, aggs=[("count", None)]),  # string join key
    ]
    for spec in bad:
        with pytest.raises(oracle.OracleError) as e:
            oracle.run_plan(want_row_ids=False, **spec)
        assert e.value.status == oracle.ERR_INVALID, spec
