"""The oracle's pins must be strong enough to catch plausible mistakes.

Each case copies ``oracle/oracle.c`` to a temporary directory, plants one
mistake (a wrong comparison, a transposed operand, a dropped term, a sign
extension, a wrong tie-break ...), builds it, swaps it in for the real oracle
and runs the pin tests: at least one of them must fail.  Nothing here touches
the committed oracle source.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from tests import test_oracle_filter as tf
from tests import test_oracle_groupby as tg
from tests import test_oracle_join as tj
from tests import test_oracle_strings as ts

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")
HDR = os.path.join(os.path.dirname(oracle.__file__), "oracle.h")

MUTANTS = {
    "le_off_by_one": ("case OR_LE: return x <= p->lo;", "case OR_LE: return x < p->lo;"),
    "between_exclusive": ("x >= p->lo && x <= p->hi", "x >= p->lo && x < p->hi"),
    "ne_as_eq": ("case OR_NE: return x != p->lo;", "case OR_NE: return x == p->lo;"),
    "sub_transposed": ("__builtin_sub_overflow(a, b, &c)", "__builtin_sub_overflow(b, a, &c)"),
    "u8_sign_extended": ("(int64_t)((const uint8_t*)c->data)[row]", "(int64_t)((const int8_t*)c->data)[row]"),
    "first_predicate_only": ("for (int j = 0; j < p->npreds && keep; ++j)", "for (int j = 0; j < 1 && j < p->npreds && keep; ++j)"),
    "count_drops_first_row": ("gcnt[g] += 1;", "gcnt[g] += (i > 0);"),
    "avg_integer_division": ("f = (double)gsum[gi * na + a] / (double)gcnt[gi];", "f = (double)(gsum[gi * na + a] / gcnt[gi]);"),
    "group_key_second_col_ignored": ("for (int i = 0; i < n; ++i)\n        if (a[i] != b[i])", "for (int i = 0; i < n && i < 1; ++i)\n        if (a[i] != b[i])"),
    "join_first_match_only": ("for (int64_t j = lower_bound(sd, p->ndim, k); j < p->ndim && sd[j].key == k; ++j)",
                              "for (int64_t j = lower_bound(sd, p->ndim, k), j0 = j; j < p->ndim && sd[j].key == k && j == j0; ++j)"),
    "join_build_order_desc": ("if (x->row != y->row) return x->row < y->row ? -1 : 1;", "if (x->row != y->row) return x->row > y->row ? -1 : 1;"),
    "topk_ascending": ("return x->rank_val > y->rank_val ? -1 : 1;", "return x->rank_val < y->rank_val ? -1 : 1;"),
    "topk_tie_key_desc": ("return cmp_keys(x->key, y->key, g_ngc);                                   /* then key asc */",
                          "return -cmp_keys(x->key, y->key, g_ngc);"),
    "min_compares_as_max": ("(fn == OR_MIN ? v < *acc : v > *acc)", "(fn == OR_MIN ? v > *acc : v > *acc)"),
    "min_max_no_first_row_init": ("if (gcnt[g] == 1 || (fn == OR_MIN", "if (0 || (fn == OR_MIN"),
    "anti_keeps_matches": ("if (has == (p->join_kind == OR_JOIN_SEMI))", "if (has == (p->join_kind != OR_JOIN_INNER))"),
    "semi_ignores_first_dim_row": ("const int has = j0 < p->ndim && sd[j0].key == k;",
                                   "const int has = j0 + 1 < p->ndim && sd[j0 + 1].key == k;"),
    "left_outer_drops_unmatched": ("if (p->join_kind == OR_JOIN_LEFT_OUTER && npairs == before) {",
                                   "if (p->join_kind == OR_JOIN_LEFT_OUTER && npairs == before && 0) {"),
    "left_outer_pads_every_row": ("if (p->join_kind == OR_JOIN_LEFT_OUTER && npairs == before) {",
                                  "if (p->join_kind == OR_JOIN_LEFT_OUTER) {"),
    "sum_skips_last_row": ("for (int64_t i = 0; i < npairs; ++i) {\n            int64_t v;",
                           "for (int64_t i = 0; i + 1 < npairs; ++i) {\n            int64_t v;"),
    "like_percent_not_empty": ("nx[j] = nx[j - 1] || ok[j];", "nx[j] = ok[j];"),
    "like_underscore_as_percent": ("if (pat[j - 1] == '%') nx[j]", "if (pat[j - 1] == '%' || pat[j - 1] == '_') nx[j]"),
    "in_strings_prefix_only": ("memcmp(s, v + k * (int64_t)c->width, (size_t)c->width)",
                               "memcmp(s, v + k * (int64_t)c->width, (size_t)(c->width < 3 ? c->width : 3))"),
    "in_numbers_skips_last": ("for (int64_t k = 0; k < p->hi; ++k)\n        if (v[k] == x) return 1;",
                              "for (int64_t k = 0; k + 1 < p->hi; ++k)\n        if (v[k] == x) return 1;"),
}

PINS = [
    tf.test_hand_worked_example,
    lambda: [tf.test_each_operator_at_boundaries(op, dt) for op in tf.NP_OPS for dt in (np.int32, np.int64, np.uint8)],
    tf.test_conjunction_and_sum_vs_numpy,
    tf.test_expression_operand_order_and_ops,
    tf.test_edge_cases,
    tg.test_hand_worked_example,
    tg.test_q1_shape_vs_numpy_and_invariants,
    tg.test_alg3_second_restatement,
    tg.test_signed_lexicographic_key_order,
    tg.test_topk_vs_full_sort_with_ties,
    tg.test_min_max_vs_numpy,
    tg.test_min_max_hand_worked_and_empty,
    tg.test_topk_by_max_with_ties,
    lambda: tj.test_nested_loop_tiny_with_duplicates(0),
    tj.test_hand_worked_example,
    tj.test_cardinality_identity_and_paper_algorithms,
    tj.test_join_group_topk_invariants,
    tj.test_semi_anti_vs_nested_loop_and_numpy,
    tj.test_left_outer_vs_nested_loop_and_identities,
    ts.test_like_hand_worked,
    lambda: ts.test_like_vs_regex_random(1),
    ts.test_in_strings_and_numbers,
    ts.test_mixed_plan_vs_row_loop,
]


def _build_mutant(tmp_path, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not unique/present: {old!r}"
    d = tmp_path / "m"
    d.mkdir()
    shutil.copy(HDR, d / "oracle.h")
    (d / "oracle.c").write_text(src.replace(old, new))
    so = d / "liboracle_mut.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", str(so), str(d / "oracle.c"), "-lm"])
    return oracle.load_variant(str(so))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path, monkeypatch):
    old, new = MUTANTS[name]
    mut = _build_mutant(tmp_path, old, new)
    monkeypatch.setattr(oracle, "_LIB", mut)
    caught = 0
    for pin in PINS:
        try:
            pin()
        except (AssertionError, oracle.OracleError, ValueError, IndexError):
            caught += 1
    assert caught > 0, f"no pin caught mutant {name}"


def test_unmutated_oracle_passes_all_pins():
    for pin in PINS:
        pin()
