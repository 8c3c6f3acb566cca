/*
 * CPU oracle for the tensor-query-processor hot path -- TEST INFRASTRUCTURE.
 *
 * Plain, slow, row-at-a-time C.  Only tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code with the CUDA
 * library.  Each step restates the operator's definition from the paper:
 *
 *   filter            Section 3.1 (Listing 1 / selection vector): keep row i
 *                     iff every predicate holds; output row ids ascending.
 *                     String columns (Section 4.1: a row's characters, one
 *                     per byte, right-padded with 0) take IN and LIKE / NOT
 *                     LIKE (Section 5's expression list); IN also applies to
 *                     numeric columns.
 *   expressions       Section 5.1: post-order evaluation of an expression
 *                     tree, here given in postfix form, in exact int64.
 *   equi-join         Sections 5.2-5.3 (Algorithms 1 and 2): the multiset of
 *                     index pairs (fact row, dim row) with equal keys (late
 *                     materialisation); emitted in (fact row, dim row) order.
 *                     Left semi / anti join (a join kind the paper lists as
 *                     supported, Section 5): each surviving fact row once,
 *                     when it has at least one / no equal-key dim row.
 *                     Left outer join (also listed there): the inner pairs,
 *                     and each surviving fact row with no equal-key dim row
 *                     once, paired with dim row -1 (no dim columns are read).
 *   group-by          Section 5.4 (Algorithm 3): sort rows by the group-key
 *                     tuple, cut the sorted list into runs of equal keys
 *                     ("unique consecutive"), evaluate the aggregates per run;
 *                     groups come out in ascending key order.
 *   top-k             the sort operator of Section 5: groups ordered by one
 *                     aggregate descending, ties by key ascending, first k.
 *
 * Arithmetic is int64 with overflow checks (decimals are x100 fixed point);
 * AVG is (double)SUM / (double)COUNT, one IEEE round-to-nearest division;
 * MIN and MAX are the smallest and largest value of the expression over the
 * group's rows (the ungrouped aggregate over no rows reports 0 with the
 * floating-point value NaN as its flag, like AVG).
 * Not thread-safe: one call at a time per process.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAX_GC 4

static int64_t col_value(const or_col* c, int64_t row) {
    switch (c->type) {
        case OR_I32: return (int64_t)((const int32_t*)c->data)[row];
        case OR_I64: return ((const int64_t*)c->data)[row];
        case OR_U8: return (int64_t)((const uint8_t*)c->data)[row];
        default: return 0;
    }
}

/* The row's string: its bytes up to the first 0, at most `width`. */
static int str_len(const uint8_t* s, int width) {
    int n = 0;
    while (n < width && s[n]) ++n;
    return n;
}

/* SQL LIKE by dynamic programming over prefixes: after reading i characters,
 * ok[j] says whether the pattern's first j bytes match them. */
static int like_match(const uint8_t* s, int n, const uint8_t* pat, int m) {
    unsigned char ok[OR_MAX_WIDTH + 1], nx[OR_MAX_WIDTH + 1];
    ok[0] = 1;
    for (int j = 1; j <= m; ++j) ok[j] = ok[j - 1] && pat[j - 1] == '%';
    for (int i = 0; i < n; ++i) {
        nx[0] = 0;
        for (int j = 1; j <= m; ++j) {
            if (pat[j - 1] == '%') nx[j] = nx[j - 1] || ok[j];  /* % takes nothing more, or s[i] too */
            else nx[j] = ok[j - 1] && (pat[j - 1] == '_' || pat[j - 1] == s[i]);
        }
        memcpy(ok, nx, (size_t)m + 1);
    }
    return ok[m];
}

static int is_set_op(int op) { return op == OR_IN || op == OR_LIKE || op == OR_NOT_LIKE; }

/* IN, LIKE and NOT LIKE at row `row` of column c (plain scans of the lists). */
static int set_pred_holds(const or_pred* p, const or_col* c, int64_t row) {
    if (c->type == OR_CHAR) {
        const uint8_t* s = (const uint8_t*)c->data + row * (int64_t)c->width;
        if (p->op == OR_IN) {
            const uint8_t* v = (const uint8_t*)(intptr_t)p->lo;
            for (int64_t k = 0; k < p->hi; ++k)
                if (memcmp(s, v + k * (int64_t)c->width, (size_t)c->width) == 0) return 1;
            return 0;
        }
        const int m = like_match(s, str_len(s, c->width), (const uint8_t*)(intptr_t)p->lo, (int)p->hi);
        return p->op == OR_LIKE ? m : !m;
    }
    const int64_t x = col_value(c, row);
    const int64_t* v = (const int64_t*)(intptr_t)p->lo;
    for (int64_t k = 0; k < p->hi; ++k)
        if (v[k] == x) return 1;
    return 0;
}

static int pred_holds(const or_pred* p, int64_t x) {
    switch (p->op) {
        case OR_LT: return x < p->lo;
        case OR_LE: return x <= p->lo;
        case OR_GT: return x > p->lo;
        case OR_GE: return x >= p->lo;
        case OR_EQ: return x == p->lo;
        case OR_NE: return x != p->lo;
        case OR_BETWEEN: return x >= p->lo && x <= p->hi;
        default: return 0;
    }
}

/* A joined row: fact row f and dim row d (d < 0 when there is no join). */
typedef struct { int64_t f; int64_t d; } or_pair;

/* Value of concatenated column `c` (fact columns first, then dim columns). */
static int64_t pair_value(const or_plan* p, int32_t c, const or_pair* r) {
    if (c < p->nfact_cols) return col_value(&p->fact[c], r->f);
    return col_value(&p->dim[c - p->nfact_cols], r->d);
}

/* Postfix evaluation in int64; returns 0 on success, 1 on overflow/invalid. */
static int expr_eval(const or_plan* p, const or_expr* e, const or_pair* r, int64_t* out) {
    int64_t st[OR_MAX_EXPR];
    int sp = 0;
    for (int i = 0; i < e->n; ++i) {
        int k = e->kind[i];
        if (k == OR_X_COL || k == OR_X_CONST) {
            if (sp >= OR_MAX_EXPR) return 1;
            st[sp++] = (k == OR_X_COL) ? pair_value(p, (int32_t)e->v[i], r) : e->v[i];
        } else {
            if (sp < 2) return 1;
            int64_t b = st[--sp], a = st[--sp], c;
            int ovf;
            if (k == OR_X_ADD) ovf = __builtin_add_overflow(a, b, &c);
            else if (k == OR_X_SUB) ovf = __builtin_sub_overflow(a, b, &c);
            else if (k == OR_X_MUL) ovf = __builtin_mul_overflow(a, b, &c);
            else return 1;
            if (ovf) return 1;
            st[sp++] = c;
        }
    }
    if (sp != 1) return 1;
    *out = st[0];
    return 0;
}

/* ---- join helpers: dim rows sorted by (key, row) ---- */
typedef struct { int64_t key; int64_t row; } or_keyrow;

static int cmp_keyrow(const void* a, const void* b) {
    const or_keyrow* x = (const or_keyrow*)a;
    const or_keyrow* y = (const or_keyrow*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->row != y->row) return x->row < y->row ? -1 : 1;
    return 0;
}

/* first index in sorted[0..n) whose key >= k */
static int64_t lower_bound(const or_keyrow* s, int64_t n, int64_t k) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (s[mid].key < k) lo = mid + 1; else hi = mid;
    }
    return lo;
}

/* ---- group-by records: key tuple + joined-row index ---- */
typedef struct { int64_t key[OR_MAX_GC]; int64_t idx; } or_grec;
static int g_ngc; /* number of key columns compared by cmp_grec (single-threaded) */

static int cmp_keys(const int64_t* a, const int64_t* b, int n) {
    for (int i = 0; i < n; ++i)
        if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
    return 0;
}

static int cmp_grec(const void* a, const void* b) {
    const or_grec* x = (const or_grec*)a;
    const or_grec* y = (const or_grec*)b;
    int c = cmp_keys(x->key, y->key, g_ngc);
    if (c) return c;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

/* ---- top-k records ---- */
typedef struct { int64_t rank_val; int64_t key[OR_MAX_GC]; int64_t g; } or_trec;

static int cmp_trec(const void* a, const void* b) {
    const or_trec* x = (const or_trec*)a;
    const or_trec* y = (const or_trec*)b;
    if (x->rank_val != y->rank_val) return x->rank_val > y->rank_val ? -1 : 1; /* descending */
    return cmp_keys(x->key, y->key, g_ngc);                                   /* then key asc */
}

static int valid_col(const or_col* c) {
    return c->type == OR_I32 || c->type == OR_I64 || c->type == OR_U8 ||
           (c->type == OR_CHAR && c->width >= 1 && c->width <= OR_MAX_WIDTH);
}

/* a numeric column (strings are read by IN / LIKE predicates only) */
static int numeric_col(const or_plan* p, int32_t c) {
    if (c < p->nfact_cols) return p->fact[c].type != OR_CHAR;
    return c - p->nfact_cols < p->ndim_cols && p->dim[c - p->nfact_cols].type != OR_CHAR;
}

static int numeric_expr(const or_plan* p, const or_expr* e) {
    for (int i = 0; i < e->n; ++i)
        if (e->kind[i] == OR_X_COL && !numeric_col(p, (int32_t)e->v[i])) return 0;
    return 1;
}

/* every column operand of the expression must address an existing column */
static int valid_expr(const or_expr* e, int ncat) {
    if (e->n < 1 || e->n > OR_MAX_EXPR) return 0;
    for (int i = 0; i < e->n; ++i)
        if (e->kind[i] == OR_X_COL && (e->v[i] < 0 || e->v[i] >= ncat)) return 0;
    return 1;
}

int oracle_plan(const or_plan* p, or_out* o) {
    if (!p || !o || p->nfact < 0 || p->npreds < 0 || p->ngc < 0 || p->ngc > OR_MAX_GC || p->naggs < 0)
        return OR_ERR_INVALID;
    for (int i = 0; i < p->nfact_cols; ++i)
        if (!valid_col(&p->fact[i])) return OR_ERR_INVALID;
    for (int i = 0; i < p->npreds; ++i) {
        const or_pred* q = &p->preds[i];
        if (q->col < 0 || q->col >= p->nfact_cols) return OR_ERR_INVALID;
        const int str = p->fact[q->col].type == OR_CHAR;
        if (q->op < OR_LT || q->op > OR_NOT_LIKE) return OR_ERR_INVALID;
        if (str && q->op != OR_IN && q->op != OR_LIKE && q->op != OR_NOT_LIKE) return OR_ERR_INVALID;
        if (!str && (q->op == OR_LIKE || q->op == OR_NOT_LIKE)) return OR_ERR_INVALID;
        if (is_set_op(q->op) && (q->hi < 0 || (q->hi > 0 && q->lo == 0))) return OR_ERR_INVALID;
        if ((q->op == OR_LIKE || q->op == OR_NOT_LIKE) && q->hi > OR_MAX_WIDTH) return OR_ERR_INVALID;
    }
    int joined = p->ndim_cols > 0;
    int ncat = p->nfact_cols + (joined ? p->ndim_cols : 0);
    for (int i = 0; i < p->ngc; ++i)
        if (p->group_cols[i] < 0 || p->group_cols[i] >= ncat) return OR_ERR_INVALID;
    for (int i = 0; i < p->ndim_cols && joined; ++i)
        if (!valid_col(&p->dim[i])) return OR_ERR_INVALID;
    for (int a = 0; a < p->naggs; ++a) {
        if (p->aggs[a].fn < OR_SUM || p->aggs[a].fn > OR_MAX) return OR_ERR_INVALID;
        if (p->aggs[a].fn != OR_COUNT && !valid_expr(&p->aggs[a].expr, ncat)) return OR_ERR_INVALID;
    }
    if (p->sum_expr && !valid_expr(p->sum_expr, ncat)) return OR_ERR_INVALID;
    /* string columns feed IN / LIKE predicates only */
    for (int i = 0; i < p->ngc; ++i)
        if (!numeric_col(p, p->group_cols[i])) return OR_ERR_INVALID;
    for (int a = 0; a < p->naggs; ++a)
        if (p->aggs[a].fn != OR_COUNT && !numeric_expr(p, &p->aggs[a].expr)) return OR_ERR_INVALID;
    if (p->sum_expr && !numeric_expr(p, p->sum_expr)) return OR_ERR_INVALID;
    if (joined && p->fact_fk >= 0 && p->fact_fk < p->nfact_cols && p->dim_key >= 0 && p->dim_key < p->ndim_cols &&
        (p->fact[p->fact_fk].type == OR_CHAR || p->dim[p->dim_key].type == OR_CHAR))
        return OR_ERR_INVALID;
    if (joined && (p->join_kind < OR_JOIN_INNER || p->join_kind > OR_JOIN_LEFT_OUTER)) return OR_ERR_INVALID;
    if (joined && p->join_kind != OR_JOIN_INNER) {  /* no dim row to read: fact columns only */
        for (int i = 0; i < p->ngc; ++i)
            if (p->group_cols[i] >= p->nfact_cols) return OR_ERR_INVALID;
        for (int a = 0; a < p->naggs; ++a)
            if (p->aggs[a].fn != OR_COUNT && !valid_expr(&p->aggs[a].expr, p->nfact_cols)) return OR_ERR_INVALID;
        if (p->sum_expr && !valid_expr(p->sum_expr, p->nfact_cols)) return OR_ERR_INVALID;
    }
    int status = OR_OK;

    /* 1. filter: ascending surviving fact rows */
    int64_t* surv = (int64_t*)malloc(sizeof(int64_t) * (size_t)(p->nfact > 0 ? p->nfact : 1));
    if (!surv) return OR_ERR_NOMEM;
    int64_t ns = 0;
    for (int64_t i = 0; i < p->nfact; ++i) {
        int keep = 1;
        for (int j = 0; j < p->npreds && keep; ++j) {
            const or_pred* q = &p->preds[j];
            keep = is_set_op(q->op) ? set_pred_holds(q, &p->fact[q->col], i)
                                    : pred_holds(q, col_value(&p->fact[q->col], i));
        }
        if (keep) surv[ns++] = i;
    }
    o->num_rows = ns;
    if (o->row_ids) {
        for (int64_t i = 0; i < ns && i < o->cap_rows; ++i) o->row_ids[i] = (int32_t)surv[i];
        if (ns > o->cap_rows) status = OR_ERR_CAPACITY;
    }

    /* 2. equi-join: for each surviving fact row, every dim row with an equal key */
    or_pair* pairs = NULL;
    int64_t npairs = 0;
    if (joined) {
        if (p->fact_fk < 0 || p->fact_fk >= p->nfact_cols || p->dim_key < 0 || p->dim_key >= p->ndim_cols) {
            free(surv);
            return OR_ERR_INVALID;
        }
        or_keyrow* sd = (or_keyrow*)malloc(sizeof(or_keyrow) * (size_t)(p->ndim > 0 ? p->ndim : 1));
        int64_t cap = ns > 16 ? ns : 16;
        pairs = (or_pair*)malloc(sizeof(or_pair) * (size_t)cap);
        if (!sd || !pairs) { free(sd); free(pairs); free(surv); return OR_ERR_NOMEM; }
        for (int64_t d = 0; d < p->ndim; ++d) {
            sd[d].key = col_value(&p->dim[p->dim_key], d);
            sd[d].row = d;
        }
        qsort(sd, (size_t)p->ndim, sizeof(or_keyrow), cmp_keyrow);
        for (int64_t i = 0; i < ns; ++i) {
            int64_t k = col_value(&p->fact[p->fact_fk], surv[i]);
            if (p->join_kind == OR_JOIN_SEMI || p->join_kind == OR_JOIN_ANTI) {  /* the fact row once, or not at all */
                const int64_t j0 = lower_bound(sd, p->ndim, k);
                const int has = j0 < p->ndim && sd[j0].key == k;
                if (has == (p->join_kind == OR_JOIN_SEMI)) {
                    pairs[npairs].f = surv[i];  /* at most ns <= cap pairs: no growth */
                    pairs[npairs].d = -1;
                    ++npairs;
                }
                continue;
            }
            const int64_t before = npairs;
            for (int64_t j = lower_bound(sd, p->ndim, k); j < p->ndim && sd[j].key == k; ++j) {
                if (npairs == cap) {
                    cap *= 2;
                    or_pair* np2 = (or_pair*)realloc(pairs, sizeof(or_pair) * (size_t)cap);
                    if (!np2) { free(sd); free(pairs); free(surv); return OR_ERR_NOMEM; }
                    pairs = np2;
                }
                pairs[npairs].f = surv[i];
                pairs[npairs].d = sd[j].row;
                ++npairs;
            }
            if (p->join_kind == OR_JOIN_LEFT_OUTER && npairs == before) {  /* no match: the fact row once */
                if (npairs == cap) {
                    cap *= 2;
                    or_pair* np2 = (or_pair*)realloc(pairs, sizeof(or_pair) * (size_t)cap);
                    if (!np2) { free(sd); free(pairs); free(surv); return OR_ERR_NOMEM; }
                    pairs = np2;
                }
                pairs[npairs].f = surv[i];
                pairs[npairs].d = -1;
                ++npairs;
            }
        }
        free(sd);
    } else {
        pairs = (or_pair*)malloc(sizeof(or_pair) * (size_t)(ns > 0 ? ns : 1));
        if (!pairs) { free(surv); return OR_ERR_NOMEM; }
        for (int64_t i = 0; i < ns; ++i) { pairs[i].f = surv[i]; pairs[i].d = -1; }
        npairs = ns;
    }
    free(surv);
    o->num_pairs = npairs;
    if (o->pair_fact || o->pair_dim) {
        for (int64_t i = 0; i < npairs && i < o->cap_pairs; ++i) {
            if (o->pair_fact) o->pair_fact[i] = (int32_t)pairs[i].f;
            if (o->pair_dim) o->pair_dim[i] = (int32_t)pairs[i].d;
        }
        if (npairs > o->cap_pairs) status = OR_ERR_CAPACITY;
    }

    /* 3. ungrouped SUM(expr) over the joined rows */
    o->sum = 0;
    if (p->sum_expr) {
        for (int64_t i = 0; i < npairs; ++i) {
            int64_t v;
            if (expr_eval(p, p->sum_expr, &pairs[i], &v) || __builtin_add_overflow(o->sum, v, &o->sum)) {
                free(pairs);
                return OR_ERR_OVERFLOW;
            }
        }
    }

    /* 4. group-by aggregation (Algorithm 3 order: sort, runs of equal keys, evaluate) */
    o->num_groups = 0;
    o->total_groups = 0;
    if (p->ngc > 0 || p->naggs > 0) {
        int64_t nrec = npairs;
        or_grec* rec = (or_grec*)malloc(sizeof(or_grec) * (size_t)(nrec > 0 ? nrec : 1));
        if (!rec) { free(pairs); return OR_ERR_NOMEM; }
        for (int64_t i = 0; i < nrec; ++i) {
            memset(rec[i].key, 0, sizeof(rec[i].key));
            for (int c = 0; c < p->ngc; ++c) rec[i].key[c] = pair_value(p, p->group_cols[c], &pairs[i]);
            rec[i].idx = i;
        }
        g_ngc = p->ngc;
        qsort(rec, (size_t)nrec, sizeof(or_grec), cmp_grec);

        /* number of groups: runs of equal keys; with no key columns exactly one group */
        int64_t ngroups = 0;
        for (int64_t i = 0; i < nrec; ++i)
            if (i == 0 || cmp_keys(rec[i].key, rec[i - 1].key, p->ngc) != 0) ++ngroups;
        if (p->ngc == 0) ngroups = 1;

        int na = p->naggs;
        int64_t* gkeys = (int64_t*)calloc((size_t)(ngroups > 0 ? ngroups : 1) * OR_MAX_GC, sizeof(int64_t));
        int64_t* gsum = (int64_t*)calloc((size_t)(ngroups > 0 ? ngroups : 1) * (size_t)(na > 0 ? na : 1), sizeof(int64_t));
        int64_t* gcnt = (int64_t*)calloc((size_t)(ngroups > 0 ? ngroups : 1), sizeof(int64_t));
        if (!gkeys || !gsum || !gcnt) {
            free(gkeys); free(gsum); free(gcnt); free(rec); free(pairs);
            return OR_ERR_NOMEM;
        }
        int64_t g = -1;
        for (int64_t i = 0; i < nrec; ++i) {
            if (p->ngc == 0) g = 0;
            else if (i == 0 || cmp_keys(rec[i].key, rec[i - 1].key, p->ngc) != 0) {
                ++g;
                memcpy(&gkeys[g * OR_MAX_GC], rec[i].key, sizeof(rec[i].key));
            }
            gcnt[g] += 1;
            const or_pair* r = &pairs[rec[i].idx];
            for (int a = 0; a < na; ++a) {
                const int fn = p->aggs[a].fn;
                if (fn == OR_COUNT) continue;
                int64_t v;
                if (expr_eval(p, &p->aggs[a].expr, r, &v)) {
                    free(gkeys); free(gsum); free(gcnt); free(rec); free(pairs);
                    return OR_ERR_OVERFLOW;
                }
                int64_t* acc = &gsum[g * na + a];
                if (fn == OR_MIN || fn == OR_MAX) {
                    /* the group's first row sets it, later rows replace it when smaller / larger */
                    if (gcnt[g] == 1 || (fn == OR_MIN ? v < *acc : v > *acc)) *acc = v;
                    continue;
                }
                if (__builtin_add_overflow(*acc, v, acc)) {
                    free(gkeys); free(gsum); free(gcnt); free(rec); free(pairs);
                    return OR_ERR_OVERFLOW;
                }
            }
        }
        free(rec);

        /* final per-group values: SUM / COUNT as int64, AVG as one IEEE division */
        int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ngroups > 0 ? ngroups : 1));
        if (!order) { free(gkeys); free(gsum); free(gcnt); free(pairs); return OR_ERR_NOMEM; }
        int64_t nout = ngroups;
        for (int64_t i = 0; i < ngroups; ++i) order[i] = i;

        /* 5. optional top-k by aggregate topk_agg descending, key ascending */
        if (p->topk > 0) {
            if (p->topk_agg < 0 || p->topk_agg >= na) {
                free(order); free(gkeys); free(gsum); free(gcnt); free(pairs);
                return OR_ERR_INVALID;
            }
            or_trec* t = (or_trec*)malloc(sizeof(or_trec) * (size_t)(ngroups > 0 ? ngroups : 1));
            if (!t) { free(order); free(gkeys); free(gsum); free(gcnt); free(pairs); return OR_ERR_NOMEM; }
            int ta = p->topk_agg;
            for (int64_t i = 0; i < ngroups; ++i) {
                t[i].rank_val = (p->aggs[ta].fn == OR_COUNT) ? gcnt[i] : gsum[i * na + ta];
                memcpy(t[i].key, &gkeys[i * OR_MAX_GC], sizeof(t[i].key));
                t[i].g = i;
            }
            g_ngc = p->ngc;
            qsort(t, (size_t)ngroups, sizeof(or_trec), cmp_trec);
            if (nout > p->topk) nout = p->topk;
            for (int64_t i = 0; i < nout; ++i) order[i] = t[i].g;
            free(t);
        }

        o->total_groups = ngroups;
        o->num_groups = nout;
        for (int64_t i = 0; i < nout && i < o->cap_groups; ++i) {
            int64_t gi = order[i];
            if (o->keys)
                for (int c = 0; c < p->ngc; ++c) o->keys[i * p->ngc + c] = gkeys[gi * OR_MAX_GC + c];
            for (int a = 0; a < na; ++a) {
                int fn = p->aggs[a].fn;
                int64_t iv = (fn == OR_COUNT) ? gcnt[gi] : gsum[gi * na + a];
                if (o->ivals) o->ivals[i * na + a] = iv;
                if (o->fvals) {
                    double f = 0.0;
                    if (fn == OR_AVG) f = (double)gsum[gi * na + a] / (double)gcnt[gi];
                    else if ((fn == OR_MIN || fn == OR_MAX) && gcnt[gi] == 0) f = NAN;
                    o->fvals[i * na + a] = f;
                }
            }
        }
        if (nout > o->cap_groups) status = OR_ERR_CAPACITY;
        free(order); free(gkeys); free(gsum); free(gcnt);
    }
    free(pairs);
    return status;
}
