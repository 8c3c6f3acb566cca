/*
 * CPU oracle for the tensor-query-processor hot path -- TEST INFRASTRUCTURE.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * call this code.  It shares nothing with the CUDA library (no header, no
 * helper, no table): it restates, row at a time, what the paper's relational
 * operators compute (Section 5: filter, expressions, hash/sort equi-join,
 * sort-based group-by aggregation) so that the GPU results can be checked
 * element by element.
 *
 * All arithmetic is exact int64 with overflow detection; AVG is the single
 * IEEE double division (double)SUM / (double)COUNT.
 */
#ifndef TQP_ORACLE_H
#define TQP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define OR_OK 0
#define OR_ERR_INVALID 1
#define OR_ERR_CAPACITY 4
#define OR_ERR_OVERFLOW 5
#define OR_ERR_NOMEM 6

/* column element types */
#define OR_I32 0
#define OR_I64 1
#define OR_U8 2
#define OR_CHAR 3   /* strings: `width` bytes per row, right-padded with 0 (paper Section 4.1) */
#define OR_MAX_WIDTH 255

/* comparison operators; BETWEEN is inclusive on both ends */
#define OR_LT 0
#define OR_LE 1
#define OR_GT 2
#define OR_GE 3
#define OR_EQ 4
#define OR_NE 5
#define OR_BETWEEN 6
/* set membership and pattern matching (paper Section 5 lists IN and LIKE):
 *   IN        lo = host address of the values, hi = their count; int64 values
 *             for a numeric column, `width`-byte 0-padded strings for a
 *             string column;
 *   LIKE, NOT LIKE (string columns only): lo = host address of the pattern
 *             bytes, hi = its length (at most OR_MAX_WIDTH); `%` matches any
 *             sequence (also none), `_` one character, any other byte itself;
 *             no escape character.  A row's string is its bytes up to the
 *             first 0 (or all `width` bytes). */
#define OR_IN 7
#define OR_LIKE 8
#define OR_NOT_LIKE 9

/* postfix expression opcodes */
#define OR_X_COL 0
#define OR_X_CONST 1
#define OR_X_ADD 2
#define OR_X_SUB 3
#define OR_X_MUL 4

/* join kinds: every equal-key (fact, dim) pair; or each fact row once if it
 * has a match (left semi) / has none (left anti), with dim row -1; or the
 * equal-key pairs plus each fact row without a match once with dim row -1
 * (left outer).  Every kind but inner reads fact columns only. */
#define OR_JOIN_INNER 0
#define OR_JOIN_SEMI 1
#define OR_JOIN_ANTI 2
#define OR_JOIN_LEFT_OUTER 3

/* aggregate functions */
#define OR_SUM 0
#define OR_COUNT 1
#define OR_AVG 2
#define OR_MIN 3
#define OR_MAX 4

#define OR_MAX_EXPR 8

typedef struct { const void* data; int32_t type; int32_t width; } or_col;  /* width: OR_CHAR only */
typedef struct { int32_t col; int32_t op; int64_t lo; int64_t hi; } or_pred;
typedef struct { int32_t n; int32_t kind[OR_MAX_EXPR]; int64_t v[OR_MAX_EXPR]; } or_expr;
typedef struct { int32_t fn; int32_t pad; or_expr expr; } or_agg;

/*
 * A query plan over a fact table and an optional dimension table:
 *   filter(fact, preds) -> [equi-join fact.fact_fk = dim.dim_key]
 *   -> [ungrouped SUM(sum_expr)] -> [GROUP BY group_cols: aggs] -> [top-k].
 * Column indices in group_cols and in expressions address the concatenation
 * (fact columns, then dim columns).  Predicates address fact columns only;
 * with a semi or anti join everything addresses fact columns only.
 */
typedef struct {
    int64_t nfact; const or_col* fact; int32_t nfact_cols; int32_t pad0;
    const or_pred* preds; int32_t npreds; int32_t pad1;
    int64_t ndim; const or_col* dim; int32_t ndim_cols;   /* ndim_cols == 0: no join */
    int32_t fact_fk; int32_t dim_key; int32_t join_kind;  /* OR_JOIN_INNER / _SEMI / _ANTI / _LEFT_OUTER */
    const int32_t* group_cols; int32_t ngc; int32_t pad3;
    const or_agg* aggs; int32_t naggs; int32_t pad4;
    const or_expr* sum_expr;                              /* NULL: no ungrouped sum */
    int32_t topk; int32_t topk_agg;                       /* topk == 0: keep all groups */
} or_plan;

typedef struct {
    int32_t* row_ids; int64_t cap_rows; int64_t num_rows;        /* surviving fact rows, ascending */
    int32_t* pair_fact; int32_t* pair_dim; int64_t cap_pairs; int64_t num_pairs;
    int64_t sum;
    int64_t* keys; int64_t* ivals; double* fvals; int64_t cap_groups;
    int64_t num_groups; int64_t total_groups;
} or_out;

int oracle_plan(const or_plan* plan, or_out* out);

/* The filter step (a plan without join or grouping) on `nthreads` threads:
 * oracle_plan over contiguous row ranges, results joined in range order --
 * identical to oracle_plan's (oracle_mt.c; timing of the CPU baseline). */
int oracle_filter_mt(const or_plan* plan, or_out* out, int nthreads);

#ifdef __cplusplus
}
#endif
#endif
