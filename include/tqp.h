/*
 * tqp.h -- C ABI of libtqp, a GB300 (sm_103a) library of columnar relational
 * operators: the data-parallel hot path of a tensor query processor
 * ("Query Processing on Tensor Computation Runtimes", VLDB 2022).
 *
 * Data model (paper Section 4.1): a table is a set of equally long columns,
 * one dense array per column, rows identified by position ("virtual ids").
 * Numeric columns (int32, int64, uint8) and string columns (n x m bytes, for
 * IN / LIKE predicates).  Decimals are int64 fixed point (value x 10^scale) so
 * every sum is an exact integer; dates are int32 day numbers.
 *
 * Conventions for every entry point
 *   - Pointers named d_* and every column's `data` are DEVICE pointers on the
 *     context's device; the structs themselves (tqp_table, tqp_pred, ...) are
 *     HOST memory read during the call only.
 *   - The caller owns all inputs and outputs.  The library owns only the
 *     context's scratch arena (hash tables, scan status words, partials),
 *     which is either caller-provided device memory or allocated once at
 *     context creation.
 *   - Calls are asynchronous and stream-ordered on `stream` (a cudaStream_t;
 *     NULL = legacy default stream).  Result counts are written to device
 *     memory: no hidden host synchronisation (contrast the size-syncing
 *     nonzero/masked_select of the paper's Section 6.5).
 *   - The return value reports argument/launch errors found on the host.
 *     Errors found on the device (output capacity exceeded, a bounded wait
 *     that expired) are latched in the context and returned, then cleared,
 *     by tqp_ctx_check().
 *   - Column data must be 16-byte aligned (as from cudaMalloc / torch); this
 *     lets the scans stage tiles with bulk asynchronous copies.
 *   - One exception to device-resident columns: tqp_filter accepts a column
 *     in pinned (page-locked) host memory when the filter reads it only at
 *     passing rows -- a column that appears in sum_expr but in no predicate
 *     while at least one predicate remains after lowering.  The GPU then
 *     reads those rows in place over the host link (late materialisation of
 *     a projected column); any other use of host memory is rejected with
 *     TQP_ERR_INVALID_ARG.
 *   - A context serialises its scratch use: two calls on one context must not
 *     overlap on the device (same stream, or ordered streams).  Use one
 *     context per concurrent stream.
 *   - Functions never abort or throw; tqp_last_error() gives the message of
 *     the last failing call on this host thread.
 */
#ifndef TQP_H
#define TQP_H

#ifndef __CUDACC_RTC__
#include <stddef.h>
#include <stdint.h>
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define TQP_VERSION 100 /* 1.0.0 */

#if defined(__GNUC__)
#define TQP_API __attribute__((visibility("default")))
#else
#define TQP_API
#endif

typedef enum {
    TQP_OK = 0,
    TQP_ERR_INVALID_ARG = 1,   /* bad pointer, size, index, enum or alignment */
    TQP_ERR_UNSUPPORTED = 2,   /* valid request outside what the kernels implement */
    TQP_ERR_OUT_OF_MEMORY = 3, /* scratch arena too small (message says how much is needed) */
    TQP_ERR_CAPACITY = 4,      /* an output or hash table was too small; counts still exact */
    TQP_ERR_OVERFLOW = 5,      /* reserved: never returned (see the expression note below) */
    TQP_ERR_TIMEOUT = 6,       /* a bounded device-side wait expired; results are invalid */
    TQP_ERR_CUDA = 7           /* a CUDA runtime call failed (message has the CUDA error) */
} tqp_status;

typedef enum { TQP_I32 = 0, TQP_I64 = 1, TQP_U8 = 2, TQP_CHAR = 3 } tqp_dtype;

/* One column: device pointer (or, for tqp_filter, see the conventions above)
 * to num_rows elements of `type`; `scale` is the
 * decimal exponent of a fixed-point column (informational; arithmetic is on
 * the stored integers).
 * String columns (paper Section 4.1: an (n x m) tensor of character codes, a
 * string right-padded with 0s to the column's width m): type TQP_CHAR, `scale`
 * = m in [1, 255], `data` = num_rows * m bytes, row i's string at
 * [i*m, (i+1)*m) -- its bytes up to the first 0.  A string column is read by
 * TQP_IN, TQP_LIKE and TQP_NOT_LIKE predicates only (a comparison, an
 * expression, a group key or a join key on it is TQP_ERR_INVALID_ARG). */
typedef struct {
    const void* data;
    int32_t type;
    int32_t scale;
} tqp_column;

typedef struct {
    int64_t num_rows;         /* < 2^31 (row ids are int32) */
    int32_t num_cols;
    int32_t reserved;
    const tqp_column* cols;   /* host array of num_cols columns */
} tqp_table;

/* Comparison predicates (paper Section 3.1 / 5.1); a list of predicates is
 * their conjunction.  Comparisons are on the column value widened to int64.
 * BETWEEN is inclusive: lo <= x <= hi. */
typedef enum { TQP_LT = 0, TQP_LE, TQP_GT, TQP_GE, TQP_EQ, TQP_NE, TQP_BETWEEN, TQP_IN, TQP_LIKE, TQP_NOT_LIKE } tqp_cmp;

/* Set membership and pattern predicates (paper Section 5's IN and LIKE):
 *   TQP_IN        lo = host address of the values, hi = their count: int64
 *                 values for a numeric column, hi strings of the column's width
 *                 (each right-padded with 0, hi * m bytes) for a string column;
 *   TQP_LIKE, TQP_NOT_LIKE (string columns only): lo = host address of the
 *                 pattern's bytes, hi = its length (at most 255); `%` matches
 *                 any sequence of characters (also none), `_` exactly one,
 *                 every other byte itself; there is no escape character.
 * The host memory is read during the call only.  tqp_filter,
 * tqp_groupby_agg and tqp_run_plan (fact predicates) evaluate them in one
 * pre-pass over the columns involved (a warp stages 32 strings in shared
 * memory, each lane matches its row) that writes a one-byte pass column to
 * the context's arena; the scan then filters on it.  The values and patterns
 * of one call take at most TQP_MAX_SET_BYTES bytes (IN values sorted and
 * deduplicated: 8 per number, m per string), else TQP_ERR_UNSUPPORTED.
 * tqp_filter_noalloc returns TQP_ERR_UNSUPPORTED for them; tqp_filter_shared
 * runs such queries alone; batches hand such plans to the single-plan path. */
#define TQP_MAX_SET_BYTES 24576

typedef struct {
    int32_t col;   /* column index in the table */
    int32_t op;    /* tqp_cmp */
    int64_t lo;    /* operand (lower bound for BETWEEN) */
    int64_t hi;    /* upper bound for BETWEEN, ignored otherwise */
} tqp_pred;

#define TQP_MAX_PREDS 8
#define TQP_MAX_EXPR 8
#define TQP_MAX_GROUP_COLS 4
#define TQP_MAX_AGGS 8
#define TQP_MAX_COLS 16

/* Arithmetic expressions (paper Section 5.1: post-order traversal of the
 * expression tree): a postfix program of at most 8 tokens over int64, stack
 * depth at most 4.  TQP_X_COL pushes column v (for plans: fact columns first,
 * then dimension columns), TQP_X_CONST pushes v, ADD/SUB/MUL pop b then a and
 * push a op b.  Results must not overflow int64: past that precondition the
 * library does not detect overflow; its sums, counts and products wrap
 * modulo 2^64 (two's complement), so a SUM is then the exact sum reduced
 * modulo 2^64 (an AVG of it is meaningless). */
typedef enum { TQP_X_COL = 0, TQP_X_CONST, TQP_X_ADD, TQP_X_SUB, TQP_X_MUL } tqp_xop;

typedef struct {
    int32_t n;
    int32_t op[TQP_MAX_EXPR];
    int64_t v[TQP_MAX_EXPR];
} tqp_expr;

/* Aggregates (paper Section 5.4, Algorithm 3): SUM(expr) and COUNT(*) are
 * exact int64; AVG(expr) is the IEEE double division SUM/COUNT.  MIN(expr)
 * and MAX(expr) are the smallest / largest int64 value over the group's rows
 * (an ungrouped MIN/MAX over no rows gives 0 with NaN in d_fvals as its
 * flag).  MIN and MAX are supported everywhere an aggregate is (group-bys,
 * plans with or without a join, top-k by a MIN/MAX value): few-group shapes
 * take the direct kernel, larger ones the sort-based group-by, joined plans
 * the fused probe's general path (an atomic maximum of an order-preserving
 * code per accumulator). */
typedef enum { TQP_SUM = 0, TQP_COUNT, TQP_AVG, TQP_MIN, TQP_MAX } tqp_aggfn;

typedef struct {
    int32_t fn;      /* tqp_aggfn */
    int32_t reserved;
    tqp_expr expr;   /* ignored for COUNT */
} tqp_agg;

typedef struct tqp_ctx tqp_ctx;

/* ---- context ------------------------------------------------------------ */

/* Create a context on CUDA device `device`.  If d_arena is non-NULL it is a
 * caller-owned device buffer of arena_bytes used as scratch (the library
 * allocates nothing); if NULL the library cudaMallocs arena_bytes once and
 * frees it in tqp_ctx_destroy.  *out receives the context. */
TQP_API tqp_status tqp_ctx_create(int device, void* d_arena, size_t arena_bytes, tqp_ctx** out);
TQP_API tqp_status tqp_ctx_destroy(tqp_ctx* ctx);

/* Synchronise `stream`, then return (and clear) the first device-side error
 * latched by calls on this context since the last check. */
TQP_API tqp_status tqp_ctx_check(tqp_ctx* ctx, void* stream);

/* Iteration cap of every device-side spin wait issued by calls on this
 * context (default 1<<22 polls with back-off, well under a second).  After
 * the cap a wait gives up and latches TQP_ERR_TIMEOUT. */
TQP_API tqp_status tqp_ctx_set_wait_limit(tqp_ctx* ctx, int64_t polls);

/* Scratch bytes of the context's arena. */
TQP_API size_t tqp_ctx_arena_bytes(const tqp_ctx* ctx);

/* Override the scan launch shape used by this context's calls: rows per
 * tile (a multiple of 1024, at most 8192), pipeline stages (2..4) and CTAs
 * per SM (1..2).  All zero restores the built-in choice.  Used by the
 * autotuner and by tuning sweeps; results never depend on it. */
TQP_API tqp_status tqp_ctx_set_tuning(tqp_ctx* ctx, int32_t tile_rows, int32_t stages, int32_t ctas_per_sm);

/* Force the algorithm of operators that have two, for this context's calls
 * (results never depend on it):
 *   tqp_hash_join / tqp_hash_join_kind: 0 = the open-addressing hash table
 *     (paper Section 5.3's hash join), 1 = the sort-based join (Section 5.2,
 *     Algorithm 1: the build keys are radix-sorted with their rows and each
 *     probe key is bucketized into them);
 *   grouped join plans with at least 2^20 fact rows: 0 = the radix-partitioned
 *     aggregation (the probe side partitioned by group, each partition
 *     aggregated in shared memory), 1 = the fused probe (every joined row
 *     added to its key's or group's accumulators with L2 reductions).
 * -1 restores the default (0, or the autotuner's choice, which times both).
 * Errors: TQP_ERR_INVALID_ARG. */
TQP_API tqp_status tqp_ctx_set_variant(tqp_ctx* ctx, int32_t variant);

/* Run-time specialisation (a query-compiler step beside the paper's
 * compilation of queries into tensor programs, Section 4): the few-groups
 * aggregate of tqp_groupby_agg (sums and counts) is compiled with NVRTC for
 * the call's shape -- column types of its conditions, keys and sum factors,
 * the factors' affine forms -- so that the kernel's per-row dispatch on them
 * folds into constants.  mode 0: never; 1 (default): a shape is compiled
 * for an input of at least 16,777,216 rows, and once compiled (or found in the
 * disk cache) it serves inputs of any size; 2: compiled for every input.  A
 * shape compiles once per process (a few seconds, on the calling thread) and
 * its cubin is kept on disk (directory $TQP_JIT_CACHE, else _jit_cache/ beside
 * libtqp.so).  Where
 * NVRTC or the kernel sources are missing, or a compile fails, the generic
 * kernel runs; results are identical either way.  Errors: TQP_ERR_INVALID_ARG. */
TQP_API tqp_status tqp_ctx_set_jit(tqp_ctx* ctx, int32_t mode);

/* Process-wide counters (out: 4 int64): kernels compiled, kernels loaded from
 * the disk cache, specialised launches, failed compiles or loads. */
TQP_API void tqp_jit_stats(int64_t* out);

/* Checks that run-time specialisation works on this machine without a GPU:
 * NVRTC and the kernel sources are found and a sample shape compiles (or is
 * in the disk cache).  TQP_OK, else TQP_ERR_UNSUPPORTED with the reason (and
 * the compiler log) in tqp_last_error(). */
TQP_API tqp_status tqp_jit_probe(void);

/* Autotuning: with it on, the first call of each shape class (operator, log2
 * of the row count, bytes per row it scans, output kinds) times every
 * candidate launch shape -- rows per tile 1024..8192, 2..4 stages, 1..2 CTAs
 * per SM, for joins that build a hash table the load factor (capacity x1 or
 * x2), and for grouped join plans the algorithm (tqp_ctx_set_variant) -- on
 * the call's stream, synchronously, and keeps the fastest for
 * later calls of the class; tqp_batch_create likewise picks the batch's tile
 * size.  Results never depend on the choice.  A tqp_ctx_set_tuning override
 * takes precedence.  The choices can be saved to and loaded from a JSON file
 * (one entry per line: key, tile_rows, stages, ctas_per_sm, ht_scale,
 * variant, ms). */
TQP_API tqp_status tqp_ctx_set_autotune(tqp_ctx* ctx, int32_t enable);
TQP_API int32_t tqp_ctx_tuned_count(const tqp_ctx* ctx);
TQP_API tqp_status tqp_ctx_save_tuning(const tqp_ctx* ctx, const char* path);
TQP_API tqp_status tqp_ctx_load_tuning(tqp_ctx* ctx, const char* path);

TQP_API const char* tqp_last_error(void);
TQP_API const char* tqp_status_string(tqp_status s);
TQP_API int tqp_version(void);

/* ---- operators ---------------------------------------------------------- */

/*
 * tqp_filter -- predicate evaluation with stream compaction and an optional
 * fused projection-sum (paper Section 3.1, Listing 1 and the selection-vector
 * form; expressions Section 5.1).
 *
 *   d_row_ids[0..k)  ascending int32 ids of the rows where every predicate
 *                    holds (may be NULL: count and sum only); at most
 *                    `capacity` ids are written.
 *   *d_count         k, the exact number of passing rows (device int64).
 *   *d_sum           SUM(sum_expr) over passing rows (device int64); both
 *                    sum_expr and d_sum NULL to skip.
 *
 * k > capacity latches TQP_ERR_CAPACITY (ids beyond capacity are dropped;
 * *d_count stays exact).  npreds may be 0 (every row passes).
 */
TQP_API tqp_status tqp_filter(tqp_ctx* ctx, const tqp_table* t,
                      const tqp_pred* preds, int32_t npreds,
                      const tqp_expr* sum_expr, int64_t* d_sum,
                      int32_t* d_row_ids, int64_t capacity, int64_t* d_count,
                      void* stream);

/*
 * tqp_groupby_agg -- hash group-by aggregation over the rows passing `preds`
 * (paper Section 5.4, Algorithm 3 semantics: one output row per distinct key
 * tuple, keys in ascending lexicographic order of the int64-widened values).
 *
 *   group_cols[0..ngc)  key column indices, 0 <= ngc <= 4; the key tuple's
 *                       total width (8 bits per uint8, 32 per int32, 64 per
 *                       int64 column) must be <= 64 bits.  ngc == 0 gives a
 *                       single ungrouped output row (COUNT 0 / AVG NaN if no
 *                       row passes).
 *   d_keys   [G][ngc]   int64 key values, row-major        (may be NULL)
 *   d_ivals  [G][naggs] SUM -> sum, COUNT -> count, AVG -> sum
 *   d_fvals  [G][naggs] AVG -> (double)sum/(double)count, others 0.0
 *                       (may be NULL when no AVG is requested)
 *   *d_num_groups       G (device int64)
 *
 * capacity_groups bounds G and sizes the internal hash table; more groups
 * latch TQP_ERR_CAPACITY and set *d_num_groups to -1.
 */
TQP_API tqp_status tqp_groupby_agg(tqp_ctx* ctx, const tqp_table* t,
                           const tqp_pred* preds, int32_t npreds,
                           const int32_t* group_cols, int32_t ngc,
                           const tqp_agg* aggs, int32_t naggs,
                           int64_t* d_keys, int64_t* d_ivals, double* d_fvals,
                           int64_t capacity_groups, int64_t* d_num_groups,
                           void* stream);

/*
 * tqp_hash_join -- inner equi-join build.key = probe.key returning index
 * pairs (late materialisation, paper Sections 5.2-5.3; Algorithm 2's
 * semantics, computed with an open-addressing table instead of collision
 * rounds).  Keys must be int32 or int64 columns.
 *
 *   (d_build_idx[i], d_probe_idx[i])  the i-th matching pair, in canonical
 *                       order: probe index ascending, then build index
 *                       ascending; at most `capacity` pairs are written.
 *   *d_count            exact number of pairs (device int64); more than
 *                       capacity latches TQP_ERR_CAPACITY.
 * Duplicate keys are allowed on both sides.
 */
TQP_API tqp_status tqp_hash_join(tqp_ctx* ctx,
                         const tqp_table* build, int32_t build_key,
                         const tqp_table* probe, int32_t probe_key,
                         int32_t* d_build_idx, int32_t* d_probe_idx,
                         int64_t capacity, int64_t* d_count, void* stream);

/*
 * Join kinds (paper Section 5 lists left-semi, left-anti and left-outer joins
 * among the supported operators; the probe side is the left side):
 *   TQP_JOIN_INNER       every (build, probe) pair with equal keys
 *   TQP_JOIN_LEFT_SEMI   each probe row with at least one equal build key, once
 *   TQP_JOIN_LEFT_ANTI   each probe row with no equal build key, once
 *   TQP_JOIN_LEFT_OUTER  the inner pairs, and each probe row with no equal
 *                        build key once, paired with build row -1
 */
typedef enum { TQP_JOIN_INNER = 0, TQP_JOIN_LEFT_SEMI = 1, TQP_JOIN_LEFT_ANTI = 2, TQP_JOIN_LEFT_OUTER = 3 } tqp_join_kind;

/*
 * tqp_hash_join_kind -- tqp_hash_join for any tqp_join_kind, with the same
 * arguments, order and errors.  Semi and anti joins report each kept probe row
 * once with d_build_idx -1; left outer reports -1 for probe rows without a
 * match.  join_kind TQP_JOIN_INNER is tqp_hash_join.
 */
TQP_API tqp_status tqp_hash_join_kind(tqp_ctx* ctx,
                              const tqp_table* build, int32_t build_key,
                              const tqp_table* probe, int32_t probe_key, int32_t join_kind,
                              int32_t* d_build_idx, int32_t* d_probe_idx,
                              int64_t capacity, int64_t* d_count, void* stream);

/*
 * tqp_filter_noalloc -- tqp_filter for callers that cannot allocate device
 * memory.  (The paper has no counterpart; this is a deployment entry point.)
 *
 * Some callers run where cudaMalloc is off limits: inside a stream capture
 * that must not allocate, in a process whose device memory is owned by
 * another allocator, or in a real-time path that may not touch the memory
 * manager.  They cannot create a context (its arena is allocated memory).
 * This call needs no context: its scratch is one file-scope device array of
 * TQP_NOALLOC_SCRATCH_BYTES bytes inside libtqp, which every GPU that loads
 * the library holds until the process exits.  The caller still provides all
 * inputs and outputs; the call itself never calls cudaMalloc, cudaFree or
 * any allocating routine.
 *
 *   device       the CUDA device the pointers live on.
 *   t, preds, npreds, sum_expr, d_sum, d_row_ids, capacity, d_count
 *                exactly as for tqp_filter; t->num_rows must not exceed
 *                TQP_NOALLOC_MAX_ROWS (larger tables: TQP_ERR_INVALID_ARG,
 *                nothing is launched).
 *   d_status     device int32 receiving the device-side status of this call
 *                (TQP_OK, or e.g. TQP_ERR_CAPACITY); may be NULL.
 *
 * The first call on a device looks up the array's device address (once per
 * device); make that first call before any stream capture.  All calls share
 * the one array and each call overwrites it: calls that overlap on the GPU
 * (different streams, or concurrent host threads without ordering) race and
 * give wrong results -- order them on one stream.
 */
#define TQP_NOALLOC_MAX_ROWS (1LL << 24)
#define TQP_NOALLOC_SCRATCH_BYTES (2228224)
TQP_API tqp_status tqp_filter_noalloc(int device, const tqp_table* t,
                                      const tqp_pred* preds, int32_t npreds,
                                      const tqp_expr* sum_expr, int64_t* d_sum,
                                      int32_t* d_row_ids, int64_t capacity, int64_t* d_count,
                                      int32_t* d_status, void* stream);

/* ---- shared scans --------------------------------------------------------- */

/*
 * Many filter queries over one table in shared passes.  The paper runs one
 * query at a time (Section 4.3), so n queries over a resident table read it n
 * times; here one scan evaluates up to 32 queries: every row is tested
 * against all of them, and each query gets what tqp_filter without row ids
 * gives it (Section 3.1 filter, Section 5.1 expressions):
 *   d_count   passing rows (required)
 *   d_sum     SUM(sum_expr) over the passing rows (exactly when has_sum != 0)
 * Results are identical to n calls of tqp_filter(ctx, t, preds, npreds,
 * has_sum ? &sum_expr : NULL, d_sum, NULL, 0, d_count).
 *
 * Packing: queries are packed, in order and first fit, into launches of at
 * most 32 queries, 8 distinct columns and 2 distinct sum expressions whose
 * lookup tables fit the kernel's shared memory (per condition column one
 * table of the value intervals cut by the queries' range bounds and by their
 * TQP_IN values, each value v the interval [v, v+1)).  A query whose sum
 * expression is not a product of two affine factors (x, x*k, x+k, x*y,
 * x*(k-y), ...), that reads more than 8 columns, or that has a predicate on a
 * string column, runs alone through tqp_filter's scan (with its pre-pass),
 * and so does every query of a launch that would hold
 * fewer than 3 queries (that scan reads the summed columns only at passing
 * rows, which is faster for one or two queries).  launch_of (host array of
 * nq, may be NULL) receives each query's launch index, or -1 for one that ran
 * alone.
 *
 * Errors: TQP_ERR_INVALID_ARG (nq < 0, NULL queries with nq > 0, a NULL
 * d_count, has_sum without d_sum or d_sum without has_sum, a predicate or
 * expression tqp_filter rejects; nothing is launched), TQP_ERR_UNSUPPORTED
 * (IN values over TQP_MAX_SET_BYTES, as tqp_filter; nothing is launched),
 * TQP_ERR_OUT_OF_MEMORY
 * (the context's arena), TQP_ERR_CUDA.  Column rules as for tqp_filter's
 * predicate columns: every column a query reads must be in device memory.
 * Each launch carries its lookup tables in its kernel parameters; the call
 * copies nothing from host memory and does not synchronise the stream.
 */
typedef struct {
    tqp_pred preds[TQP_MAX_PREDS];
    int32_t npreds;
    int32_t has_sum;
    tqp_expr sum_expr;
    int64_t* d_count;
    int64_t* d_sum;
} tqp_scan_query;

TQP_API tqp_status tqp_filter_shared(tqp_ctx* ctx, const tqp_table* t, const tqp_scan_query* queries, int32_t nq,
                                     int32_t* launch_of, void* stream);

/* ---- fixed operator plans ------------------------------------------------ */

/*
 * A fixed query plan (the executor of paper Section 4.2.5 runs a plan's
 * operators in topological order; this is one fixed shape of such a plan):
 *
 *   scan(fact) -> filter(preds) -> [hash join fact.fact_fk = dim.dim_key]
 *     -> [SUM(sum_expr)] -> [GROUP BY group_cols: aggs] -> [top-k]
 *
 * Column indices in group_cols and in expressions address fact columns
 * 0..F-1 and then dim columns F..F+D-1.  With an inner join, each passing
 * fact row contributes once per matching dim row.  With join_kind
 * TQP_JOIN_LEFT_SEMI / TQP_JOIN_LEFT_ANTI each passing fact row contributes
 * once if it has a matching dim row / has none; group columns and
 * expressions then address fact columns only (a dim column is
 * TQP_ERR_INVALID_ARG), and d_num_joined counts the kept fact rows.  Left
 * outer joins are for tqp_hash_join_kind only (TQP_ERR_UNSUPPORTED here).
 * topk > 0 keeps the k groups with the largest aggregate `topk_agg` (ties:
 * smaller key first), in that order.
 */
typedef struct {
    const tqp_table* fact;
    tqp_pred preds[TQP_MAX_PREDS];
    int32_t npreds;
    int32_t emit_row_ids;       /* write passing fact row ids (ascending) */
    const tqp_table* dim;       /* NULL: no join */
    int32_t fact_fk;
    int32_t dim_key;
    int32_t group_cols[TQP_MAX_GROUP_COLS];
    int32_t ngc;
    int32_t naggs;
    tqp_agg aggs[TQP_MAX_AGGS];
    int32_t has_sum;            /* ungrouped SUM(sum_expr) over joined rows */
    int32_t topk;               /* 0 = all groups in key order */
    tqp_expr sum_expr;
    int32_t topk_agg;
    int32_t join_kind;          /* tqp_join_kind: TQP_JOIN_INNER (0), LEFT_SEMI or LEFT_ANTI */
    int64_t max_groups;         /* bound on distinct groups, sizes the aggregation
                                   table; 0 = the dim row count when grouping by
                                   dim columns, else res->capacity_groups */
    const struct tqp_dim* prepared; /* NULL, or `dim` prepared by tqp_dim_prepare with
                                   this plan's dim_key and group columns: the join
                                   then reuses its resident hash table */
} tqp_plan;

typedef struct {
    int32_t* d_row_ids;        int64_t capacity_rows;   int64_t* d_num_rows;   /* passing fact rows */
    int64_t* d_sum;                                                          /* ungrouped sum */
    int64_t* d_keys;           int64_t* d_ivals;        double* d_fvals;
    int64_t capacity_groups;   int64_t* d_num_groups;   int64_t* d_total_groups;
    int64_t* d_num_joined;                                                   /* joined rows */
} tqp_result;

/* A dimension table prepared once for many joined plans (resident build
 * side).  tqp_dim_prepare builds the chained hash table of `dim` on key_col
 * (direct-mapped when the keys span at most twice the row count, else
 * hashed) and the dense group id of every dim row for group_cols (dim column
 * indices, at most TQP_MAX_GROUP_COLS; ngc = 0: one group), and keeps them in a
 * long-lived region at the top of the context's arena until tqp_dim_destroy
 * (regions are freed newest first; all of them once no batch, server or
 * prepared dimension is left); plans on any context of the same device may
 * use it while the preparing context lives.  max_groups bounds the distinct groups (0: the
 * row count).  It synchronizes `stream` (setup, not a hot-path call).  The
 * dim table's device columns must stay valid and unchanged while plans use
 * the prepared form.  A plan uses it by setting plan.prepared; plan.dim,
 * plan.dim_key and the plan's group columns (as F + group_cols[i]) must match
 * (else TQP_ERR_INVALID_ARG).  Errors: TQP_ERR_INVALID_ARG, TQP_ERR_CAPACITY
 * (more groups than max_groups), TQP_ERR_OUT_OF_MEMORY (arena too small). */
typedef struct tqp_dim tqp_dim;
TQP_API tqp_status tqp_dim_prepare(tqp_ctx* ctx, const tqp_table* dim, int32_t key_col, const int32_t* group_cols,
                                   int32_t ngc, int64_t max_groups, void* stream, tqp_dim** out);
/* Number of groups of a prepared dimension (host value). */
TQP_API int64_t tqp_dim_groups(const tqp_dim* d);
TQP_API tqp_status tqp_dim_destroy(tqp_dim* d);

/* Run one plan.  All outputs are device pointers (any may be NULL when the
 * plan does not produce it); capacity rules as in the operator calls.
 *   d_num_rows    passing fact rows (before the join)
 *   d_num_joined  joined rows (= passing fact rows without a join)
 *   d_total_groups all groups (d_num_groups is min(topk, groups) with top-k)
 * With a join, group columns must all be dim columns and every expression
 * must use fact columns only (else TQP_ERR_UNSUPPORTED); without a join every
 * column is a fact column. */
TQP_API tqp_status tqp_run_plan(tqp_ctx* ctx, const tqp_plan* plan, const tqp_result* res, void* stream);

/* Run n independent plans as one batch.  The paper runs one query at a time
 * with intra-operator parallelism (Section 4.3); here each phase of all plans
 * is one kernel launch, and the scans of every plan are chunks that ONE
 * persistent launch of the staged scan engine drains from a shared ticket
 * counter, so small plans do not each pay a launch and a ramp-up.  Results
 * (every output of every tqp_result) are identical to n calls of
 * tqp_run_plan; plans whose group table needs the multi-kernel sort (more than
 * 4096 table slots without top-k) run through the tqp_run_plan path after the
 * batched kernels.  A malformed plan fails the call with its tqp_run_plan
 * error (plans before it may already have been launched).
 * Scratch comes from the context's arena (stream-ordered, like every call):
 * the job descriptors are copied with cudaMemcpyAsync on `stream`. */
TQP_API tqp_status tqp_run_plans(tqp_ctx* ctx, const tqp_plan* plans, const tqp_result* res, int32_t n, void* stream);

/* A batch lowered once and replayed: tqp_batch_create lowers n plans as
 * tqp_run_plans does, takes their scratch from a long-lived region at the top
 * of the context's arena (released by tqp_batch_destroy; the region of the
 * most recently created live batch is released first, all regions once no
 * batch is left) and captures every kernel into a CUDA graph; tqp_batch_run
 * launches that graph on `stream` (one launch per run).  The plans, tables
 * and result structs are read during create only; the device buffers they
 * point to must stay valid, and are re-read on every run, until destroy.
 * Runs of one batch must not overlap one another (they share scratch).
 * Errors: TQP_ERR_INVALID_ARG (NULL or n < 0), TQP_ERR_OUT_OF_MEMORY (arena
 * too small for the long-lived region), any error tqp_run_plan would report
 * for one of the plans.  tqp_batch_destroy synchronizes the device first. */
typedef struct tqp_batch tqp_batch;
TQP_API tqp_status tqp_batch_create(tqp_ctx* ctx, const tqp_plan* plans, const tqp_result* res, int32_t n,
                                    tqp_batch** out);
TQP_API tqp_status tqp_batch_run(tqp_batch* batch, void* stream);
TQP_API tqp_status tqp_batch_destroy(tqp_batch* batch);

/* ---- serving ------------------------------------------------------------ */

/* A server runs submitted plans with continuous batching (the paper runs one
 * query at a time, Section 4.3): a host dispatcher thread takes pending plans
 * in arrival order into free in-flight slots as one batch each (the batched
 * executor of tqp_run_plans), while earlier batches are still on the device.
 * Each slot has its own stream and its own share of a scratch budget taken
 * from a long-lived region of the context's arena: a batch is admitted only
 * if its scratch (hash tables, selection masks, group tables) fits the share
 * (an oversized batch is split).  A single plan that does not fit its share
 * is admitted by the device's free memory: when cudaMemGetInfo shows room for
 * its scratch with 1 GiB to spare, it runs in a region taken from the
 * stream-ordered allocator on the slot's stream (released there when it
 * retires); otherwise it completes with TQP_ERR_OUT_OF_MEMORY.  Results are
 * identical to tqp_run_plan of each plan alone.
 *   max_batch     plans per batch (1 = one query at a time)
 *   max_inflight  batches on the device at once (1..8)
 *   budget_bytes  scratch for all in-flight batches together
 * The context must not be used for other calls while the server lives. */
typedef struct {
    int32_t max_batch;
    int32_t max_inflight;
    int64_t budget_bytes;
} tqp_server_config;

/* One finished request: its tag, status, the size of the batch it ran in,
 * and host-clock seconds from submission to launch and to completion (seen
 * by the dispatcher polling the batch's event). */
typedef struct {
    uint64_t tag;
    int32_t status;
    int32_t batch_size;
    double queue_s;
    double latency_s;
} tqp_completion;

typedef struct tqp_server tqp_server;
TQP_API tqp_status tqp_server_create(tqp_ctx* ctx, const tqp_server_config* cfg, tqp_server** out);
/* Queue a plan (copied; its tables, prepared dimension and result buffers
 * must stay valid until the request completes).  Thread-safe. */
TQP_API tqp_status tqp_server_submit(tqp_server* s, const tqp_plan* plan, const tqp_result* res, uint64_t tag);
/* Move up to max finished requests into out[]; returns how many (>= 0), or
 * -1 if s or out is NULL.  Thread-safe. */
TQP_API int32_t tqp_server_poll(tqp_server* s, tqp_completion* out, int32_t max);
/* Wait until every submitted request has finished (TQP_ERR_TIMEOUT after
 * timeout_s seconds). */
TQP_API tqp_status tqp_server_drain(tqp_server* s, double timeout_s);
/* Stop the dispatcher after the queued work and release the region. */
TQP_API tqp_status tqp_server_destroy(tqp_server* s);

/* ---- measurement --------------------------------------------------------- */

/*
 * tqp_measure_scan_rate -- the ceiling of the staged scans on given columns.
 * (The paper has no counterpart: a measurement entry point.)  Streams every
 * column of t (at most 8, numeric, device memory) through the staged scan
 * engine with the launch shape tile_rows x stages at ctas_per_sm CTAs per SM,
 * with a body that only reads each staged 16-byte word once (their checksum
 * is added to *d_out, caller-owned device memory).  Time the call with events
 * on `stream`; bytes moved = rows x the columns' element sizes.  Errors:
 * TQP_ERR_INVALID_ARG (shape outside tqp_ctx_set_tuning's ranges, more than 8
 * or string columns, host columns), TQP_ERR_UNSUPPORTED (the shape does not
 * fit shared memory), TQP_ERR_CUDA.
 */
TQP_API tqp_status tqp_measure_scan_rate(tqp_ctx* ctx, const tqp_table* t, int32_t tile_rows, int32_t stages,
                                         int32_t ctas_per_sm, unsigned long long* d_out, void* stream);

/*
 * tqp_measure_l2_red -- the reduction-rate roofline of the joined
 * aggregation.  (The paper has no counterpart: a measurement entry point.)
 * Launches blocks_per_sm x (number of SMs) blocks of `threads` threads on
 * `stream`; row i (0 <= i < rows) picks a uniformly random key k in
 * [0, table_words / adds_per_row) and adds 1 to d_table[k * adds_per_row]
 * and i to each of the following adds_per_row - 1 words, with
 * fire-and-forget 8-byte reductions (the accumulator updates of the joined
 * aggregation).  d_table: caller-owned device memory of table_words uint64
 * words (contents change).  Time the call with events on `stream`.
 * Errors: TQP_ERR_INVALID_ARG (adds_per_row outside 1..8, table smaller
 * than one entry, threads not a multiple of 32 in 32..1024, blocks_per_sm
 * outside 1..32), TQP_ERR_CUDA.
 */
TQP_API tqp_status tqp_measure_l2_red(int device, unsigned long long* d_table, int64_t table_words, int64_t rows,
                                      int32_t adds_per_row, int32_t blocks_per_sm, int32_t threads, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* TQP_H */
