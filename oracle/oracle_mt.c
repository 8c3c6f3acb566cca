/*
 * Row-range parallel driver of the oracle's filter step -- TEST / TIMING
 * INFRASTRUCTURE ONLY (the benchmark's all-core CPU baseline).
 *
 * The fact rows are cut into `nthreads` contiguous ranges.  Each range is
 * evaluated by oracle_plan itself -- the same row-at-a-time predicate and
 * expression code -- on its own thread, over column pointers offset to the
 * range start.  The per-range results are then joined in range order: row
 * ids shifted by the range start and concatenated (so they stay ascending),
 * counts and int64 sums added with overflow checks.  The result is the one
 * oracle_plan gives for the whole table.  Only filter plans (no join, no
 * grouping) are accepted: oracle_plan's grouping sort keeps process-wide
 * state and is not run concurrently.
 */
#include "oracle.h"

#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define OR_MT_MAX_THREADS 256
#define OR_MT_MAX_COLS 64

typedef struct {
    or_plan plan;                 /* the range's plan (columns offset) */
    or_col cols[OR_MT_MAX_COLS];
    or_out out;
    int64_t row0;
    int status;
} or_range;

static void* run_range(void* arg) {
    or_range* r = (or_range*)arg;
    r->status = oracle_plan(&r->plan, &r->out);
    return NULL;
}

static int elem_bytes(int32_t type) { return type == OR_I64 ? 8 : (type == OR_I32 ? 4 : 1); }

int oracle_filter_mt(const or_plan* p, or_out* o, int nthreads) {
    if (!p || !o || p->nfact < 0 || p->ndim_cols != 0 || p->ngc != 0 || p->naggs != 0 ||
        p->nfact_cols < 1 || p->nfact_cols > OR_MT_MAX_COLS)
        return OR_ERR_INVALID;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > OR_MT_MAX_THREADS) nthreads = OR_MT_MAX_THREADS;
    if ((int64_t)nthreads > p->nfact) nthreads = p->nfact > 0 ? (int)p->nfact : 1;
    or_range* R = (or_range*)calloc((size_t)nthreads, sizeof(or_range));
    pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!R || !th) { free(R); free(th); return OR_ERR_NOMEM; }
    int status = OR_OK;
    int started = 0;
    for (int t = 0; t < nthreads; ++t) {
        const int64_t r0 = p->nfact * t / nthreads, r1 = p->nfact * (t + 1) / nthreads;
        or_range* r = &R[t];
        r->plan = *p;
        r->plan.nfact = r1 - r0;
        for (int c = 0; c < p->nfact_cols; ++c) {
            r->cols[c] = p->fact[c];
            r->cols[c].data = (const char*)p->fact[c].data +
                              (size_t)r0 * (size_t)(p->fact[c].type == OR_CHAR ? p->fact[c].width
                                                                                 : elem_bytes(p->fact[c].type));
        }
        r->plan.fact = r->cols;
        r->row0 = r0;
        if (o->row_ids) {
            r->out.row_ids = (int32_t*)malloc(sizeof(int32_t) * (size_t)(r1 - r0 > 0 ? r1 - r0 : 1));
            if (!r->out.row_ids) { status = OR_ERR_NOMEM; break; }
            r->out.cap_rows = r1 - r0;
        }
        if (pthread_create(&th[t], NULL, run_range, r) != 0) {
            free(r->out.row_ids);
            r->out.row_ids = NULL;
            status = OR_ERR_NOMEM;
            break;
        }
        ++started;
    }
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    int64_t n = 0, sum = 0;
    for (int t = 0; t < started && status == OR_OK; ++t) {
        const or_range* r = &R[t];
        if (r->status != OR_OK) { status = r->status; break; }
        if (o->row_ids) {
            for (int64_t i = 0; i < r->out.num_rows; ++i, ++n)
                if (n < o->cap_rows) o->row_ids[n] = (int32_t)(r->out.row_ids[i] + r->row0);
        } else {
            n += r->out.num_rows;
        }
        if (__builtin_add_overflow(sum, r->out.sum, &sum)) status = OR_ERR_OVERFLOW;
    }
    for (int t = 0; t < nthreads; ++t) free(R[t].out.row_ids);
    free(R);
    free(th);
    if (status != OR_OK) return status;
    o->num_rows = n;
    o->sum = sum;
    if (o->row_ids && n > o->cap_rows) return OR_ERR_CAPACITY;
    return OR_OK;
}
