// The autotuner: scan launch shapes (rows per tile, pipeline stages, CTAs
// per SM) and the hash-table load factor, chosen per shape class by timing.
//
// A shape class is a string an entry point derives from what decides the
// best launch shape -- the operator, log2 of the row count, the bytes per
// row it stages and similar.  With autotuning on, the first call of a class
// runs the whole operator once per candidate (warm-up + one timed run on the
// caller's stream, CUDA events, synchronous), keeps the fastest, and every
// later call of the class uses it.  Candidates differ only in launch shape,
// so every run writes the same outputs; the last run's outputs stand.
// Choices can be saved to and loaded from a small JSON file.
#include <cstdio>
#include <map>
#include <mutex>
#include <string>

#include "host.h"

namespace tqp {

int ht_scale(const tqp_ctx* ctx) {
    if (ctx->forced.tile_rows > 0) return ctx->forced.ht_scale > 1 ? 2 : 1;
    tqp_tuning t;
    if (ctx->tuner && ctx->cur_key[0] && ctx->tuner->lookup(ctx->cur_key, &t)) return t.ht_scale > 1 ? 2 : 1;
    return 1;
}

int tuned_variant(const tqp_ctx* ctx) {
    if (ctx->force_variant >= 0) return ctx->force_variant;
    if (ctx->forced.tile_rows > 0) return ctx->forced.variant;
    tqp_tuning t;
    if (ctx->tuner && ctx->cur_key[0] && ctx->tuner->lookup(ctx->cur_key, &t)) return t.variant;
    return 0;
}

int row_bytes(const tqp_table* t, std::vector<int> cols) {
    std::sort(cols.begin(), cols.end());
    cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
    int b = 0;
    for (int c : cols)
        if (c >= 0 && c < t->num_cols) b += t->cols[c].type == TQP_I64 ? 8 : (t->cols[c].type == TQP_I32 ? 4 : 1);
    return b;
}

void expr_col_ids(const tqp_expr* e, std::vector<int>& cols) {
    if (!e) return;
    for (int i = 0; i < e->n && i < TQP_MAX_EXPR; ++i)
        if (e->op[i] == TQP_X_COL) cols.push_back(static_cast<int>(e->v[i]));
}

int rows_class(long long n) {
    int k = 0;
    while ((2LL << k) <= n) ++k;
    return k;
}

namespace {

struct KeyScope {
    tqp_ctx* ctx;
    char saved[sizeof(tqp_ctx::cur_key)];
    KeyScope(tqp_ctx* c, const char* key) : ctx(c) {
        memcpy(saved, c->cur_key, sizeof(saved));
        snprintf(c->cur_key, sizeof(c->cur_key), "%s", key);
    }
    ~KeyScope() { memcpy(ctx->cur_key, saved, sizeof(saved)); }
};

}  // namespace

tqp_status tuned_call(tqp_ctx* ctx, const char* key, cudaStream_t stream, int opts, tqp_status (*run)(void*),
                      void* arg) {
    KeyScope ks(ctx, key);
    tqp_tuning known;
    if (!ctx->tuner || !ctx->tuner->enabled || ctx->forced.tile_rows > 0 || ctx->tuner->lookup(key, &known))
        return run(arg);
    cudaEvent_t ev[2] = {nullptr, nullptr};
    TQP_CUDA(cudaEventCreate(&ev[0]));
    TQP_CUDA(cudaEventCreate(&ev[1]));
    tqp_tuning best{0, 0, 0, 0, 0};
    double best_ms = 1e30;
    const int hts = (opts & kTuneHt) ? 2 : 1;
    const int nvar = (opts & kTuneVariant) ? 2 : 1;
    for (int V = nvar - 1; V >= 0; --V)
    for (int T = kRowQuantum; T <= kMaxTileRows; T *= 2)
        for (int S = 2; S <= kMaxStages; ++S)
            for (int C = 1; C <= 2; ++C)
                for (int H = 1; H <= hts; ++H) {
                    // variant 0 of a two-variant operator does not use the scan launch shape
                    const bool shapeless = ((opts & kTuneV0Shapeless) && V == 0) || ((opts & kTuneV1Shapeless) && V == 1);
                    if (shapeless && (T != kRowQuantum || S != 2 || C != 1)) continue;
                    ctx->forced = tqp_tuning{T, S, C, H, V};
                    if (run(arg) != TQP_OK) continue;  // infeasible (shared memory): refused on the host
                    cudaEventRecord(ev[0], stream);
                    const tqp_status s = run(arg);
                    cudaEventRecord(ev[1], stream);
                    if (s != TQP_OK || cudaEventSynchronize(ev[1]) != cudaSuccess) continue;
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, ev[0], ev[1]);
                    if (ms < best_ms) {
                        best_ms = ms;
                        best = ctx->forced;
                    }
                }
    ctx->forced = tqp_tuning{0, 0, 0, 0, 0};
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    clear_error();
    if (best.tile_rows == 0) return run(arg);  // no candidate ran: report the built-in shape's result
    {
        std::lock_guard<std::mutex> lk(ctx->tuner->mu);
        ctx->tuner->table[key] = best;
        ctx->tuner->ms[key] = best_ms;
    }
    return run(arg);  // the chosen shape, so that its outputs are the call's
}

void tuner_destroy(tqp_ctx* ctx) {
    delete ctx->tuner;
    ctx->tuner = nullptr;
}

}  // namespace tqp

using namespace tqp;

extern "C" {

tqp_status tqp_ctx_set_autotune(tqp_ctx* ctx, int32_t enable) {
    clear_error();
    TQP_TRY(check_ctx(ctx));
    if (!ctx->tuner) ctx->tuner = new (std::nothrow) Tuner();
    if (!ctx->tuner) return fail(TQP_ERR_OUT_OF_MEMORY, "host allocation failed");
    ctx->tuner->enabled = enable != 0;
    return TQP_OK;
}

int32_t tqp_ctx_tuned_count(const tqp_ctx* ctx) {
    if (!ctx || !ctx->tuner) return 0;
    std::lock_guard<std::mutex> lk(ctx->tuner->mu);
    return static_cast<int32_t>(ctx->tuner->table.size());
}

tqp_status tqp_ctx_save_tuning(const tqp_ctx* ctx, const char* path) {
    clear_error();
    TQP_TRY(check_ctx(ctx));
    if (!path) return fail(TQP_ERR_INVALID_ARG, "path is NULL");
    FILE* f = fopen(path, "w");
    if (!f) return fail(TQP_ERR_INVALID_ARG, "cannot write %s", path);
    fprintf(f, "{\"version\": 1, \"entries\": [");
    if (ctx->tuner) {
        std::lock_guard<std::mutex> lk(ctx->tuner->mu);
        bool first = true;
        for (const auto& e : ctx->tuner->table) {
            const double ms = ctx->tuner->ms.count(e.first) ? ctx->tuner->ms.at(e.first) : 0.0;
            fprintf(f, "%s\n  {\"key\": \"%s\", \"tile_rows\": %d, \"stages\": %d, \"ctas_per_sm\": %d, \"ht_scale\": %d, "
                       "\"variant\": %d, \"ms\": %.6f}",
                    first ? "" : ",", e.first.c_str(), e.second.tile_rows, e.second.stages, e.second.ctas_per_sm,
                    e.second.ht_scale, e.second.variant, ms);
            first = false;
        }
    }
    fprintf(f, "\n]}\n");
    const bool ok = fclose(f) == 0;
    return ok ? TQP_OK : fail(TQP_ERR_INVALID_ARG, "cannot write %s", path);
}

// Reads the file tqp_ctx_save_tuning writes (one entry per line).
tqp_status tqp_ctx_load_tuning(tqp_ctx* ctx, const char* path) {
    clear_error();
    TQP_TRY(check_ctx(ctx));
    if (!path) return fail(TQP_ERR_INVALID_ARG, "path is NULL");
    FILE* f = fopen(path, "r");
    if (!f) return fail(TQP_ERR_INVALID_ARG, "cannot read %s", path);
    if (!ctx->tuner) ctx->tuner = new (std::nothrow) Tuner();
    if (!ctx->tuner) {
        fclose(f);
        return fail(TQP_ERR_OUT_OF_MEMORY, "host allocation failed");
    }
    char line[512];
    int loaded = 0;
    while (fgets(line, sizeof(line), f)) {
        char key[sizeof(tqp_ctx::cur_key)];
        tqp_tuning t{0, 0, 0, 0, 0};
        double ms = 0;
        const bool with_variant =
            sscanf(line, " {\"key\": \"%95[^\"]\", \"tile_rows\": %d, \"stages\": %d, \"ctas_per_sm\": %d, \"ht_scale\": %d, "
                         "\"variant\": %d, \"ms\": %lf",
                   key, &t.tile_rows, &t.stages, &t.ctas_per_sm, &t.ht_scale, &t.variant, &ms) == 7;
        if (with_variant ||
            sscanf(line, " {\"key\": \"%95[^\"]\", \"tile_rows\": %d, \"stages\": %d, \"ctas_per_sm\": %d, \"ht_scale\": %d, "
                         "\"ms\": %lf",
                   key, &t.tile_rows, &t.stages, &t.ctas_per_sm, &t.ht_scale, &ms) == 6) {
            if (!with_variant) t.variant = 0;
            if (t.tile_rows < kRowQuantum || t.tile_rows > kMaxTileRows || t.tile_rows % kRowQuantum ||
                t.stages < 2 || t.stages > kMaxStages || t.ctas_per_sm < 1 || t.ctas_per_sm > 2 || t.variant < 0 ||
                t.variant > 1)
                continue;
            std::lock_guard<std::mutex> lk(ctx->tuner->mu);
            ctx->tuner->table[key] = t;
            ctx->tuner->ms[key] = ms;
            ++loaded;
        }
    }
    fclose(f);
    (void)loaded;
    return TQP_OK;
}

}  // extern "C"
