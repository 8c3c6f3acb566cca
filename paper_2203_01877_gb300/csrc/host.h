// Host-side internals shared by the libtqp translation units: the context,
// its scratch arena, error reporting and the lowering of API structs
// (predicates, expressions, tables) into kernel parameter blocks.
#pragma once

#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstddef>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "engine.cuh"

// Tile/launch choices for one scan; filled by the tuner (tune.cu).
struct tqp_tuning {
    int tile_rows;      // T, multiple of tqp::kRowQuantum
    int stages;         // 2..kMaxStages
    int ctas_per_sm;    // 0: as many as fit
    int ht_scale;       // hash-table capacity multiplier (1 or 2: half the load factor); 0 = 1
    int variant;        // algorithm variant of operators that have two (0 = the default)
};

namespace tqp {
// Autotuner state: the chosen launch shape (and its time) per shape class.
struct Tuner {
    bool enabled = false;
    std::mutex mu;
    std::map<std::string, tqp_tuning> table;
    std::map<std::string, double> ms;
    bool lookup(const char* key, tqp_tuning* out) {
        std::lock_guard<std::mutex> lk(mu);
        auto it = table.find(key);
        if (it == table.end()) return false;
        *out = it->second;
        return true;
    }
};
}  // namespace tqp

struct tqp_ctx {
    int device;
    int num_sms;
    int smem_optin;        // max dynamic shared memory per block (bytes)
    int l2_bytes;
    unsigned char* arena;  // device scratch
    size_t arena_bytes;
    bool owns_arena;
    size_t used;           // bump offset of the current call
    size_t top;            // start of the long-lived region (batches) at the arena's end
    int live_regions;      // long-lived regions (batches, prepared dimensions, servers)
    int* d_err;            // latched device error (persistent, arena start)
    long long wait_cap;
    tqp_tuning forced;     // tile_rows == 0: no override
    int force_variant;     // >= 0: algorithm variant forced by tqp_ctx_set_variant
    tqp::Tuner* tuner;     // autotuner state (owned by the context; shared by sub-contexts)
    int jit;               // run-time specialisation: 0 off, 1 inputs of kJitMinRows or more, 2 always
    char cur_key[96];      // shape class of the running call ("" outside tuned calls)
};

namespace tqp {

constexpr size_t kPersistentBytes = 256;   // arena prefix kept across calls (error word)
constexpr long long kDefaultWaitCap = 1LL << 22;

tqp_status fail(tqp_status s, const char* fmt, ...);
tqp_status cuda_fail(cudaError_t e, const char* what);
void clear_error();

#define TQP_CUDA(call)                                          \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return ::tqp::cuda_fail(e_, #call); \
    } while (0)

#define TQP_TRY(expr)                       \
    do {                                    \
        tqp_status s_ = (expr);             \
        if (s_ != TQP_OK) return s_;        \
    } while (0)

// Scratch arena: bump allocation, reset at the start of every API call.
void arena_reset(tqp_ctx* ctx);
// Returns nullptr (and records the shortfall) when the arena is exhausted.
void* arena_alloc(tqp_ctx* ctx, size_t bytes, size_t align = 256);
// Long-lived allocation from the arena's end (survives arena_reset; freed by
// moving ctx->top back, newest first).
void* arena_alloc_top(tqp_ctx* ctx, size_t bytes, size_t align = 256);
tqp_status arena_oom(tqp_ctx* ctx, size_t bytes);
// Long-lived regions at the arena's top (batches, prepared dimensions,
// servers): open one before its first arena_alloc_top, close it with the top
// offsets seen before and after its allocations.  Regions are freed newest
// first; once none is left the whole top is free again.
void top_open(tqp_ctx* ctx);
void top_close(tqp_ctx* ctx, size_t before, size_t after);
// Synchronize `stream` and return (and clear) the context's latched device error.
tqp_status take_device_error(tqp_ctx* ctx, cudaStream_t stream);

// Select the context's device for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev);
    ~DeviceGuard();
};

tqp_status check_ctx(const tqp_ctx* ctx);
tqp_status check_table(const tqp_table* t, const char* what);
tqp_status check_device_cols(const tqp_table* t, const std::vector<int>& cols, const char* what);
// Columns read in place at passing rows: device, managed or mapped page-locked host memory.
tqp_status check_visible_cols(const tqp_table* t, const std::vector<int>& cols, const char* what);

// Lower predicates to range conditions on `t`'s columns.
tqp_status lower_preds(const tqp_table* t, const tqp_pred* preds, int32_t npreds, Cond* out, int* ncond);
// Fast-path form of the conditions for geometry G; *fast is false when some
// condition column is not staged (the general path is used then).
void lower_fast(const Cond* conds, int ncond, const ScanGeom& G, CondFast* out, int32_t* fast);

// Lower a postfix expression whose column operands address `ncols` columns.
tqp_status lower_expr(const tqp_expr* e, int ncols, DExpr* out);
// Closed form of an expression whose columns are staged in G (see ProdForm);
// false when it is not a product of two affine factors or reads an unstaged
// column (the interpreter handles it then).
bool lower_prod(const DExpr& e, const ScanGeom& G, ProdForm* out);
// Column ids referenced by an expression.
void expr_cols(const DExpr& e, std::vector<int>& cols);

// Fill G for table t with the given staged columns (deduplicated, <= 8);
// columns beyond the table (dim columns of a plan) are appended by callers.
tqp_status make_geom(const tqp_ctx* ctx, const tqp_table* t, std::vector<int> staged, const tqp_tuning& tu,
                     int body_smem, ScanGeom* G, size_t* smem_bytes);

// Default tuning for a scan staging `bytes_per_row` bytes per row (the
// context's override, when set, wins).
tqp_tuning default_tuning(const tqp_ctx* ctx, int bytes_per_row, int body_smem);

// Hash-table capacity multiplier of the running call (forced or tuned; 1 by default).
int ht_scale(const tqp_ctx* ctx);
// Algorithm variant of the running call (forced or tuned; 0 by default).
int tuned_variant(const tqp_ctx* ctx);
// What a tuned call's candidates vary besides the scan launch shape.
constexpr int kTuneHt = 1;       // the hash-table load factor
constexpr int kTuneVariant = 2;  // the operator's algorithm variant (0 or 1)
constexpr int kTuneV0Shapeless = 4;  // variant 0 does not use the scan launch shape (time one of them)
constexpr int kTuneV1Shapeless = 8;  // variant 1 does not use the scan launch shape

// Run `run` (a whole operator call, idempotent) under the tuning of shape
// class `key`: with autotuning on and `key` new, every candidate launch shape
// (and hash-table load factor when `has_ht`) is timed on `stream` first and
// the fastest is remembered; the outputs are the same for every candidate.
tqp_status tuned_call(tqp_ctx* ctx, const char* key, cudaStream_t stream, int opts, tqp_status (*run)(void*),
                      void* arg);
template <class F>
tqp_status tuned(tqp_ctx* ctx, const char* key, cudaStream_t stream, int opts, F& f) {
    return tuned_call(ctx, key, stream, opts, [](void* a) { return (*static_cast<F*>(a))(); }, &f);
}
void tuner_destroy(tqp_ctx* ctx);
// Bytes per row of the distinct columns `cols` of t.
int row_bytes(const tqp_table* t, std::vector<int> cols);
// Columns an expression reads (expression may be NULL).
void expr_col_ids(const tqp_expr* e, std::vector<int>& cols);
// floor(log2(max(n, 1))): the row-count part of a shape class.
int rows_class(long long n);

// Persistent grid size for an engine kernel.
int engine_grid(const tqp_ctx* ctx, const void* kernel, size_t smem, int64_t ntiles, int ctas_per_sm);

constexpr int kMaxDevices = 64;
// Once-per-device flags of allow_smem: any host thread (a server's
// dispatcher, callers on other contexts, context-free callers) may reach it,
// so the flags are atomic.
struct SmemFlags {
    std::atomic<bool> done[kMaxDevices];
};
// Raise a kernel's dynamic shared-memory limit once per device.
tqp_status allow_smem(const tqp_ctx* ctx, const void* kernel, SmemFlags& flags);

// Stream-ordered store of a host value into device memory (a one-thread
// kernel: unlike a pageable memcpy it can be captured in a CUDA graph).
tqp_status set_device_i64(long long* d_ptr, long long value, cudaStream_t stream);

// IN / LIKE / NOT LIKE predicates and string columns (strings.cu): whether a
// predicate list needs the pre-pass, and the pre-pass itself.  With active
// set, `t` is the input table with one uint8 pass column appended (index
// t->num_cols, in the arena) and `preds` the numeric predicates plus
// "pass column == 1"; otherwise `t` and `preds` are the inputs.  `t.cols`
// points into `cols`: not copyable.
struct StrLowered {
    bool active = false;
    tqp_table t{};
    std::vector<tqp_column> cols;
    tqp_pred preds[TQP_MAX_PREDS];
    int32_t npreds = 0;
    StrLowered() = default;
    StrLowered(const StrLowered&) = delete;
    StrLowered& operator=(const StrLowered&) = delete;
};
bool has_set_preds(const tqp_table* t, const tqp_pred* preds, int32_t npreds);
// With check_only, only the host checks run: out->preds receives the other
// predicates and nothing is allocated or launched.
tqp_status str_prepass(tqp_ctx* ctx, const tqp_table* t, const tqp_pred* preds, int32_t npreds, cudaStream_t st,
                       StrLowered* out, bool check_only = false);
// Columns read by arithmetic, keys or comparisons must be numeric (a string
// column feeds IN / LIKE predicates only).
tqp_status check_numeric_cols(const tqp_table* t, const std::vector<int>& cols, const char* what);

// Run-time specialisation (jit.cu): the few-groups aggregate compiled for D's
// shape (sums only), or nullptr (the generic kernel then runs).  A shape is
// compiled for calls on at least kJitMinRows rows (every call in mode 2);
// once compiled, or found in the disk cache, it serves calls of any size.
constexpr long long kJitMinRows = 16LL << 20;
struct GroupDirectArgs;
const void* jit_group_direct(const tqp_ctx* ctx, const GroupDirectArgs& D, long long rows);
void jit_count_launch();

// The single-query filter scan (tqp_filter's body, in the caller's arena).
tqp_status launch_filter(tqp_ctx* ctx, const tqp_table* t, const tqp_pred* preds, int32_t npreds,
                         const tqp_expr* sum_expr, int64_t* d_sum, int32_t* d_row_ids, int64_t capacity,
                         int64_t* d_count, cudaStream_t stream, const tqp_tuning* force);

// One-shot batched run of n plans in ctx's per-call scratch on `stream` (the
// body of tqp_run_plans; the server calls it with a slot's sub-context).
tqp_status run_plans_on(tqp_ctx* ctx, const tqp_plan* plans, const tqp_result* res, int32_t n, cudaStream_t stream);

}  // namespace tqp
