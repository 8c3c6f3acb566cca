// Context, scratch arena, error reporting and API-struct lowering.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>

#include "host.h"

namespace {
thread_local std::string g_last_error;
}

namespace tqp {

tqp_status fail(tqp_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

tqp_status cuda_fail(cudaError_t e, const char* what) {
    return fail(TQP_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

void clear_error() { g_last_error.clear(); }

DeviceGuard::DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    ok = (prev == dev) || (cudaSetDevice(dev) == cudaSuccess);
}
DeviceGuard::~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
}

void arena_reset(tqp_ctx* ctx) { ctx->used = kPersistentBytes; }

void* arena_alloc(tqp_ctx* ctx, size_t bytes, size_t align) {
    size_t off = (ctx->used + align - 1) / align * align;
    if (off + bytes > ctx->top) {
        ctx->used = off + bytes;  // remember the demand for the error message
        return nullptr;
    }
    ctx->used = off + bytes;
    return ctx->arena + off;
}

void* arena_alloc_top(tqp_ctx* ctx, size_t bytes, size_t align) {
    if (bytes > ctx->top) return nullptr;
    const size_t start = (ctx->top - bytes) / align * align;
    if (start < ctx->used || start < kPersistentBytes) return nullptr;
    ctx->top = start;
    return ctx->arena + start;
}

void top_open(tqp_ctx* ctx) { ++ctx->live_regions; }

void top_close(tqp_ctx* ctx, size_t before, size_t after) {
    if (--ctx->live_regions <= 0) {
        ctx->live_regions = 0;
        ctx->top = ctx->arena_bytes;
    } else if (ctx->top < before && ctx->top == after) {
        ctx->top = before;
    }
}

tqp_status take_device_error(tqp_ctx* ctx, cudaStream_t stream) {
    TQP_CUDA(cudaStreamSynchronize(stream));
    int err = 0;
    TQP_CUDA(cudaMemcpy(&err, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err != 0) {
        TQP_CUDA(cudaMemset(ctx->d_err, 0, sizeof(int)));
        return fail(static_cast<tqp_status>(err), "device reported: %s", tqp_status_string(static_cast<tqp_status>(err)));
    }
    return TQP_OK;
}

tqp_status arena_oom(tqp_ctx* ctx, size_t bytes) {
    return fail(TQP_ERR_OUT_OF_MEMORY, "scratch arena too small: need at least %zu bytes (arena holds %zu)",
                std::max(ctx->used, bytes), ctx->arena_bytes);
}

tqp_status check_ctx(const tqp_ctx* ctx) {
    if (!ctx) return fail(TQP_ERR_INVALID_ARG, "ctx is NULL");
    return TQP_OK;
}

tqp_status check_table(const tqp_table* t, const char* what) {
    if (!t) return fail(TQP_ERR_INVALID_ARG, "%s: table is NULL", what);
    if (t->num_rows < 0 || t->num_rows > INT32_MAX)
        return fail(TQP_ERR_INVALID_ARG, "%s: num_rows %lld outside [0, 2^31)", what, (long long)t->num_rows);
    if (t->num_cols < 1 || t->num_cols > TQP_MAX_COLS)
        return fail(TQP_ERR_INVALID_ARG, "%s: num_cols %d outside [1, %d]", what, t->num_cols, TQP_MAX_COLS);
    if (!t->cols) return fail(TQP_ERR_INVALID_ARG, "%s: cols is NULL", what);
    for (int c = 0; c < t->num_cols; ++c) {
        const tqp_column& col = t->cols[c];
        if (col.type != TQP_I32 && col.type != TQP_I64 && col.type != TQP_U8 && col.type != TQP_CHAR)
            return fail(TQP_ERR_INVALID_ARG, "%s: column %d has unknown type %d", what, c, col.type);
        if (col.type == TQP_CHAR && (col.scale < 1 || col.scale > 255))
            return fail(TQP_ERR_INVALID_ARG, "%s: string column %d has width %d outside [1, 255]", what, c, col.scale);
        if (t->num_rows > 0 && !col.data) return fail(TQP_ERR_INVALID_ARG, "%s: column %d data is NULL", what, c);
        if (reinterpret_cast<uintptr_t>(col.data) % 16 != 0)
            return fail(TQP_ERR_INVALID_ARG, "%s: column %d is not 16-byte aligned", what, c);
    }
    return TQP_OK;
}

tqp_status check_numeric_cols(const tqp_table* t, const std::vector<int>& cols, const char* what) {
    for (int c : cols)
        if (c >= 0 && c < t->num_cols && t->cols[c].type == TQP_CHAR)
            return fail(TQP_ERR_INVALID_ARG, "%s: string column %d is read by IN / LIKE predicates only", what, c);
    return TQP_OK;
}

// Columns `cols` of t must be device (or managed) memory: they are staged
// with bulk asynchronous copies.
tqp_status check_device_cols(const tqp_table* t, const std::vector<int>& cols, const char* what) {
    for (int c : cols) {
        if (c < 0 || c >= t->num_cols || !t->cols[c].data) continue;
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, t->cols[c].data) != cudaSuccess) {
            cudaGetLastError();
            return fail(TQP_ERR_INVALID_ARG, "%s: column %d is not CUDA-visible memory", what, c);
        }
        if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
            return fail(TQP_ERR_INVALID_ARG,
                        "%s: column %d is host memory; only columns read at passing rows may be", what, c);
    }
    return TQP_OK;
}

// Columns `cols` of t are read by the GPU in place (at passing rows only):
// device, managed or page-locked host memory that the device can address.
// Anything else (pageable host memory, a foreign pointer) is rejected here,
// before any launch could dereference it.
tqp_status check_visible_cols(const tqp_table* t, const std::vector<int>& cols, const char* what) {
    for (int c : cols) {
        if (c < 0 || c >= t->num_cols || !t->cols[c].data) continue;
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, t->cols[c].data) != cudaSuccess) {
            cudaGetLastError();
            return fail(TQP_ERR_INVALID_ARG, "%s: column %d is not CUDA-visible memory", what, c);
        }
        if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) continue;
        if (a.type == cudaMemoryTypeHost && a.devicePointer != nullptr) continue;
        return fail(TQP_ERR_INVALID_ARG,
                    "%s: column %d is neither device memory nor page-locked host memory the GPU can address", what,
                    c);
    }
    return TQP_OK;
}

tqp_status lower_preds(const tqp_table* t, const tqp_pred* preds, int32_t npreds, Cond* out, int* ncond) {
    if (npreds < 0 || npreds > TQP_MAX_PREDS)
        return fail(TQP_ERR_INVALID_ARG, "npreds %d outside [0, %d]", npreds, TQP_MAX_PREDS);
    if (npreds > 0 && !preds) return fail(TQP_ERR_INVALID_ARG, "preds is NULL");
    for (int i = 0; i < npreds; ++i) {
        if (preds[i].op == TQP_IN || preds[i].op == TQP_LIKE || preds[i].op == TQP_NOT_LIKE)
            return fail(TQP_ERR_UNSUPPORTED, "predicate %d: IN / LIKE need the pre-pass, which this call does not run", i);
        if (preds[i].col >= 0 && preds[i].col < t->num_cols && t->cols[preds[i].col].type == TQP_CHAR)
            return fail(TQP_ERR_INVALID_ARG, "predicate %d: string column %d takes IN / LIKE / NOT LIKE only", i,
                        preds[i].col);
    }
    // Merge every non-NE comparison on a column into one inclusive range.
    std::vector<int64_t> lo(t->num_cols, INT64_MIN), hi(t->num_cols, INT64_MAX);
    std::vector<bool> used(t->num_cols, false), empty(t->num_cols, false);
    int n = 0;
    for (int i = 0; i < npreds; ++i) {
        const tqp_pred& p = preds[i];
        if (p.col < 0 || p.col >= t->num_cols)
            return fail(TQP_ERR_INVALID_ARG, "predicate %d: column %d out of range", i, p.col);
        const int c = p.col;
        switch (p.op) {
            case TQP_LT:
                if (p.lo == INT64_MIN) empty[c] = true; else hi[c] = std::min(hi[c], p.lo - 1);
                break;
            case TQP_LE: hi[c] = std::min(hi[c], p.lo); break;
            case TQP_GT:
                if (p.lo == INT64_MAX) empty[c] = true; else lo[c] = std::max(lo[c], p.lo + 1);
                break;
            case TQP_GE: lo[c] = std::max(lo[c], p.lo); break;
            case TQP_EQ:
                lo[c] = std::max(lo[c], p.lo);
                hi[c] = std::min(hi[c], p.lo);
                break;
            case TQP_BETWEEN:
                lo[c] = std::max(lo[c], p.lo);
                hi[c] = std::min(hi[c], p.hi);
                break;
            case TQP_NE:
                out[n].col = c;
                out[n].negate = 1;
                out[n].lo = p.lo;
                out[n].span = 0;
                ++n;
                continue;
            default: return fail(TQP_ERR_INVALID_ARG, "predicate %d: unknown operator %d", i, p.op);
        }
        used[c] = true;
    }
    for (int c = 0; c < t->num_cols; ++c) {
        if (!used[c]) continue;
        out[n].col = c;
        if (empty[c] || lo[c] > hi[c]) {  // never true: negate a range that holds for every value
            out[n].negate = 1;
            out[n].lo = 0;
            out[n].span = ~0ULL;
        } else if (lo[c] == INT64_MIN && hi[c] == INT64_MAX) {
            continue;  // always true
        } else {
            out[n].negate = 0;
            out[n].lo = lo[c];
            out[n].span = static_cast<uint64_t>(hi[c]) - static_cast<uint64_t>(lo[c]);
        }
        ++n;
    }
    *ncond = n;
    return TQP_OK;
}

void lower_fast(const Cond* conds, int ncond, const ScanGeom& G, CondFast* out, int32_t* fast) {
    *fast = 1;
    for (int q = 0; q < ncond; ++q) {
        const Cond& c = conds[q];
        const ColRef& cr = G.col[c.col];
        if (cr.slot < 0) *fast = 0;
        CondFast& f = out[q];
        f.soff = cr.soff;
        f.type = cr.type;
        f.pad = 0;
        // clamp [lo, hi] to the values the column type can hold
        const int64_t tmin = cr.type == TQP_U8 ? 0 : (cr.type == TQP_I32 ? INT32_MIN : INT64_MIN);
        const int64_t tmax = cr.type == TQP_U8 ? 255 : (cr.type == TQP_I32 ? INT32_MAX : INT64_MAX);
        f.negate = c.negate;
        f.lo = 0;
        f.span = ~0ULL;  // a test that holds for every value (also in 32 bits)
        if (c.span == ~0ULL) continue;  // the range covers everything already
        // lower_preds emits lo <= hi = lo + span without wrap-around
        const int64_t lo = c.lo;
        const int64_t hi = static_cast<int64_t>(static_cast<uint64_t>(lo) + c.span);
        const int64_t clo = std::max(lo, tmin), chi = std::min(hi, tmax);
        if (clo > chi) {
            // no value of the type is in range: the test never holds, so the
            // condition is the constant `negate`; express it with the
            // always-true test and the opposite negation
            f.negate = c.negate ? 0 : 1;
        } else {
            f.lo = clo;
            f.span = static_cast<uint64_t>(chi) - static_cast<uint64_t>(clo);
        }
    }
}

tqp_status lower_expr(const tqp_expr* e, int ncols, DExpr* out) {
    if (!e) return fail(TQP_ERR_INVALID_ARG, "expression is NULL");
    if (e->n < 1 || e->n > TQP_MAX_EXPR)
        return fail(TQP_ERR_INVALID_ARG, "expression length %d outside [1, %d]", e->n, TQP_MAX_EXPR);
    int depth = 0;
    for (int i = 0; i < e->n; ++i) {
        const int op = e->op[i];
        if (op == TQP_X_COL) {
            if (e->v[i] < 0 || e->v[i] >= ncols)
                return fail(TQP_ERR_INVALID_ARG, "expression token %d: column %lld out of range", i,
                            (long long)e->v[i]);
            ++depth;
        } else if (op == TQP_X_CONST) {
            ++depth;
        } else if (op == TQP_X_ADD || op == TQP_X_SUB || op == TQP_X_MUL) {
            if (depth < 2) return fail(TQP_ERR_INVALID_ARG, "expression token %d: operator needs two operands", i);
            --depth;
        } else {
            return fail(TQP_ERR_INVALID_ARG, "expression token %d: unknown opcode %d", i, op);
        }
        if (depth > 4) return fail(TQP_ERR_UNSUPPORTED, "expression stack deeper than 4");
    }
    if (depth != 1) return fail(TQP_ERR_INVALID_ARG, "expression leaves %d values on the stack", depth);
    out->n = e->n;
    for (int i = 0; i < TQP_MAX_EXPR; ++i) {
        out->op[i] = i < e->n ? e->op[i] : 0;
        out->v[i] = i < e->n ? e->v[i] : 0;
    }
    return TQP_OK;
}

// Symbolic evaluation of the postfix program over affine terms a * x + b
// (x one column, or none for a constant), mod 2^64.
namespace {
struct Aff {
    int col;  // -1: constant b
    uint64_t a, b;
};
struct Sym {
    int nf;   // 1: affine f[0]; 2: product f[0] * f[1]
    Aff f[2];
};
bool is_const(const Sym& s) { return s.nf == 1 && s.f[0].col < 0; }
Aff scale(Aff t, uint64_t k) {
    t.a *= k;
    t.b *= k;
    return t;
}
}  // namespace

bool lower_prod(const DExpr& e, const ScanGeom& G, ProdForm* out) {
    Sym st[TQP_MAX_EXPR];
    int sp = 0;
    for (int i = 0; i < e.n; ++i) {
        const int op = e.op[i];
        if (op == TQP_X_COL || op == TQP_X_CONST) {
            Sym s;
            s.nf = 1;
            s.f[0] = op == TQP_X_COL ? Aff{static_cast<int>(e.v[i]), 1u, 0u}
                                     : Aff{-1, 0u, static_cast<uint64_t>(e.v[i])};
            st[sp++] = s;
            continue;
        }
        if (sp < 2) return false;
        const Sym y = st[--sp];
        const Sym x = st[--sp];
        Sym r;
        if (op == TQP_X_ADD || op == TQP_X_SUB) {
            if (x.nf != 1 || y.nf != 1) return false;
            if (x.f[0].col >= 0 && y.f[0].col >= 0 && x.f[0].col != y.f[0].col) return false;
            const uint64_t sg = op == TQP_X_ADD ? 1u : ~0ull;  // +1 or -1 mod 2^64
            r.nf = 1;
            r.f[0].col = x.f[0].col >= 0 ? x.f[0].col : y.f[0].col;
            r.f[0].a = x.f[0].a + sg * y.f[0].a;
            r.f[0].b = x.f[0].b + sg * y.f[0].b;
        } else {  // MUL
            if (is_const(y)) {
                r = x;
                r.f[0] = scale(x.f[0], y.f[0].b);
            } else if (is_const(x)) {
                r = y;
                r.f[0] = scale(y.f[0], x.f[0].b);
            } else if (x.nf == 1 && y.nf == 1) {
                r.nf = 2;
                r.f[0] = x.f[0];
                r.f[1] = y.f[0];
            } else {
                return false;
            }
        }
        st[sp++] = r;
    }
    if (sp != 1) return false;
    const Sym& s = st[0];
    memset(out, 0, sizeof(*out));
    for (int k = 0; k < 2; ++k) {
        Aff t = k < s.nf ? s.f[k] : Aff{-1, 0u, 1u};
        if (t.col >= 0 && t.a == 0) t.col = -1;  // 0 * x + b is the constant b
        if (t.col >= 0) {
            if (t.col >= G.ncols || G.col[t.col].slot < 0) return false;
            out->soff[k] = G.col[t.col].soff;
            out->type[k] = G.col[t.col].type;
            out->kind[k] = t.a == 1u ? (t.b == 0u ? kFacPlain : kFacAdd) : (t.a == ~0ull ? kFacRsub : kFacAffine);
        } else {
            out->type[k] = -1;
            out->kind[k] = kFacConst;
        }
        out->a[k] = static_cast<int64_t>(t.a);
        out->b[k] = static_cast<int64_t>(t.b);
    }
    return true;
}

void expr_cols(const DExpr& e, std::vector<int>& cols) {
    for (int i = 0; i < e.n; ++i)
        if (e.op[i] == TQP_X_COL) cols.push_back(static_cast<int>(e.v[i]));
}

static int esize_host(int type) { return type == TQP_I64 ? 8 : (type == TQP_I32 ? 4 : 1); }

tqp_tuning default_tuning(const tqp_ctx* ctx, int bytes_per_row, int body_smem) {
    if (ctx->forced.tile_rows > 0) return ctx->forced;
    tqp_tuning tu{0, 0, 0, 1};
    if (ctx->tuner && ctx->cur_key[0] && ctx->tuner->lookup(ctx->cur_key, &tu)) return tu;
    const int per_sm = 227 * 1024;
    // Two CTAs per SM: one can compute while the other waits on look-back.
    int budget = per_sm / 2 - kHeaderBytes - body_smem - 1024;
    tu.ctas_per_sm = 2;
    if (bytes_per_row * kRowQuantum * 2 > budget) {
        budget = std::min(ctx->smem_optin, per_sm) - kHeaderBytes - body_smem - 1024;
        tu.ctas_per_sm = 1;
    }
    int T = kRowQuantum;
    for (int cand = 4096; cand >= kRowQuantum; cand /= 2) {
        if (static_cast<long long>(cand) * std::max(bytes_per_row, 1) * 3 <= budget) {
            T = cand;
            break;
        }
    }
    tu.tile_rows = T;
    const int stage = std::max(bytes_per_row, 1) * T + 128 * kMaxStaged;
    tu.stages = std::max(2, std::min(kMaxStages, budget / stage));
    return tu;
}

tqp_status make_geom(const tqp_ctx* ctx, const tqp_table* t, std::vector<int> staged, const tqp_tuning& tu,
                     int body_smem, ScanGeom* G, size_t* smem_bytes) {
    std::sort(staged.begin(), staged.end());
    staged.erase(std::unique(staged.begin(), staged.end()), staged.end());
    if (static_cast<int>(staged.size()) > kMaxStaged) staged.resize(kMaxStaged);
    if (tu.tile_rows < kRowQuantum || tu.tile_rows > kMaxTileRows || tu.tile_rows % kRowQuantum)
        return fail(TQP_ERR_INVALID_ARG, "tile rows %d invalid", tu.tile_rows);
    memset(G, 0, sizeof(*G));
    G->n = t->num_rows;
    G->T = tu.tile_rows;
    G->ntiles = (t->num_rows + G->T - 1) / G->T;
    G->nstages = std::max(2, std::min(kMaxStages, tu.stages));
    G->ncols = t->num_cols;
    for (int c = 0; c < t->num_cols; ++c) {
        G->col[c].ptr = static_cast<const unsigned char*>(t->cols[c].data);
        G->col[c].type = t->cols[c].type;
        G->col[c].slot = -1;
        G->col[c].soff = 0;
    }
    int off = 0;
    G->nstaged = static_cast<int>(staged.size());
    for (int k = 0; k < G->nstaged; ++k) {
        const int c = staged[k];
        G->staged[k] = c;
        G->col[c].slot = k;
        G->col[c].soff = off;
        off += (G->T * esize_host(t->cols[c].type) + 127) / 128 * 128;
    }
    G->stage_bytes = std::max(off, 128);
    *smem_bytes = static_cast<size_t>(kHeaderBytes) + body_smem + static_cast<size_t>(G->nstages) * G->stage_bytes;
    if (*smem_bytes > static_cast<size_t>(ctx->smem_optin))
        return fail(TQP_ERR_UNSUPPORTED, "scan needs %zu bytes of shared memory (device allows %d)", *smem_bytes,
                    ctx->smem_optin);
    return TQP_OK;
}

int engine_grid(const tqp_ctx* ctx, const void* kernel, size_t smem, int64_t ntiles, int ctas_per_sm) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kEngineThreads, smem) != cudaSuccess || occ < 1)
        occ = 1;
    if (ctas_per_sm > 0) occ = std::min(occ, ctas_per_sm);
    const int64_t g = std::min<int64_t>(static_cast<int64_t>(ctx->num_sms) * occ, ntiles);
    return static_cast<int>(std::max<int64_t>(g, 1));
}

__global__ void k_set_i64(long long* p, long long v) { *p = v; }

tqp_status set_device_i64(long long* d_ptr, long long value, cudaStream_t stream) {
    k_set_i64<<<1, 1, 0, stream>>>(d_ptr, value);
    TQP_CUDA(cudaGetLastError());
    return TQP_OK;
}

tqp_status allow_smem(const tqp_ctx* ctx, const void* kernel, SmemFlags& flags) {
    if (ctx->device < kMaxDevices && flags.done[ctx->device].load(std::memory_order_acquire)) return TQP_OK;
    cudaFuncAttributes fa;
    TQP_CUDA(cudaFuncGetAttributes(&fa, kernel));
    const int dyn = ctx->smem_optin - static_cast<int>(fa.sharedSizeBytes);
    TQP_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn));
    if (ctx->device < kMaxDevices) flags.done[ctx->device].store(true, std::memory_order_release);
    return TQP_OK;
}

}  // namespace tqp

using namespace tqp;

extern "C" {

const char* tqp_last_error(void) { return g_last_error.c_str(); }

int tqp_version(void) { return TQP_VERSION; }

const char* tqp_status_string(tqp_status s) {
    switch (s) {
        case TQP_OK: return "ok";
        case TQP_ERR_INVALID_ARG: return "invalid argument";
        case TQP_ERR_UNSUPPORTED: return "unsupported";
        case TQP_ERR_OUT_OF_MEMORY: return "out of scratch memory";
        case TQP_ERR_CAPACITY: return "output capacity exceeded";
        case TQP_ERR_OVERFLOW: return "integer overflow";
        case TQP_ERR_TIMEOUT: return "device wait timed out";
        case TQP_ERR_CUDA: return "CUDA error";
    }
    return "unknown status";
}

tqp_status tqp_ctx_create(int device, void* d_arena, size_t arena_bytes, tqp_ctx** out) {
    clear_error();
    if (!out) return fail(TQP_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (arena_bytes < kPersistentBytes + 4096)
        return fail(TQP_ERR_INVALID_ARG, "arena_bytes %zu too small (minimum %zu)", arena_bytes,
                    kPersistentBytes + 4096);
    if (d_arena && reinterpret_cast<uintptr_t>(d_arena) % 256 != 0)
        return fail(TQP_ERR_INVALID_ARG, "d_arena must be 256-byte aligned");
    int ndev = 0;
    TQP_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(TQP_ERR_INVALID_ARG, "device %d out of range", device);
    DeviceGuard g(device);
    if (!g.ok) return fail(TQP_ERR_CUDA, "cannot select device %d", device);
    tqp_ctx* ctx = new (std::nothrow) tqp_ctx();
    if (!ctx) return fail(TQP_ERR_OUT_OF_MEMORY, "host allocation failed");
    ctx->device = device;
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    cudaDeviceGetAttribute(&ctx->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    cudaDeviceGetAttribute(&ctx->l2_bytes, cudaDevAttrL2CacheSize, device);
    ctx->arena_bytes = arena_bytes;
    ctx->top = arena_bytes;
    ctx->force_variant = -1;
    ctx->wait_cap = kDefaultWaitCap;
    ctx->jit = 1;
    if (d_arena) {
        ctx->arena = static_cast<unsigned char*>(d_arena);
        ctx->owns_arena = false;
    } else {
        cudaError_t e = cudaMalloc(&ctx->arena, arena_bytes);
        if (e != cudaSuccess) {
            delete ctx;
            return cuda_fail(e, "cudaMalloc(arena)");
        }
        ctx->owns_arena = true;
    }
    ctx->d_err = reinterpret_cast<int*>(ctx->arena);
    cudaError_t e = cudaMemset(ctx->arena, 0, kPersistentBytes);
    if (e != cudaSuccess) {
        if (ctx->owns_arena) cudaFree(ctx->arena);
        delete ctx;
        return cuda_fail(e, "cudaMemset(arena)");
    }
    arena_reset(ctx);
    *out = ctx;
    return TQP_OK;
}

tqp_status tqp_ctx_destroy(tqp_ctx* ctx) {
    clear_error();
    if (!ctx) return TQP_OK;
    tqp_status s = TQP_OK;
    tuner_destroy(ctx);
    if (ctx->owns_arena) {
        DeviceGuard g(ctx->device);
        cudaError_t e = cudaFree(ctx->arena);
        if (e != cudaSuccess) s = cuda_fail(e, "cudaFree(arena)");
    }
    delete ctx;
    return s;
}

tqp_status tqp_ctx_set_wait_limit(tqp_ctx* ctx, int64_t polls) {
    clear_error();
    TQP_TRY(check_ctx(ctx));
    if (polls < 1) return fail(TQP_ERR_INVALID_ARG, "wait limit must be >= 1");
    ctx->wait_cap = polls;
    return TQP_OK;
}

size_t tqp_ctx_arena_bytes(const tqp_ctx* ctx) { return ctx ? ctx->arena_bytes : 0; }

tqp_status tqp_ctx_set_variant(tqp_ctx* ctx, int32_t variant) {
    clear_error();
    TQP_TRY(check_ctx(ctx));
    if (variant < -1 || variant > 1) return fail(TQP_ERR_INVALID_ARG, "variant must be -1, 0 or 1");
    ctx->force_variant = variant;
    return TQP_OK;
}

tqp_status tqp_ctx_set_tuning(tqp_ctx* ctx, int32_t tile_rows, int32_t stages, int32_t ctas_per_sm) {
    clear_error();
    TQP_TRY(check_ctx(ctx));
    if (tile_rows == 0 && stages == 0 && ctas_per_sm == 0) {
        ctx->forced = tqp_tuning{0, 0, 0, 0};
        return TQP_OK;
    }
    if (tile_rows < kRowQuantum || tile_rows > kMaxTileRows || tile_rows % kRowQuantum)
        return fail(TQP_ERR_INVALID_ARG, "tile_rows must be a multiple of %d in [%d, %d]", kRowQuantum,
                    kRowQuantum, kMaxTileRows);
    if (stages < 2 || stages > kMaxStages) return fail(TQP_ERR_INVALID_ARG, "stages must be in [2, %d]", kMaxStages);
    if (ctas_per_sm < 1 || ctas_per_sm > 2) return fail(TQP_ERR_INVALID_ARG, "ctas_per_sm must be 1 or 2");
    ctx->forced = tqp_tuning{tile_rows, stages, ctas_per_sm, 1};
    return TQP_OK;
}

tqp_status tqp_ctx_check(tqp_ctx* ctx, void* stream) {
    clear_error();
    TQP_TRY(check_ctx(ctx));
    DeviceGuard g(ctx->device);
    return take_device_error(ctx, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
