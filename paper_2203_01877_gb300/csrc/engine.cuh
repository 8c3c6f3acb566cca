// The staged scan engine: one persistent, warp-specialised CTA per SM slot.
//
// Rows are cut into tiles of T rows and tiles into contiguous chunks; a CTA
// draws a chunk ticket from a global atomic counter and streams the chunk's
// tiles.  The last warp (one elected lane) is the producer: for each tile it
// issues one bulk asynchronous copy (cp.async.bulk, TMA engine) per staged
// column into a ring of NS shared-memory stages, completion tracked with
// transaction-count mbarriers.  Warps 0..kConsumerWarps-1 consume the stages
// and run an operator-specific Body on every tile, then once per chunk.
//
// Chunk tickets (not blockIdx) order the chunks, so a chunk's predecessors
// were always taken by CTAs already running -- the forward-progress
// condition of a decoupled look-back over chunks.  Keeping the look-back at
// chunk granularity (one per CTA, not one per tile) takes it off the
// streaming path: with per-tile look-back the published-prefix frontier
// advances only ~32 tiles per L2 round trip, far below HBM rate.
//
// A tile's column region holds floor16(rows * esize) bytes; the last < 16
// bytes of a ragged final tile (and every column that is not staged) are
// read with ordinary global loads.
#pragma once

#include "common.cuh"

namespace tqp {

constexpr int kConsumerWarps = 8;
constexpr int kConsumers = kConsumerWarps * kWarp;
constexpr int kEngineThreads = kConsumers + kWarp;
constexpr int kMaxStages = 4;
constexpr int kMaxStaged = 8;
constexpr int kUnroll = 4;                                  // 32-row chunks per inner step
constexpr int kRowQuantum = kConsumerWarps * kWarp * kUnroll;  // T must be a multiple
constexpr int kMaxTileRows = 8192;
constexpr int kMaxChunksPerWarp = kMaxTileRows / (kConsumerWarps * kWarp);
constexpr int kBarConsumers = 1;                            // named barrier id

struct ColRef {
    const unsigned char* ptr;  // device column base
    int32_t type;              // tqp_dtype
    int32_t slot;              // staged slot, or -1
    int32_t soff;              // byte offset of this column inside a stage
    int32_t pad;
};

// Geometry and inputs of one scan (one table).
struct ScanGeom {
    int64_t n;         // rows
    int64_t ntiles;
    int32_t T;         // rows per tile, multiple of kRowQuantum
    int32_t nstages;   // 2..kMaxStages
    int32_t stage_bytes;
    int32_t nstaged;
    int32_t staged[kMaxStaged];  // column index per staged slot
    int32_t ncols;
    ColRef col[TQP_MAX_COLS];
};

// Range conditions: a row passes iff ((u64)(x - lo) <= span) != negate.
// Every tqp_cmp maps onto one of these (NE is the negated point range).
struct Cond {
    int32_t col;
    int32_t negate;
    int64_t lo;
    uint64_t span;
};

// Postfix expression with stack depth <= 4, evaluated in registers.
struct DExpr {
    int32_t n;
    int32_t op[TQP_MAX_EXPR];
    int64_t v[TQP_MAX_EXPR];
};

// A condition lowered for the full-tile fast path: the column is staged at
// byte `soff` of every stage and [lo, lo + span] has been clamped to the
// column type's value range, so int32 / uint8 columns compare in 32 bits.
struct CondFast {
    int32_t soff;
    int32_t type;
    int32_t negate;
    int32_t pad;
    int64_t lo;
    uint64_t span;
};

// An expression in closed form over staged columns: the product of two affine
// factors (a_i * x_i + b_i), evaluated mod 2^64 like the postfix program it
// came from (ring arithmetic, so the rewrite is exact).  Each factor is
// classified on the host so that the common shapes cost no multiply:
// constant b, x, x + b, b - x, or a * x + b.  Covers x, x * k, x + k, x * y
// and x * (k - y), the shapes of the paper's aggregates (Section 5.4).
enum : int32_t { kFacConst = 0, kFacPlain = 1, kFacAdd = 2, kFacRsub = 3, kFacAffine = 4 };

struct ProdForm {
    int32_t soff[2];
    int32_t type[2];
    int32_t kind[2];
    int32_t pad[2];
    int64_t a[2];
    int64_t b[2];
};

// x[j] = column value of tile row r0 + 32 j (the column is staged at `col`).
template <int U>
__device__ __forceinline__ void load_rows(const unsigned char* col, int type, int r0, int64_t (&x)[U]) {
    if (type == TQP_I64) {
#pragma unroll
        for (int j = 0; j < U; ++j) x[j] = reinterpret_cast<const int64_t*>(col)[r0 + 32 * j];
    } else if (type == TQP_I32) {
#pragma unroll
        for (int j = 0; j < U; ++j) x[j] = reinterpret_cast<const int32_t*>(col)[r0 + 32 * j];
    } else {
#pragma unroll
        for (int j = 0; j < U; ++j) x[j] = col[r0 + 32 * j];
    }
}

template <int U>
__device__ __forceinline__ void factor_eval(const ProdForm& f, int i, const unsigned char* stage, int r0,
                                            int64_t (&x)[U]) {
    const int kind = f.kind[i];
    const int64_t b = f.b[i];
    if (kind == kFacConst) {
#pragma unroll
        for (int j = 0; j < U; ++j) x[j] = b;
        return;
    }
    load_rows<U>(stage + f.soff[i], f.type[i], r0, x);
    if (kind == kFacPlain) return;
    if (kind == kFacAdd) {
#pragma unroll
        for (int j = 0; j < U; ++j) x[j] = static_cast<int64_t>(static_cast<uint64_t>(x[j]) + static_cast<uint64_t>(b));
    } else if (kind == kFacRsub) {
#pragma unroll
        for (int j = 0; j < U; ++j) x[j] = static_cast<int64_t>(static_cast<uint64_t>(b) - static_cast<uint64_t>(x[j]));
    } else {
        const uint64_t a = static_cast<uint64_t>(f.a[i]);
#pragma unroll
        for (int j = 0; j < U; ++j)
            x[j] = static_cast<int64_t>(static_cast<uint64_t>(x[j]) * a + static_cast<uint64_t>(b));
    }
}

template <int U>
__device__ __forceinline__ void prod_eval(const ProdForm& f, const unsigned char* stage, int r0, int64_t (&out)[U]) {
    factor_eval<U>(f, 0, stage, r0, out);
    if (f.kind[1] == kFacConst) {
        if (f.b[1] != 1) {
            const uint64_t k = static_cast<uint64_t>(f.b[1]);
#pragma unroll
            for (int j = 0; j < U; ++j) out[j] = static_cast<int64_t>(static_cast<uint64_t>(out[j]) * k);
        }
        return;
    }
    int64_t y[U];
    factor_eval<U>(f, 1, stage, r0, y);
#pragma unroll
    for (int j = 0; j < U; ++j)
        out[j] = static_cast<int64_t>(static_cast<uint64_t>(out[j]) * static_cast<uint64_t>(y[j]));
}

// Operand descriptors held in registers by the scan bodies (loaded once per
// CTA from the argument block): bits 0..19 stage byte offset, 20..21 column
// type, 22..24 factor kind, 25 negated condition.
__device__ __forceinline__ uint32_t hot_desc(int soff, int type, int kind, int negate) {
    return static_cast<uint32_t>(soff) | (static_cast<uint32_t>(type & 3) << 20) |
           (static_cast<uint32_t>(kind & 7) << 22) | (static_cast<uint32_t>(negate & 1) << 25);
}

template <int U>
__device__ __forceinline__ void hot_factor(uint32_t d, int64_t a, int64_t b, const unsigned char* stage, int r0,
                                           int64_t (&x)[U]) {
    const int kind = (d >> 22) & 7;
    if (kind == kFacConst) {
#pragma unroll
        for (int j = 0; j < U; ++j) x[j] = b;
        return;
    }
    load_rows<U>(stage + (d & 0xFFFFFu), (d >> 20) & 3, r0, x);
    if (kind == kFacPlain) return;
    if (kind == kFacAdd) {
#pragma unroll
        for (int j = 0; j < U; ++j) x[j] = static_cast<int64_t>(static_cast<uint64_t>(x[j]) + static_cast<uint64_t>(b));
    } else if (kind == kFacRsub) {
#pragma unroll
        for (int j = 0; j < U; ++j) x[j] = static_cast<int64_t>(static_cast<uint64_t>(b) - static_cast<uint64_t>(x[j]));
    } else {
#pragma unroll
        for (int j = 0; j < U; ++j)
            x[j] = static_cast<int64_t>(static_cast<uint64_t>(x[j]) * static_cast<uint64_t>(a) + static_cast<uint64_t>(b));
    }
}

// A closed-form expression (ProdForm) held in registers.
struct HotProd {
    uint32_t d[2];
    int64_t a[2], b[2];
    __device__ __forceinline__ void load(const ProdForm& f) {
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            d[i] = hot_desc(f.soff[i], f.type[i] < 0 ? 0 : f.type[i], f.kind[i], 0);
            a[i] = f.a[i];
            b[i] = f.b[i];
        }
    }
    template <int U>
    __device__ __forceinline__ void eval(const unsigned char* stage, int r0, int64_t (&out)[U]) const {
        hot_factor<U>(d[0], a[0], b[0], stage, r0, out);
        if (((d[1] >> 22) & 7) == kFacConst) {
            if (b[1] != 1) {
#pragma unroll
                for (int j = 0; j < U; ++j)
                    out[j] = static_cast<int64_t>(static_cast<uint64_t>(out[j]) * static_cast<uint64_t>(b[1]));
            }
            return;
        }
        int64_t y[U];
        hot_factor<U>(d[1], a[1], b[1], stage, r0, y);
#pragma unroll
        for (int j = 0; j < U; ++j)
            out[j] = static_cast<int64_t>(static_cast<uint64_t>(out[j]) * static_cast<uint64_t>(y[j]));
    }
};

// A full-tile range condition (CondFast) held in registers.
struct HotCond {
    uint32_t d;
    int64_t lo;
    uint64_t span;
    __device__ __forceinline__ void load(const CondFast& c) {
        d = hot_desc(c.soff, c.type, 0, c.negate);
        lo = c.lo;
        span = c.span;
    }
    // pass bits of rows r0 + 32 j
    template <int U>
    __device__ __forceinline__ uint32_t eval(const unsigned char* stage, int r0) const {
        const unsigned char* b = stage + (d & 0xFFFFFu);
        const int type = (d >> 20) & 3;
        uint32_t m = 0;
        if (type == TQP_I64) {
#pragma unroll
            for (int j = 0; j < U; ++j) {
                const uint64_t x = reinterpret_cast<const uint64_t*>(b)[r0 + kWarp * j];
                m |= static_cast<uint32_t>(x - static_cast<uint64_t>(lo) <= span) << j;
            }
        } else if (type == TQP_I32) {
            const uint32_t l = static_cast<uint32_t>(lo), sp = static_cast<uint32_t>(span);
#pragma unroll
            for (int j = 0; j < U; ++j) {
                const uint32_t x = reinterpret_cast<const uint32_t*>(b)[r0 + kWarp * j];
                m |= static_cast<uint32_t>(x - l <= sp) << j;
            }
        } else {
            const uint32_t l = static_cast<uint32_t>(lo), sp = static_cast<uint32_t>(span);
#pragma unroll
            for (int j = 0; j < U; ++j) {
                const uint32_t x = b[r0 + kWarp * j];
                m |= static_cast<uint32_t>(x - l <= sp) << j;
            }
        }
        return (d >> 25) & 1u ? ~m : m;
    }
};

struct TileView {
    const unsigned char* stage;  // shared-memory stage base
    int64_t tile;
    int64_t row0;
    int32_t rows;
    int32_t full;                // rows == T: every staged element is in smem
};

// Elements of a staged column present in shared memory: the bulk copy moves
// floor16(rows * esize) bytes.
__device__ __forceinline__ int staged_elems(int rows, int type) {
    const int es = esize_of(type);
    return static_cast<int>((static_cast<uint32_t>(rows) * es & ~15u) / es);
}

// Column value of tile row r (0 <= r < rows).
__device__ __forceinline__ int64_t col_val(const ScanGeom& G, const TileView& v, int c, int r) {
    const ColRef& cr = G.col[c];
    if (cr.slot >= 0 && (v.full || r < staged_elems(v.rows, cr.type))) return load_typed(v.stage + cr.soff, cr.type, r);
    return ldg_typed(cr.ptr, cr.type, v.row0 + r);
}

// The same expression for global row `grow`, every column read from global
// memory (used once a row's stage has been released).
__device__ __forceinline__ int64_t eval_expr_global(const ScanGeom& G, const DExpr& e, int64_t grow) {
    int64_t s0 = 0, s1 = 0, s2 = 0, s3 = 0;
#pragma unroll
    for (int i = 0; i < TQP_MAX_EXPR; ++i) {
        if (i >= e.n) break;
        const int op = e.op[i];
        if (op <= TQP_X_CONST) {
            int64_t x = e.v[i];
            if (op == TQP_X_COL) {
                const ColRef& cr = G.col[static_cast<int>(e.v[i])];
                x = ldg_typed(cr.ptr, cr.type, grow);
            }
            s3 = s2; s2 = s1; s1 = s0; s0 = x;
        } else {
            const int64_t b = s0, a = s1;
            s0 = (op == TQP_X_ADD) ? a + b : (op == TQP_X_SUB) ? a - b : a * b;
            s1 = s2; s2 = s3;
        }
    }
    return s0;
}

// Position of the n-th (0-based) set bit of m (n < popc(m)).
__device__ __forceinline__ int nth_set_bit(uint32_t m, int n) {
    int pos = 0;
    int c = __popc(m & 0xFFFFu);
    if (n >= c) { n -= c; pos += 16; m >>= 16; }
    c = __popc(m & 0xFFu);
    if (n >= c) { n -= c; pos += 8; m >>= 8; }
    c = __popc(m & 0xFu);
    if (n >= c) { n -= c; pos += 4; m >>= 4; }
    c = __popc(m & 0x3u);
    if (n >= c) { n -= c; pos += 2; m >>= 2; }
    if (n >= static_cast<int>(m & 1u)) pos += 1;
    return pos;
}

// Full-tile fast path: pass bits (bit j <-> row r0 + 32 j) of the conjunction,
// every condition column staged.  U rows per lane amortise each condition's
// setup; the range test is one subtract and one unsigned compare.
template <int U>
__device__ __forceinline__ uint32_t conds_full(const unsigned char* stage, const CondFast* cf, int ncond, int r0) {
    uint32_t ok = (U >= 32) ? 0xffffffffu : ((1u << U) - 1u);
    for (int q = 0; q < ncond; ++q) {
        const CondFast c = cf[q];
        const unsigned char* b = stage + c.soff;
        uint32_t m = 0;
        if (c.type == TQP_I64) {
            const uint64_t lo = static_cast<uint64_t>(c.lo);
#pragma unroll
            for (int j = 0; j < U; ++j) {
                const uint64_t x = reinterpret_cast<const uint64_t*>(b)[r0 + kWarp * j];
                m |= static_cast<uint32_t>(x - lo <= c.span) << j;
            }
        } else if (c.type == TQP_I32) {
            const uint32_t lo = static_cast<uint32_t>(c.lo), span = static_cast<uint32_t>(c.span);
#pragma unroll
            for (int j = 0; j < U; ++j) {
                const uint32_t x = reinterpret_cast<const uint32_t*>(b)[r0 + kWarp * j];
                m |= static_cast<uint32_t>(x - lo <= span) << j;
            }
        } else {
            const uint32_t lo = static_cast<uint32_t>(c.lo), span = static_cast<uint32_t>(c.span);
#pragma unroll
            for (int j = 0; j < U; ++j) {
                const uint32_t x = b[r0 + kWarp * j];
                m |= static_cast<uint32_t>(x - lo <= span) << j;
            }
        }
        ok &= c.negate ? ~m : m;
    }
    return ok;
}

// General path (ragged last tile, unstaged condition columns): 64-bit tests.
template <int U>
__device__ __forceinline__ uint32_t conds_general(const ScanGeom& G, const TileView& v, const Cond* conds,
                                                  int ncond, int r0) {
    uint32_t ok = 0;
#pragma unroll
    for (int j = 0; j < U; ++j) ok |= static_cast<uint32_t>(r0 + kWarp * j < v.rows) << j;
    for (int q = 0; q < ncond; ++q) {
        const Cond cd = conds[q];
#pragma unroll
        for (int j = 0; j < U; ++j) {
            if ((ok >> j) & 1u) {
                const int64_t x = col_val(G, v, cd.col, r0 + kWarp * j);
                const bool in = static_cast<uint64_t>(x) - static_cast<uint64_t>(cd.lo) <= cd.span;
                if (in == (cd.negate != 0)) ok &= ~(1u << j);
            }
        }
    }
    return ok;
}

template <int U>
__device__ __forceinline__ uint32_t eval_rows(const ScanGeom& G, const TileView& v, const CondFast* cf,
                                              const Cond* conds, int ncond, bool fast, int r0) {
    if (fast && v.full) return conds_full<U>(v.stage, cf, ncond, r0);
    return conds_general<U>(G, v, conds, ncond, r0);
}

// Evaluate a postfix expression for tile row r.  The stack lives in four
// registers that shift on push/pop, so no dynamic indexing is needed.
__device__ __forceinline__ int64_t eval_expr(const ScanGeom& G, const TileView& v, const DExpr& e, int r) {
    int64_t s0 = 0, s1 = 0, s2 = 0, s3 = 0;
#pragma unroll
    for (int i = 0; i < TQP_MAX_EXPR; ++i) {
        if (i >= e.n) break;
        const int op = e.op[i];
        if (op <= TQP_X_CONST) {
            const int64_t x = (op == TQP_X_COL) ? col_val(G, v, (int)e.v[i], r) : e.v[i];
            s3 = s2; s2 = s1; s1 = s0; s0 = x;
        } else {
            const int64_t b = s0, a = s1;
            s0 = (op == TQP_X_ADD) ? a + b : (op == TQP_X_SUB) ? a - b : a * b;
            s1 = s2; s2 = s3;
        }
    }
    return s0;
}

// Poll limit of the producer's final wait for its own bulk copies (with the
// back-off of mbar_wait, seconds): a CTA never exits with a copy in flight.
constexpr long long kDrainPolls = 1LL << 24;

// Shared-memory header of every engine CTA.
struct EngineHeader {
    uint64_t full[kMaxStages];
    uint64_t empty[kMaxStages];
    long long chunk;
    int abort;   // a wait of this CTA gave up: no more copies or tiles (sticky)
};
constexpr int kHeaderBytes = 128;
static_assert(sizeof(EngineHeader) <= kHeaderBytes, "engine header too large");

// Work split: tiles are grouped into `nchunks` contiguous chunks of
// `chunk_tiles` tiles; CTAs draw chunk tickets from `ticket`.
struct EngineCtl {
    unsigned long long* ticket;  // zeroed before the launch
    int* err;
    long long wait_cap;
    long long chunk_tiles;
    long long nchunks;
};

// Wait for phase `parity` of `bar` for at most `cap` polls, giving up early
// once the CTA's abort flag is set: 1 = complete, 0 = timed out, -1 = aborted.
__device__ __forceinline__ int mbar_wait_or_abort(uint64_t* bar, uint32_t parity, long long cap,
                                                  const volatile int* abort) {
    for (long long i = 0; i < cap; ++i) {
        if (mbar_test_wait(bar, parity)) return 1;
        if (*abort) return -1;
        if (i >= 16) __nanosleep(i < 1024 ? 32 : 256);
    }
    return 0;
}

// Body interface (all consumer threads call each member):
//   pass1(G, v, cw, lane)                  once per tile, reads the stage
//   chunk_end(G, chunk, t0, t1, cw, lane)  after the chunk's last tile
//   finish(G, cw, lane)                    after the CTA's last chunk
// Body::kSmemBytes bytes of shared memory precede the stages.
// One chunk [t0, t1) of tiles through the stage ring.  `it` (the pipeline
// position) persists across chunks; producer and consumers advance it
// identically, so every stage's mbarrier phase parity stays consistent.
//
// Bounded waits.  A wait that runs out (the context's wait limit) latches
// TQP_ERR_TIMEOUT and sets the CTA's abort flag; every other wait of the CTA
// gives up as soon as it sees the flag.  From then on the producer issues no
// copy and no arrival, and consumers process no tile and release no stage
// (a warp processes a tile with all lanes or not at all: the bodies use
// full-warp collectives).  The ring's invariants hold throughout: a stage is
// released only after its copy has landed, so the producer never starts a
// second copy into a stage, and no barrier receives more arrivals than it
// expects.  At the end of every chunk the producer waits -- with its own long
// limit, abort or not -- for each copy it issued that may still be landing.
// Bodies see the skipped tiles as tiles they were never given (chunk_end
// still runs).
template <class Body>
__device__ __forceinline__ void run_chunk(const ScanGeom& G, const EngineCtl& ctl, Body& body, long long chunk,
                                          long long t0, long long t1, EngineHeader* h, unsigned char* stages,
                                          long long& it, bool& aborted, uint64_t stream_policy, int warp, int lane) {
    volatile int* abort_flag = &h->abort;
    if (warp == kConsumerWarps) {
        // ---------------- producer: stage every tile of the chunk ----------------
        if (lane == 0) {
            uint32_t pend = 0;        // stages with a copy issued in this chunk
            uint32_t pend_par = 0;    // their phase parities
            for (long long t = t0; t < t1; ++t, ++it) {
                if (aborted) continue;
                const int s = static_cast<int>(it % G.nstages);
                const uint32_t ph = static_cast<uint32_t>((it / G.nstages) & 1);
                const int w = mbar_wait_or_abort(&h->empty[s], ph ^ 1u, ctl.wait_cap, abort_flag);
                if (w != 1) {
                    if (w == 0) latch_error(ctl.err, TQP_ERR_TIMEOUT);
                    *abort_flag = 1;
                    aborted = true;
                    continue;
                }
                const int64_t row0 = static_cast<int64_t>(t) * G.T;
                const int rows = static_cast<int>(G.n - row0 < G.T ? G.n - row0 : G.T);
                uint32_t total = 0;
                for (int k = 0; k < G.nstaged; ++k)
                    total += (static_cast<uint32_t>(rows) * esize_of(G.col[G.staged[k]].type)) & ~15u;
                unsigned char* dst = stages + static_cast<size_t>(s) * G.stage_bytes;
                if (total == 0) {
                    // no copy: this phase completes now, and the stage's
                    // earlier copy landed before its consumers released it
                    mbar_arrive(&h->full[s]);
                    pend &= ~(1u << s);
                } else {
                    mbar_arrive_expect_tx(&h->full[s], total);
                    for (int k = 0; k < G.nstaged; ++k) {
                        const ColRef& cr = G.col[G.staged[k]];
                        const int es = esize_of(cr.type);
                        const uint32_t bytes = (static_cast<uint32_t>(rows) * es) & ~15u;
                        if (bytes) bulk_g2s(dst + cr.soff, cr.ptr + row0 * es, bytes, &h->full[s], stream_policy);
                    }
                    pend |= 1u << s;
                    pend_par = (pend_par & ~(1u << s)) | (ph << s);
                }
            }
            // Drain: every copy of this chunk has landed before the chunk (or
            // the CTA) ends.  Only the producer advances a full barrier, so
            // the last issued phase of a stage is the one to wait for.
            const long long drain_cap = ctl.wait_cap > kDrainPolls ? ctl.wait_cap : kDrainPolls;
            for (int s = 0; s < G.nstages; ++s)
                if (((pend >> s) & 1u) && !mbar_wait(&h->full[s], (pend_par >> s) & 1u, drain_cap))
                    latch_error(ctl.err, TQP_ERR_TIMEOUT);
        } else {
            it += t1 - t0;
        }
    } else {
        // ---------------- consumers ----------------
        const int cw = warp;
        for (long long t = t0; t < t1; ++t, ++it) {
            if (aborted) continue;
            const int s = static_cast<int>(it % G.nstages);
            const uint32_t ph = static_cast<uint32_t>((it / G.nstages) & 1);
            const int w = mbar_wait_or_abort(&h->full[s], ph, ctl.wait_cap, abort_flag);
            if (!__all_sync(0xffffffffu, w == 1)) {
                const bool timed_out = __any_sync(0xffffffffu, w == 0);
                if (lane == 0) {
                    if (timed_out) latch_error(ctl.err, TQP_ERR_TIMEOUT);
                    *abort_flag = 1;
                }
                aborted = true;
                continue;
            }
            TileView v;
            v.stage = stages + static_cast<size_t>(s) * G.stage_bytes;
            v.tile = t;
            v.row0 = static_cast<int64_t>(t) * G.T;
            v.rows = static_cast<int>(G.n - v.row0 < G.T ? G.n - v.row0 : G.T);
            v.full = v.rows == G.T;
            body.pass1(G, v, cw, lane);
            __syncwarp();
            if (lane == 0) mbar_arrive(&h->empty[s]);
        }
        body.chunk_end(G, chunk, t0, t1, cw, lane);
    }
}

// Initialise the stage ring's mbarriers (thread 0; callers __syncthreads after).
__device__ __forceinline__ void init_stage_ring(EngineHeader* h, int nstages) {
    if (threadIdx.x == 0) {
        h->abort = 0;
        for (int s = 0; s < nstages; ++s) {
            mbar_init(&h->full[s], 1);
            mbar_init(&h->empty[s], kConsumerWarps);
        }
        fence_mbar_init();
    }
}

// Kernel arguments copied into shared memory (after the engine header): the
// hot loops then read them with shared-memory loads instead of dynamically
// indexed constant-bank or generic parameter loads.
template <class Args>
constexpr int args_bytes() { return (static_cast<int>(sizeof(Args)) + 127) / 128 * 128; }

template <class Args>
__device__ __forceinline__ const Args& stage_args(const Args& p, unsigned char* dst) {
    static_assert(sizeof(Args) % 4 == 0, "argument blocks are copied in 4-byte words");
    const uint32_t* src = reinterpret_cast<const uint32_t*>(&p);
    uint32_t* d = reinterpret_cast<uint32_t*>(dst);
    for (int i = threadIdx.x; i < static_cast<int>(sizeof(Args) / 4); i += blockDim.x) d[i] = src[i];
    __syncthreads();
    return *reinterpret_cast<const Args*>(dst);
}

// Dynamic shared memory: header | `extra` bytes (the staged arguments) |
// body_bytes (Body::kSmemBytes unless the body sizes its region per launch) |
// stages.
template <class Body>
__device__ __forceinline__ void run_engine(const ScanGeom& G, const EngineCtl& ctl, Body& body,
                                           unsigned char* smem, int extra = 0, int body_bytes = Body::kSmemBytes) {
    EngineHeader* h = reinterpret_cast<EngineHeader*>(smem);
    unsigned char* stages = smem + kHeaderBytes + extra + body_bytes;
    const int warp = threadIdx.x / kWarp;
    const int lane = threadIdx.x % kWarp;
    init_stage_ring(h, G.nstages);
    __syncthreads();

    long long it = 0;
    bool aborted = false;
    const uint64_t stream_policy = l2_evict_first_policy();
    while (true) {
        if (threadIdx.x == 0) h->chunk = static_cast<long long>(atomicAdd(ctl.ticket, 1ULL));
        __syncthreads();
        const long long chunk = h->chunk;
        __syncthreads();
        if (chunk >= ctl.nchunks) break;
        const long long t0 = chunk * ctl.chunk_tiles;
        const long long t1 = (t0 + ctl.chunk_tiles < G.ntiles) ? t0 + ctl.chunk_tiles : G.ntiles;
        run_chunk(G, ctl, body, chunk, t0, t1, h, stages, it, aborted, stream_policy, warp, lane);
        __syncthreads();
    }
    if (warp != kConsumerWarps) body.finish(G, warp, lane);
}

// ---- decoupled look-back (Merrill & Garland, "Single-pass Parallel Prefix
// Scan with Decoupled Look-back", NVIDIA TR 2016) ----------------------------
// Status word per tile: bits 63..62 flag (0 empty, 1 aggregate, 2 inclusive
// prefix), bits 61..0 value.  Called by one full warp; returns the exclusive
// prefix of `tile` and publishes its inclusive prefix.
constexpr unsigned long long kFlagA = 1ULL << 62;
constexpr unsigned long long kFlagP = 2ULL << 62;
constexpr unsigned long long kValMask = (1ULL << 62) - 1;

__device__ __forceinline__ unsigned long long lookback(unsigned long long* status, long long tile,
                                                       unsigned long long agg, int lane, int* err,
                                                       long long cap) {
    if (tile == 0) {
        if (lane == 0) st_relaxed_u64(&status[0], kFlagP | agg);
        return 0;
    }
    if (lane == 0) st_relaxed_u64(&status[tile], kFlagA | agg);
    unsigned long long excl = 0;
    long long base = tile - 1;
    long long polls = 0;
    bool gave_up = false;
    while (true) {
        const long long idx = base - lane;
        unsigned long long w = (idx >= 0) ? ld_relaxed_u64(&status[idx]) : kFlagP;
        // wait until every lane sees a published word (warp-uniform decisions)
        while (true) {
            const bool pending = (w >> 62) == 0;
            if (!__any_sync(0xffffffffu, pending)) break;
            const bool stop = (++polls > cap) || read_error(err) == TQP_ERR_TIMEOUT;
            if (__any_sync(0xffffffffu, stop)) {
                gave_up = true;
                break;
            }
            if (pending) {
                __nanosleep(32);
                w = ld_relaxed_u64(&status[idx]);
            }
        }
        if (gave_up) break;
        const uint32_t pmask = __ballot_sync(0xffffffffu, (w >> 62) == 2);
        // lanes up to and including the nearest inclusive prefix contribute
        const int stop = pmask ? (__ffs(pmask) - 1) : (kWarp - 1);
        unsigned long long contrib = (lane <= stop) ? (w & kValMask) : 0ULL;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) contrib += __shfl_xor_sync(0xffffffffu, contrib, o);
        excl += contrib;
        if (pmask) break;
        base -= kWarp;
    }
    if (gave_up && lane == 0) latch_error(err, TQP_ERR_TIMEOUT);
    if (lane == 0) st_relaxed_u64(&status[tile], kFlagP | ((excl + agg) & kValMask));
    return excl;
}

}  // namespace tqp
