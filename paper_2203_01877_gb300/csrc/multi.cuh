// Shared scans: one pass over a table evaluates the filters of up to 32
// queries at once (each query: a conjunction of range predicates, a count of
// its passing rows and optionally the sum of a closed-form expression over
// them, exactly what tqp_filter computes without row ids).
//
// The paper runs one query at a time (Section 4.3); a served workload of many
// filter queries over one resident table would read the table once per
// query.  Here the staged scan engine streams the table once and every row is
// tested against all queries:
//   * predicates, per column: the breakpoints of every query's range
//     conditions on that column cut the value line into elementary intervals
//     on which each condition's outcome is constant; the host tabulates, per
//     interval, the 32-bit mask of queries whose conditions on that column all
//     pass.  A row's pass mask is the AND over the condition columns of the
//     mask of the interval its value falls in: a direct table lookup when the
//     breakpoints span at most kMqDirectMax values, else a branch-free binary
//     search over the sorted breakpoints.  The cost per row grows with the
//     number of condition columns, not with the number of queries;
//   * accumulation: every consumer warp keeps a count and a sum per query in
//     shared memory; each lane walks the set bits of its rows' pass masks and
//     adds to those queries with shared-memory atomics (the work is the
//     number of (row, passing query) pairs, spread over the lanes; rows that
//     pass no query cost nothing).  At the end of a chunk lane q moves query
//     q's totals of its warp to global memory;
//   * per-query row ranges: a query may cover only rows [rlo, rhi) of the
//     scan (queries over slices of one table).  Per tile a ballot splits the
//     queries into those covering the whole tile and those touching part of
//     it; only the latter are tested row by row.
// At most two distinct sum expressions per launch (each a product of two
// affine factors of staged columns, the ProdForm of the single-query scan);
// the host splits larger query sets into groups, one launch each.
#pragma once

#include <vector>

#include "bodies.cuh"

namespace tqp {

constexpr int kMqMax = 32;          // queries per launch: one per lane
constexpr int kMqExprs = 2;         // distinct sum expressions per launch
constexpr int kMqMinPack = 3;       // smaller packs run through the single-query scan (faster there)
constexpr int kMqWords = 5120;      // mask words of all lookup tables (shared memory)
constexpr int kMqBreaks = 512;      // breakpoints of the searched tables (shared memory)
constexpr int kMqDirectMax = 4096;  // direct tables: at most this many entries per column
// per-warp accumulators: 32 sums (8 bytes) and 32 counts (4 bytes) per consumer warp
constexpr int kMqAccBytes = kConsumerWarps * kMqMax * 12;

// Shared memory of one launch's body: accumulators | mask words | breakpoints.
__host__ __device__ constexpr int mq_words_bytes(int nwords) { return (nwords * 4 + 15) / 16 * 16; }
__host__ __device__ constexpr int mq_body_bytes(int nwords, int nbreaks) {
    return (kMqAccBytes + mq_words_bytes(nwords) + nbreaks * 8 + 127) / 128 * 128;
}

// One condition column of a launch.
struct MqCol {
    int32_t col;     // table column
    int32_t soff;    // byte offset of the column inside a stage
    int32_t type;
    int32_t direct;  // 1: direct table, 0: searched breakpoints
    int64_t base;    // direct: the value of entry 1 (entry 0: every smaller value)
    int32_t len;     // direct: entries (the last one: its value and every larger value);
                     // searched: breakpoints (len + 1 masks)
    int32_t off;     // first mask word
    int32_t boff;    // searched: first breakpoint
    int32_t steps;   // searched: the largest power of two <= len (0 when len == 0)
};

// Outputs and row range of one query (device memory; read at the end of the
// launch and once per chunk).
struct MqOut {
    int64_t* count;   // passing rows (nullable)
    int64_t* count2;  // a second copy of the count (nullable)
    int64_t* sum;     // sum of the query's expression (nullable)
    int64_t rlo, rhi; // rows [rlo, rhi) of the scanned table
};

struct MultiArgs {
    ScanGeom G;
    EngineCtl ctl;
    int32_t nq;
    int32_t ncols;        // condition columns
    int32_t nexpr;        // distinct sum expressions (0..kMqExprs)
    uint32_t esel;        // bit q: query q sums expression 1 (else expression 0)
    uint32_t all;         // bits of the nq queries
    int32_t nwords;       // mask words used
    int32_t nbreaks;      // breakpoints used
    int32_t body_bytes;   // shared memory of the body (mq_body_bytes, or the largest in a batch)
    MqCol c[kMaxStaged];
    ProdForm e[kMqExprs];
    int32_t ecol[kMqExprs][2];   // table column of each factor (-1: constant)
    const uint32_t* words;       // lookup masks (device)
    const int64_t* breaks;       // sorted breakpoints of searched tables (device)
    const MqOut* out;            // nq entries (device)
    unsigned long long* acc;     // [2 q] sum, [2 q + 1] count, [2 kMqMax] completions (zeroed)
};

// Mask of the interval containing x in column table `mc`.
__device__ __forceinline__ uint32_t mq_lookup(const MqCol& mc, int64_t x, const uint32_t* w, const int64_t* bk) {
    if (mc.direct) {
        int idx;
        if (x < mc.base) {
            idx = 0;
        } else {
            const uint64_t d = static_cast<uint64_t>(x) - static_cast<uint64_t>(mc.base);
            idx = d >= static_cast<uint64_t>(mc.len - 1) ? mc.len - 1 : static_cast<int>(d) + 1;
        }
        return w[mc.off + idx];
    }
    // number of breakpoints <= x, by halving steps over the sorted breakpoints
    const int64_t* b = bk + mc.boff;
    int pos = 0;
    for (int s = mc.steps; s > 0; s >>= 1)
        if (pos + s <= mc.len && b[pos + s - 1] <= x) pos += s;
    return w[mc.off + pos];
}

// Value of one affine factor at tile row r of a tile that is not full.
__device__ __forceinline__ int64_t mq_factor_row(const ScanGeom& G, const TileView& v, const ProdForm& f, int i,
                                                 int col, int r) {
    const int kind = f.kind[i];
    if (kind == kFacConst) return f.b[i];
    const uint64_t x = static_cast<uint64_t>(col_val(G, v, col, r));
    const uint64_t a = static_cast<uint64_t>(f.a[i]), b = static_cast<uint64_t>(f.b[i]);
    if (kind == kFacPlain) return static_cast<int64_t>(x);
    if (kind == kFacAdd) return static_cast<int64_t>(x + b);
    if (kind == kFacRsub) return static_cast<int64_t>(b - x);
    return static_cast<int64_t>(x * a + b);
}

// 64-bit add to shared memory as two 32-bit atomic adds (low word, then the
// high word with the carry): measured faster than a 64-bit atomic add on
// shared memory.  Readers see the sum only after the warp's adds are done.
__device__ __forceinline__ void add_shared_u64(unsigned long long* p, unsigned long long x) {
    unsigned int* w = reinterpret_cast<unsigned int*>(p);
    const unsigned int lo = static_cast<unsigned int>(x);
    const unsigned int old = atomicAdd(w, lo);
    const unsigned int hi = static_cast<unsigned int>(x >> 32) + (old + lo < old ? 1u : 0u);
    if (hi) atomicAdd(w + 1, hi);
}

// A direct-table condition column held in registers by the fast path: the
// value is clamped to [lo, lo + span] and indexes the table at word off.
struct MqHot {
    uint32_t d;     // stage byte offset | type << 20
    int32_t off;    // first mask word
    int32_t span;   // entries - 1
    int64_t lo;     // the value of entry 0's upper end (base - 1)
};
constexpr int kMqFastCols = 4;  // condition columns of the fast path

struct MultiBody {
    static constexpr int kMinBlocks = 2;
    static constexpr int kSmemBytes = mq_body_bytes(kMqWords, kMqBreaks);  // the largest launch
    static constexpr int kU = 4;  // rows per lane per step

    const MultiArgs& A;
    const uint32_t* w;         // shared-memory copy of the masks
    const int64_t* bk;         // shared-memory copy of the breakpoints
    unsigned long long* wsum;  // this warp's 32 sums
    unsigned int* wcnt;        // this warp's 32 counts
    int64_t rlo = 0, rhi = 0;  // lane q: query q's row range
    MqHot hot[kMqFastCols];    // fast path: the condition columns
    bool fast = false;         // every condition column has a direct table (at most kMqFastCols)

    const MqOut* outp;         // the queries' outputs and row ranges

    // Every thread of the CTA copies its share of the tables and each
    // consumer warp clears its accumulators; the caller synchronises the CTA
    // before the first tile.  The tables and outputs come from the argument
    // block's pointers, or from the explicit ones (kernel parameters).
    __device__ MultiBody(const MultiArgs& a, unsigned char* sm) : MultiBody(a, sm, a.words, a.breaks, a.out) {}
    __device__ MultiBody(const MultiArgs& a, unsigned char* sm, const uint32_t* words, const int64_t* breaks,
                         const MqOut* out)
        : A(a), outp(out) {
        unsigned long long* acc = reinterpret_cast<unsigned long long*>(sm);
        unsigned int* cnt = reinterpret_cast<unsigned int*>(sm + kConsumerWarps * kMqMax * 8);
        uint32_t* ws = reinterpret_cast<uint32_t*>(sm + kMqAccBytes);
        int64_t* bs = reinterpret_cast<int64_t*>(sm + kMqAccBytes + mq_words_bytes(a.nwords));
        for (int i = threadIdx.x; i < a.nwords; i += blockDim.x) ws[i] = words[i];
        for (int i = threadIdx.x; i < a.nbreaks; i += blockDim.x) bs[i] = breaks[i];
        w = ws;
        bk = bs;
        const int warp = threadIdx.x / kWarp;
        const int lane = threadIdx.x % kWarp;
        const int cw = warp < kConsumerWarps ? warp : 0;
        wsum = acc + cw * kMqMax;
        wcnt = cnt + cw * kMqMax;
        if (warp < kConsumerWarps) {
            wsum[lane] = 0;
            wcnt[lane] = 0;
        }
        if (lane < a.nq) {
            rlo = out[lane].rlo;
            rhi = out[lane].rhi;
        }
        fast = a.ncols <= kMqFastCols;
#pragma unroll
        for (int k = 0; k < kMqFastCols; ++k) {
            hot[k] = MqHot{0u, 0, 0, 0};
            if (k < a.ncols) {
                const MqCol& mc = a.c[k];
                fast = fast && mc.direct;
                hot[k] = MqHot{static_cast<uint32_t>(mc.soff) | (static_cast<uint32_t>(mc.type) << 20), mc.off,
                               mc.len - 1, mc.base - 1};
            }
        }
    }

    // Full tiles with direct tables only: descriptors in registers, each
    // lookup a clamp and one shared-memory load.  Rows rb + lane + 32 j.
    __device__ __forceinline__ void fast_step(const TileView& v, int rb, int lane, uint32_t full, uint32_t part) {
        constexpr int U = kU;
        const int r0 = rb + lane;
        uint32_t m[U];
#pragma unroll
        for (int j = 0; j < U; ++j) m[j] = full;
        if (part) row_ranges<U>(v, r0, part, m);
#pragma unroll
        for (int k = 0; k < kMqFastCols; ++k) {
            if (k >= A.ncols) break;
            const MqHot h = hot[k];
            const unsigned char* col = v.stage + (h.d & 0xFFFFFu);
            const int type = static_cast<int>(h.d >> 20);
            if (type == TQP_I64) {
                const int64_t hi = h.lo + h.span;
#pragma unroll
                for (int j = 0; j < U; ++j) {
                    int64_t x = reinterpret_cast<const int64_t*>(col)[r0 + kWarp * j];
                    x = x < h.lo ? h.lo : (x > hi ? hi : x);
                    m[j] &= w[h.off + static_cast<int>(x - h.lo)];
                }
            } else {
                // 32- and 8-bit columns: the clamp bounds are values of the type
                const int lo = static_cast<int>(h.lo), hi = lo + h.span;
                int x[U];
                if (type == TQP_I32) {
#pragma unroll
                    for (int j = 0; j < U; ++j) x[j] = reinterpret_cast<const int*>(col)[r0 + kWarp * j];
                } else {
#pragma unroll
                    for (int j = 0; j < U; ++j) x[j] = col[r0 + kWarp * j];
                }
#pragma unroll
                for (int j = 0; j < U; ++j) m[j] &= w[h.off + (min(max(x[j], lo), hi) - lo)];
            }
        }
        accumulate<U>(v, r0, m);
    }

    // Queries whose row range ends inside the tile: their bits, row by row.
    template <int U>
    __device__ __forceinline__ void row_ranges(const TileView& v, int r0, uint32_t part, uint32_t (&m)[U]) {
        uint32_t p = part;
        while (p) {
            const int q = __ffs(p) - 1;
            p &= p - 1;
            const long long lo = __shfl_sync(0xffffffffu, static_cast<long long>(rlo), q);
            const long long hi = __shfl_sync(0xffffffffu, static_cast<long long>(rhi), q);
#pragma unroll
            for (int j = 0; j < U; ++j) {
                const long long row = v.row0 + r0 + kWarp * j;
                if (r0 + kWarp * j < v.rows && row >= lo && row < hi) m[j] |= 1u << q;
            }
        }
    }

    // Sum expressions of full-tile rows and every (row, passing query) pair.
    template <int U>
    __device__ __forceinline__ void accumulate(const TileView& v, int r0, const uint32_t (&m)[U]) {
        uint32_t mor = 0;
#pragma unroll
        for (int j = 0; j < U; ++j) mor |= m[j];
        if (!__any_sync(0xffffffffu, mor != 0u)) return;
        int64_t v0[U], v1[U];
#pragma unroll
        for (int j = 0; j < U; ++j) v0[j] = v1[j] = 0;
        if (A.nexpr > 0) {
            prod_eval<U>(A.e[0], v.stage, r0, v0);
            if (A.nexpr > 1) prod_eval<U>(A.e[1], v.stage, r0, v1);
        }
        add_pairs<U>(m, v0, v1);
    }

    // One work list per lane over its U rows: the warp iterates as often as
    // its busiest lane has (row, passing query) pairs.
    template <int U>
    __device__ __forceinline__ void add_pairs(const uint32_t (&m)[U], const int64_t (&v0)[U], const int64_t (&v1)[U]) {
        const uint32_t esel = A.esel;
        uint32_t mm[U];
#pragma unroll
        for (int j = 0; j < U; ++j) mm[j] = m[j];
        while (true) {
            int64_t a0 = v0[U - 1], a1 = v1[U - 1];
            uint32_t cur = mm[U - 1];
            int jj = U - 1;
#pragma unroll
            for (int j = U - 2; j >= 0; --j) {
                if (mm[j]) {
                    a0 = v0[j];
                    a1 = v1[j];
                    cur = mm[j];
                    jj = j;
                }
            }
            if (!cur) break;
            const int q = __ffs(cur) - 1;
#pragma unroll
            for (int j = 0; j < U; ++j)
                if (j == jj) mm[j] = cur & (cur - 1);
            add_shared_u64(&wsum[q], static_cast<unsigned long long>(((esel >> q) & 1u) ? a1 : a0));
            atomicAdd(&wcnt[q], 1u);
        }
    }

    // General path (a ragged last tile, searched tables, more than
    // kMqFastCols condition columns): rows rb + lane + 32 j of the tile.
    __device__ __forceinline__ void step(const ScanGeom& G, const TileView& v, int rb, int lane, uint32_t full,
                                         uint32_t part) {
        constexpr int U = kU;
        const int r0 = rb + lane;
        uint32_t m[U];
#pragma unroll
        for (int j = 0; j < U; ++j) m[j] = (r0 + kWarp * j < v.rows) ? full : 0u;
        if (part) row_ranges<U>(v, r0, part, m);
        // predicates: the interval masks of every condition column
        for (int k = 0; k < A.ncols; ++k) {
            const MqCol& mc = A.c[k];
            int64_t x[U];
            if (v.full) {
                load_rows<U>(v.stage + mc.soff, mc.type, r0, x);
            } else {
#pragma unroll
                for (int j = 0; j < U; ++j) x[j] = (r0 + kWarp * j < v.rows) ? col_val(G, v, mc.col, r0 + kWarp * j) : 0;
            }
#pragma unroll
            for (int j = 0; j < U; ++j) m[j] &= mq_lookup(mc, x[j], w, bk);
        }
        if (v.full) {
            accumulate<U>(v, r0, m);
            return;
        }
        uint32_t mor = 0;
#pragma unroll
        for (int j = 0; j < U; ++j) mor |= m[j];
        if (!__any_sync(0xffffffffu, mor != 0u)) return;
        // sum expressions of the passing rows, the columns read through col_val
        int64_t v0[U], v1[U];
#pragma unroll
        for (int j = 0; j < U; ++j) {
            v0[j] = v1[j] = 0;
            const int r = r0 + kWarp * j;
            if (m[j] && A.nexpr > 0) {
                v0[j] = static_cast<int64_t>(static_cast<uint64_t>(mq_factor_row(G, v, A.e[0], 0, A.ecol[0][0], r)) *
                                             static_cast<uint64_t>(mq_factor_row(G, v, A.e[0], 1, A.ecol[0][1], r)));
                if (A.nexpr > 1)
                    v1[j] = static_cast<int64_t>(
                        static_cast<uint64_t>(mq_factor_row(G, v, A.e[1], 0, A.ecol[1][0], r)) *
                        static_cast<uint64_t>(mq_factor_row(G, v, A.e[1], 1, A.ecol[1][1], r)));
            }
        }
        add_pairs<U>(m, v0, v1);
    }

    __device__ void pass1(const ScanGeom& G, const TileView& v, int cw, int lane) {
        const long long t0 = v.row0, t1 = v.row0 + v.rows;
        const bool covers = rlo <= t0 && t1 <= rhi;
        const bool touches = rlo < t1 && rhi > t0;
        const uint32_t full = __ballot_sync(0xffffffffu, covers) & A.all;
        const uint32_t part = __ballot_sync(0xffffffffu, touches && !covers) & A.all;
        if (!(full | part)) return;
        const int rw = G.T / kConsumerWarps;  // a multiple of 128
        if (v.full && fast) {
            for (int r = 0; r < rw; r += kU * kWarp) fast_step(v, cw * rw + r, lane, full, part);
            return;
        }
        for (int r = 0; r < rw; r += kU * kWarp) {
            if (cw * rw + r >= v.rows) return;
            step(G, v, cw * rw + r, lane, full, part);
        }
    }

    __device__ void chunk_end(const ScanGeom&, long long, long long, long long, int, int lane) {
        __syncwarp();
        const unsigned long long ls = wsum[lane];
        const unsigned long long lc = wcnt[lane];
        wsum[lane] = 0;
        wcnt[lane] = 0;
        if (lane < A.nq) {
            if (ls) atomicAdd(&A.acc[2 * lane], ls);
            if (lc) atomicAdd(&A.acc[2 * lane + 1], lc);
        }
        __threadfence();
        __syncwarp();
        bool last = false;
        if (lane == 0) last = last_completion(&A.acc[2 * kMqMax], A.ctl.nchunks);
        last = __shfl_sync(0xffffffffu, last, 0);
        if (last && lane < A.nq) {
            __threadfence();
            const unsigned long long ts = atomicAdd(&A.acc[2 * lane], 0ULL);
            const unsigned long long tc = atomicAdd(&A.acc[2 * lane + 1], 0ULL);
            const MqOut& o = outp[lane];
            if (o.count) *o.count = static_cast<int64_t>(tc);
            if (o.count2) *o.count2 = static_cast<int64_t>(tc);
            if (o.sum) *o.sum = static_cast<int64_t>(ts);
        }
    }

    __device__ void finish(const ScanGeom&, int, int) {}
};

}  // namespace tqp

namespace tqp {

// The argument block of a stand-alone launch: the tables and outputs travel
// as kernel parameters (no upload, nothing to synchronise with).
struct MultiLaunch {
    MultiArgs A;
    uint32_t words[kMqWords];
    int64_t breaks[kMqBreaks];
    MqOut out[kMqMax];
};
static_assert(sizeof(MultiLaunch) <= 32764, "kernel parameters are limited to 32764 bytes");

}  // namespace tqp

// ---- host side (multi.cu) ------------------------------------------------------
namespace tqp {

// One filter query of a shared scan, lowered.
struct MqQuery {
    Cond cond[TQP_MAX_PREDS];
    int ncond = 0;
    bool has_sum = false;
    bool closed = false;   // the sum expression has the closed product form
    DExpr sum{};
    MqOut out{};
    std::vector<int> cols; // condition and expression columns, ascending
    std::vector<int> ecols; // expression columns
    std::vector<std::pair<int, int64_t>> bps;  // (column, breakpoint inside the column type's range)
    std::vector<std::pair<int, std::vector<int64_t>>> ins;  // numeric IN lists: (column, sorted values)
    bool alone = false;    // LIKE or string columns: runs through the single-query scan (and its pre-pass)
};

tqp_status mq_lower_query(const tqp_table* t, const tqp_pred* preds, int32_t npreds, const tqp_expr* sum_expr,
                          MqQuery* q);
// Pack queries into launches (first fit, in order); queries that fit no
// launch (an expression without the closed form, more than 8 columns) and
// packs of fewer than kMqMinPack queries go to `singles`, for the
// single-query scan (it reads the summed columns only at passing rows, which
// wins for one or two queries).
void mq_pack(const tqp_table* t, const std::vector<MqQuery>& qs, std::vector<std::vector<int>>* groups,
             std::vector<int>* singles);
// Lower one launch: its arguments (device pointers as offsets into `blob`,
// resolved by mq_bind once the blob is in device memory), the blob itself
// (lookup tables and per-query outputs) and the launch's shared memory.
// extra_smem: shared memory before the body (staged arguments, a batch job);
// fixed_body: the body takes MultiBody::kSmemBytes (a batch's common layout)
// instead of what this launch's tables need.  tu: NULL for the default tuning.
tqp_status mq_lower_group(const tqp_ctx* ctx, const tqp_table* t, const std::vector<MqQuery>& qs,
                          const std::vector<int>& members, const tqp_tuning* tu, int extra_smem, bool fixed_body,
                          MultiArgs* A, std::vector<unsigned char>* blob, size_t* smem, int* ctas_per_sm);
void mq_bind(MultiArgs* A, const unsigned char* d_blob);

}  // namespace tqp
