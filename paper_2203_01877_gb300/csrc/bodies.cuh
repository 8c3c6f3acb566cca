// Consumer bodies of the staged scan engine, shared by the single-operator
// kernels (k_filter, k_groupby, k_plan_join) and the batched multi-plan
// kernel.  A body sees one tile at a time (pass1) and then the end of each
// chunk (chunk_end): every body flushes its partial results at chunk end and
// counts (chunk, warp) completions, so the same body works whether a CTA
// streams one table or chunks of many.  The warp that completes the last
// chunk of a scan publishes the scan's totals.
#pragma once

#include "engine.cuh"
#include "group.cuh"
#include "join.cuh"

namespace tqp {

constexpr int kCompactRows = 65536;                  // rows per compaction block of the selection mask
constexpr int kCompactWords = kCompactRows / kWarp;  // 2048 mask words
constexpr int kCompactThreads = 1024;

// Count one (chunk, warp) completion; true for the very last one of the scan.
__device__ __forceinline__ bool last_completion(unsigned long long* done, long long nchunks) {
    __threadfence();
    const unsigned long long d = atomicAdd(done, 1ULL);
    if (d != static_cast<unsigned long long>(nchunks) * kConsumerWarps - 1) return false;
    __threadfence();
    return true;
}

// ---- filter: predicates + selection mask + count + projection-sum ----------------

struct FilterArgs {
    ScanGeom G;
    EngineCtl ctl;
    int32_t ncond;
    int32_t has_sum;
    int32_t fast;                // every condition column is staged
    int32_t pad;
    Cond cond[TQP_MAX_PREDS];
    CondFast cf[TQP_MAX_PREDS];
    DExpr sum;
    int64_t* d_count;
    int64_t* d_count2;           // nullable: a second copy of the count
    int64_t* d_sum;              // nullable
    int64_t capacity;            // row-id capacity, for the CAPACITY latch
    uint32_t* mask;              // one ballot word per 32 rows; nullptr: count/sum only
    uint32_t* block_tot;         // passing rows per kCompactRows block (zeroed)
    unsigned long long* acc;     // [0] sum, [1] count, [2] completions (zeroed)
};

struct FilterBody {
    static constexpr int kMinBlocks = 2;
    // Per consumer warp: passing global row ids whose sum expression is still
    // to be evaluated (one step's <= 256 rows plus a partial round of < 32).
    static constexpr int kQueue = 8 * kWarp + kWarp;
    static constexpr int kSmemBytes = kConsumerWarps * kQueue * 4;

    const FilterArgs& A;
    uint32_t* q;
    int qn = 0;                     // queued rows (warp-uniform)
    long long my_sum = 0;
    unsigned long long my_cnt = 0;  // lane 0: rows passed by this warp

    __device__ FilterBody(const FilterArgs& a, unsigned char* sm) : A(a) {
        q = reinterpret_cast<uint32_t*>(sm) + (threadIdx.x / kWarp) * kQueue;
    }

    // Sparse passing rows: evaluate the expression 32 rows at a time with
    // global loads (the staged values are gone by then; the rows were streamed
    // moments ago, so their sectors are usually still in L2).
    __device__ __forceinline__ void drain(const ScanGeom& G, int lane, bool all) {
        int h = 0;
        while (qn - h >= kWarp) {
            my_sum += eval_expr_global(G, A.sum, q[h + lane]);
            h += kWarp;
        }
        if (all && qn > h) {
            if (lane < qn - h) my_sum += eval_expr_global(G, A.sum, q[h + lane]);
            h = qn;
        }
        if (h) {
            const uint32_t keep = lane < qn - h ? q[h + lane] : 0u;
            __syncwarp();
            if (lane < qn - h) q[lane] = keep;
            qn -= h;
            __syncwarp();
        }
    }

    // U rows per lane (32 U rows per warp) starting at tile row rbase.
    template <int U>
    __device__ __forceinline__ void step(const ScanGeom& G, const TileView& v, int rbase, int lane) {
        const uint32_t ok = eval_rows<U>(G, v, A.cf, A.cond, A.ncond, A.fast != 0, rbase + lane);
        uint32_t b[U];
        uint32_t cnt = 0;
#pragma unroll
        for (int j = 0; j < U; ++j) {
            b[j] = __ballot_sync(0xffffffffu, (ok >> j) & 1u);
            cnt += __popc(b[j]);
        }
        if (lane == 0) {
            my_cnt += cnt;
            if (A.mask) {
                const long long row = v.row0 + rbase;
#pragma unroll
                for (int j = 0; j < U; j += 4)
                    *reinterpret_cast<uint4*>(A.mask + row / kWarp + j) = make_uint4(b[j], b[j + 1], b[j + 2], b[j + 3]);
                if (cnt) atomicAdd(&A.block_tot[row / kCompactRows], cnt);
            }
        }
        if (A.has_sum && cnt) {
            if (cnt * 2 >= static_cast<uint32_t>(U * kWarp)) {
                // dense: every lane evaluates its own rows from the staged tile
#pragma unroll
                for (int j = 0; j < U; ++j)
                    if ((ok >> j) & 1u) my_sum += eval_expr(G, v, A.sum, rbase + kWarp * j + lane);
            } else {
                // sparse: queue the passing rows (in order), evaluate in full rounds
                const uint32_t lt = lanemask_lt();
                int pos = qn;
#pragma unroll
                for (int j = 0; j < U; ++j) {
                    if (b[j]) {
                        if ((b[j] >> lane) & 1u)
                            q[pos + __popc(b[j] & lt)] = static_cast<uint32_t>(v.row0 + rbase + kWarp * j + lane);
                        pos += __popc(b[j]);
                    }
                }
                qn = pos;
                __syncwarp();
                if (qn >= kWarp) drain(G, lane, false);
            }
        }
    }

    __device__ void pass1(const ScanGeom& G, const TileView& v, int cw, int lane) {
        const int rw = G.T / kConsumerWarps;  // a multiple of 128
        int r = 0;
        for (; r + 8 * kWarp <= rw; r += 8 * kWarp) {
            if (cw * rw + r >= v.rows) return;  // mask words wholly past the table end are never read
            step<8>(G, v, cw * rw + r, lane);
        }
        if (r < rw && cw * rw + r < v.rows) step<4>(G, v, cw * rw + r, lane);
    }

    __device__ void chunk_end(const ScanGeom& G, long long, long long, long long, int, int lane) {
        if (A.has_sum && qn) drain(G, lane, true);
        long long s = my_sum;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        my_sum = 0;
        if (lane == 0) {
            if (s) atomicAdd(&A.acc[0], static_cast<unsigned long long>(s));
            if (my_cnt) atomicAdd(&A.acc[1], my_cnt);
            my_cnt = 0;
            if (last_completion(&A.acc[2], A.ctl.nchunks)) {
                const unsigned long long tot_sum = atomicAdd(&A.acc[0], 0ULL);
                const unsigned long long tot_cnt = atomicAdd(&A.acc[1], 0ULL);
                *A.d_count = static_cast<int64_t>(tot_cnt);
                if (A.d_count2) *A.d_count2 = static_cast<int64_t>(tot_cnt);
                if (A.d_sum) *A.d_sum = static_cast<int64_t>(tot_sum);
                if (A.mask && static_cast<long long>(tot_cnt) > A.capacity) latch_error(A.ctl.err, TQP_ERR_CAPACITY);
            }
        }
    }

    __device__ void finish(const ScanGeom&, int, int) {}
};

// ---- group-by: warp pre-aggregation into the global table -------------------------

constexpr int kWarpSlots = 32;   // groups of a warp's collective cache
constexpr int kThrashAdds = 8;   // a cache refilled within this many adds is thrashing
constexpr int kFastSums = 4;     // sum accumulators of the closed-form fast path
constexpr int kLaneSlots = 8;    // groups of a warp's lane-private tables
constexpr int kLaneAcc = 4;      // accumulators (count + sums) the lane-private tables hold

struct GroupArgs {
    ScanGeom G;
    EngineCtl ctl;
    int32_t ncond;
    int32_t fast;
    Cond cond[TQP_MAX_PREDS];
    CondFast cf[TQP_MAX_PREDS];
    GroupSpec S;
    int32_t kfast;                          // full tiles: keys and sums straight from the stage
    int32_t pad;
    int32_t key_soff[TQP_MAX_GROUP_COLS];
    int32_t key_type[TQP_MAX_GROUP_COLS];
    ProdForm pf[kFastSums];                 // accumulator a + 1 in closed form
};

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Aggregation staged by locality (the paper reduces per group with a
// scatter-add, Section 5.4):
//   lane    while a warp has seen at most kLaneSlots distinct keys in the
//           chunk and the plan has at most kLaneAcc accumulators, every lane
//           adds its own rows into its own accumulators in shared memory,
//           laid out [group][accumulator][lane] (no bank conflicts, no
//           atomics, no warp collectives per row); group ids come from the
//           warp's key list, held in registers.  At chunk end the 32 lane
//           partials of each group are summed with shuffles and added to the
//           global table, one atomic per accumulator.
//   warp    otherwise lanes whose rows share a key are combined
//           (__match_any_sync, exact 64-bit sums through the warp reduction
//           unit) and the group's leader lane adds them to the warp's cache
//           of kWarpSlots groups, flushed to the global table when full and
//           at chunk end.  A warp whose key list overflows switches to this
//           mode for the rest of the chunk.
struct GroupBody {
    static constexpr int kLaneBytes = kLaneSlots * kLaneAcc * kWarp * 8;
    static constexpr int kCacheBytes = kWarpSlots * 8 + kWarpSlots * kMaxAcc * 8;  // aliases the lane area
    static constexpr int kAreaBytes = kLaneBytes > kCacheBytes ? kLaneBytes : kCacheBytes;
    static constexpr int kWarpBytes = kAreaBytes + kLaneSlots * 8 + 16;
    static constexpr int kSmemBytes = kConsumerWarps * kWarpBytes;
    static constexpr int kMinBlocks = 1;  // the lane tables leave room for one CTA per SM

    const GroupArgs& A;
    unsigned long long* area;    // lane mode: [kLaneSlots][kLaneAcc][32]; warp mode: keys[32], acc[32][kMaxAcc]
    unsigned long long* dkeys;   // lane mode: the warp's keys, in id order
    uint32_t* wocc;              // warp mode: occupancy bits of the cache slots
    uint64_t dk[kLaneSlots];     // lane mode: the warp's keys (the same in every lane)
    int nused = 0;               // lane mode: keys in dk (warp-uniform)
    int mode = 0;                // 0 lane, 1 warp, 2 direct (warp-uniform)
    int since = 0;               // warp mode: adds since the cache was last flushed
    int thrash = 0;              // warp mode: flushes that came within kThrashAdds adds
    bool kw32 = false;           // packed keys fit 32 bits
    // Full-tile fast path operands in registers (the argument block is in
    // shared memory, and the accumulator stores would force it to be re-read).
    static constexpr int kHotConds = 2;
    static constexpr int kHotSums = 3;
    HotCond hc[kHotConds];
    HotProd hp[kHotSums];
    uint32_t hk[TQP_MAX_GROUP_COLS];  // key columns
    int hncond = 0, hngc = 0, hnsum = 0;

    __device__ GroupBody(const GroupArgs& a, unsigned char* sm) : A(a) {
        const int w = threadIdx.x / kWarp;
        const int ww = w < kConsumerWarps ? w : 0;
        area = reinterpret_cast<unsigned long long*>(sm + ww * kWarpBytes);
        dkeys = area + kAreaBytes / 8;
        wocc = reinterpret_cast<uint32_t*>(dkeys + kLaneSlots);
        uint4* z = reinterpret_cast<uint4*>(sm);
        for (int i = threadIdx.x; i < kSmemBytes / 16; i += blockDim.x) z[i] = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int d = 0; d < kLaneSlots; ++d) dk[d] = 0;
        mode = A.S.nacc <= kLaneAcc ? 0 : 1;
        kw32 = A.S.width <= 32;
        if (A.kfast) {
            hncond = A.ncond;
            hngc = A.S.ngc;
            hnsum = A.S.nacc - 1;
#pragma unroll
            for (int q = 0; q < kHotConds; ++q)
                if (q < hncond) hc[q].load(A.cf[q]);
#pragma unroll
            for (int i = 0; i < TQP_MAX_GROUP_COLS; ++i)
                hk[i] = i < hngc ? hot_desc(A.key_soff[i], A.key_type[i], 0, 0) : 0u;
#pragma unroll
            for (int a2 = 0; a2 < kHotSums; ++a2)
                if (a2 < hnsum) hp[a2].load(A.pf[a2]);
        }
    }

    // ---- lane mode ----

    // Every group's lane partials into the global table; the tables are empty afterwards.
    __device__ __forceinline__ void flush_lanes(int lane) {
        __syncwarp();
        const GroupSpec& S = A.S;
        const long long gl = lane < nused ? gtab_slot(S, dkeys[lane], A.ctl.err) : -1;
        for (int d = 0; d < nused; ++d) {
            const long long g = __shfl_sync(0xffffffffu, gl, d);
#pragma unroll
            for (int a = 0; a < kLaneAcc; ++a) {
                if (a < S.nacc) {
                    unsigned long long* p = area + (d * kLaneAcc + a) * kWarp + lane;
                    const unsigned long long x = warp_sum_u64(*p);
                    *p = 0;
                    if (lane == 0 && x && g >= 0) red_add_u64(&S.acc[g * S.nacc + a], x);
                }
            }
        }
        nused = 0;
        __syncwarp();
    }

    // Rows of one lane each into the lane tables; false (nothing added) when
    // the warp's key list overflows: the caller switches to warp mode.
    __device__ __forceinline__ bool lane_add(bool act, uint64_t key, const int64_t (&val)[kFastSums], int lane) {
        int id = -1;
        if (kw32) {  // packed keys of at most 32 bits compare in 32 bits
            const uint32_t k = static_cast<uint32_t>(key);
#pragma unroll
            for (int d = 0; d < kLaneSlots; ++d)
                if (d < nused && k == static_cast<uint32_t>(dk[d])) id = d;
        } else {
#pragma unroll
            for (int d = 0; d < kLaneSlots; ++d)
                if (d < nused && key == dk[d]) id = d;
        }
        bool miss = act && id < 0;
        while (__any_sync(0xffffffffu, miss)) {
            if (nused == kLaneSlots) return false;
            const int src = __ffs(__ballot_sync(0xffffffffu, miss)) - 1;
            const uint64_t k = __shfl_sync(0xffffffffu, key, src);
#pragma unroll
            for (int d = 0; d < kLaneSlots; ++d)
                if (d == nused) dk[d] = k;
            if (lane == 0) dkeys[nused] = k;
            if (miss && key == k) {
                id = nused;
                miss = false;
            }
            ++nused;
        }
        if (act) {
            unsigned long long* p = area + id * (kLaneAcc * kWarp) + lane;
            p[0] += 1;
#pragma unroll
            for (int a = 0; a < kLaneAcc - 1; ++a)
                if (a + 1 < A.S.nacc) p[(a + 1) * kWarp] += static_cast<unsigned long long>(val[a]);
        }
        return true;
    }

    // The U rows of every lane (pass bits `ok`) into the lane tables at once:
    // ids first, rows of one lane with the same id folded together, then the
    // accumulators read, summed and written with the addresses of a lane's
    // rows all distinct -- independent chains instead of one serial
    // read-modify-write per row.  False (nothing added) if the key list
    // overflows.
    template <int U>
    __device__ __forceinline__ bool lane_step(uint32_t ok, const uint64_t (&key)[U], int64_t (&val)[kFastSums][U],
                                              int lane) {
        int id[U];
        bool miss = false;
#pragma unroll
        for (int j = 0; j < U; ++j) {
            id[j] = -1;
            if (kw32) {
                const uint32_t k = static_cast<uint32_t>(key[j]);
#pragma unroll
                for (int d = 0; d < kLaneSlots; ++d)
                    if (d < nused && k == static_cast<uint32_t>(dk[d])) id[j] = d;
            } else {
#pragma unroll
                for (int d = 0; d < kLaneSlots; ++d)
                    if (d < nused && key[j] == dk[d]) id[j] = d;
            }
            miss |= ((ok >> j) & 1u) && id[j] < 0;
        }
        if (__any_sync(0xffffffffu, miss)) {  // new keys: extend the warp's list, row by row (rare)
#pragma unroll
            for (int j = 0; j < U; ++j) {
                bool m = ((ok >> j) & 1u) && id[j] < 0;
                while (__any_sync(0xffffffffu, m)) {
                    if (nused == kLaneSlots) return false;
                    const int src = __ffs(__ballot_sync(0xffffffffu, m)) - 1;
                    const uint64_t k = __shfl_sync(0xffffffffu, key[j], src);
#pragma unroll
                    for (int d = 0; d < kLaneSlots; ++d)
                        if (d == nused) dk[d] = k;
                    if (lane == 0) dkeys[nused] = k;
#pragma unroll
                    for (int i = 0; i < U; ++i)
                        if (((ok >> i) & 1u) && id[i] < 0 && key[i] == k) id[i] = nused;
                    ++nused;
                    m = ((ok >> j) & 1u) && id[j] < 0;
                }
            }
        }
        // fold rows of this lane that share a group
        uint32_t act = ok;
        unsigned long long cnt[U];
#pragma unroll
        for (int j = 0; j < U; ++j) cnt[j] = 1;
#pragma unroll
        for (int j = 1; j < U; ++j) {
            bool done = false;
#pragma unroll
            for (int k = 0; k < j; ++k) {
                if (!done && ((act >> k) & 1u) && ((act >> j) & 1u) && id[k] == id[j]) {
                    cnt[k] += cnt[j];
#pragma unroll
                    for (int a = 0; a < kFastSums; ++a) val[a][k] += val[a][j];
                    act &= ~(1u << j);
                    done = true;
                }
            }
        }
        const int nacc = A.S.nacc;
        unsigned long long* p[U];
#pragma unroll
        for (int j = 0; j < U; ++j) p[j] = area + (id[j] < 0 ? 0 : id[j]) * (kLaneAcc * kWarp) + lane;
#pragma unroll
        for (int a = 0; a < kLaneAcc; ++a) {
            if (a < nacc) {
                unsigned long long old[U];
#pragma unroll
                for (int j = 0; j < U; ++j)
                    if ((act >> j) & 1u) old[j] = p[j][a * kWarp];
#pragma unroll
                for (int j = 0; j < U; ++j)
                    if ((act >> j) & 1u)
                        p[j][a * kWarp] = old[j] + (a == 0 ? cnt[j] : static_cast<unsigned long long>(val[a - 1][j]));
            }
        }
        return true;
    }

    // ---- warp mode ----

    // Every cached group into the global table; the cache is empty (and the
    // area all zero) afterwards.
    __device__ __forceinline__ void flush_cache(int lane) {
        __syncwarp();
        const uint32_t occ = *reinterpret_cast<volatile uint32_t*>(wocc);
        const GroupSpec& S = A.S;
        unsigned long long* wkeys = area;
        unsigned long long* wacc = area + kWarpSlots;
        if ((occ >> lane) & 1u) {
            const long long g = gtab_slot(S, wkeys[lane], A.ctl.err);
            for (int a = 0; a < S.nacc; ++a) {
                const unsigned long long x = wacc[lane * kMaxAcc + a];
                if (x && g >= 0) red_add_u64(&S.acc[g * S.nacc + a], x);
                wacc[lane * kMaxAcc + a] = 0;
            }
        }
        wkeys[lane] = 0;
        __syncwarp();
        if (lane == 0) *wocc = 0;
        __syncwarp();
    }

    // Warp-collective: the cache slot of each leader's key (claimed if new;
    // the cache is flushed first if some leader finds no free slot).
    __device__ __forceinline__ int slot_of(bool lead, uint64_t key, int lane) {
        unsigned long long* wkeys = area;
        const unsigned h0 = static_cast<unsigned>(mix64(key)) & (kWarpSlots - 1);
        unsigned h = h0;
        int s = -1, tries = 0;
        while (true) {
            const bool need = lead && s < 0;
            if (!__any_sync(0xffffffffu, need)) break;
            if (need) {
                const uint32_t occ = *reinterpret_cast<volatile uint32_t*>(wocc);
                if ((occ >> h) & 1u) {
                    if (wkeys[h] == key) s = static_cast<int>(h);
                } else if (!((atomicOr(wocc, 1u << h) >> h) & 1u)) {
                    wkeys[h] = key;
                    s = static_cast<int>(h);
                }
                if (s < 0) {
                    h = (h + 1) & (kWarpSlots - 1);
                    ++tries;
                }
            }
            __syncwarp();
            if (__any_sync(0xffffffffu, need && s < 0 && tries >= kWarpSlots)) {
                flush_cache(lane);  // all leaders start over in an empty cache
                thrash += since < kThrashAdds ? 1 : 0;
                since = 0;
                s = -1;
                tries = 0;
                h = h0;
            }
        }
        return s;
    }

    // Lanes with act set hold one row each (key, count 1, sums val[0..nsum)).
    template <int NS>
    __device__ __forceinline__ void warp_add(bool act, uint64_t key, const int64_t (&val)[NS], int nsum, int lane) {
        const uint32_t actm = __ballot_sync(0xffffffffu, act);
        if (!actm) return;
        const uint32_t peers = __match_any_sync(0xffffffffu, key) & actm;
        const bool lead = act && lane == __ffs(peers) - 1;
        const int s = slot_of(lead, key, lane);
        if (!act) return;
        unsigned long long* a = area + kWarpSlots + (s < 0 ? 0 : s) * kMaxAcc;
        if (lead) a[0] += __popc(peers);
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            if (i < nsum) {
                const long long x = group_sum_i64(peers, val[i]);
                if (lead) a[i + 1] += static_cast<unsigned long long>(x);
            }
        }
    }

    // Direct mode (keys too many for the cache: it refilled within a few adds,
    // twice): each row goes straight into the global table.  Rows are not
    // summed per key within the warp first: with keys this spread few rows
    // share one, and a reduction over lane groups with different masks
    // proceeds one group at a time.
    template <int NS>
    __device__ __forceinline__ void direct_add(bool act, uint64_t key, const int64_t (&val)[NS], int nsum) {
        if (!act) return;
        const GroupSpec& S = A.S;
        const long long g = gtab_slot(S, key, A.ctl.err);
        if (g < 0) return;
        unsigned long long* acc = S.acc + g * S.nacc;
        red_add_u64(acc, 1ULL);
#pragma unroll
        for (int i = 0; i < NS; ++i)
            if (i < nsum && val[i]) red_add_u64(acc + 1 + i, static_cast<unsigned long long>(val[i]));
    }

    // One row per lane (act: the row passed) in the warp's current mode.
    template <int NS>
    __device__ __forceinline__ void add(bool act, uint64_t key, const int64_t (&val)[NS], int lane) {
        const int nsum = A.S.nacc - 1;
        if (mode == 2) {
            direct_add<NS>(act, key, val, nsum);
            return;
        }
        if (mode == 0) {
            int64_t v4[kFastSums];
#pragma unroll
            for (int i = 0; i < kFastSums; ++i) v4[i] = i < NS ? val[i < NS ? i : 0] : 0;
            if (lane_add(act, key, v4, lane)) return;
            flush_lanes(lane);  // key list full: warp mode for the rest of the chunk
            mode = 1;
        }
        warp_add<NS>(act, key, val, nsum, lane);
        ++since;
        if (thrash >= 2) {  // the cache keeps refilling: direct mode for the rest of the chunk
            flush_cache(lane);
            mode = 2;
        }
    }

    // Full tile, closed-form sums: U rows per lane, operands from registers.
    template <int U>
    __device__ __forceinline__ void step_fast(const TileView& v, int rbase, int lane) {
        const int r0 = rbase + lane;
        uint32_t ok = (1u << U) - 1u;
#pragma unroll
        for (int q = 0; q < kHotConds; ++q)
            if (q < hncond) ok &= hc[q].template eval<U>(v.stage, r0);
        if (hncond > kHotConds) ok &= conds_full<U>(v.stage, A.cf + kHotConds, hncond - kHotConds, r0);
        if (!__any_sync(0xffffffffu, ok)) return;
        uint64_t key[U];
#pragma unroll
        for (int j = 0; j < U; ++j) key[j] = 0;
#pragma unroll
        for (int i = 0; i < TQP_MAX_GROUP_COLS; ++i) {
            if (i >= hngc) break;
            int64_t x[U];
            const int t = (hk[i] >> 20) & 3;
            load_rows<U>(v.stage + (hk[i] & 0xFFFFFu), t, r0, x);
            if (t == TQP_U8) {
#pragma unroll
                for (int j = 0; j < U; ++j) key[j] = (key[j] << 8) | (static_cast<uint64_t>(x[j]) & 0xFFu);
            } else if (t == TQP_I32) {
#pragma unroll
                for (int j = 0; j < U; ++j)
                    key[j] = (key[j] << 32) | static_cast<uint64_t>(static_cast<uint32_t>(x[j]) ^ 0x80000000u);
            } else {
#pragma unroll
                for (int j = 0; j < U; ++j) key[j] = static_cast<uint64_t>(x[j]) ^ 0x8000000000000000ull;
            }
        }
        int64_t val[kFastSums][U];
#pragma unroll
        for (int a = 0; a < kFastSums; ++a) {
            if (a < hnsum) {
                if (a < kHotSums) hp[a < kHotSums ? a : 0].template eval<U>(v.stage, r0, val[a]);
                else prod_eval<U>(A.pf[a], v.stage, r0, val[a]);
            } else {
#pragma unroll
                for (int j = 0; j < U; ++j) val[a][j] = 0;
            }
        }
        if (mode == 0) {
            if (lane_step<U>(ok, key, val, lane)) return;
            flush_lanes(lane);  // key list full: warp mode for the rest of the chunk
            mode = 1;
        }
#pragma unroll
        for (int j = 0; j < U; ++j) {
            int64_t vj[kFastSums];
#pragma unroll
            for (int a = 0; a < kFastSums; ++a) vj[a] = val[a][j];
            add<kFastSums>((ok >> j) & 1u, key[j], vj, lane);
        }
    }

    // Any tile and expression: one row per lane, interpreted.
    __device__ __forceinline__ void step_general(const ScanGeom& G, const TileView& v, int r, bool act, int lane) {
        const GroupSpec& S = A.S;
        uint64_t key = 0;
        int64_t vals[kMaxAcc - 1];
#pragma unroll
        for (int i = 0; i < kMaxAcc - 1; ++i) vals[i] = 0;
        if (act) {
            key = pack_key(S, G, v, r);
#pragma unroll
            for (int i = 0; i < kMaxAcc - 1; ++i)
                if (i < S.nacc - 1) vals[i] = eval_expr(G, v, S.acc_expr[i], r);
        }
        add<kMaxAcc - 1>(act, key, vals, lane);
    }

    __device__ void pass1(const ScanGeom& G, const TileView& v, int cw, int lane) {
        const int rw = G.T / kConsumerWarps;  // a multiple of 128
        if (A.kfast && A.fast && v.full) {
            for (int r = 0; r < rw; r += kUnroll * kWarp) step_fast<kUnroll>(v, cw * rw + r, lane);
            return;
        }
        for (int r = 0; r < rw; r += kUnroll * kWarp) {
            const int rbase = cw * rw + r;
            if (rbase >= v.rows) break;
            const uint32_t ok = eval_rows<kUnroll>(G, v, A.cf, A.cond, A.ncond, A.fast != 0, rbase + lane);
#pragma unroll
            for (int j = 0; j < kUnroll; ++j)
                if (__any_sync(0xffffffffu, (ok >> j) & 1u))
                    step_general(G, v, rbase + kWarp * j + lane, (ok >> j) & 1u, lane);
        }
    }

    __device__ void chunk_end(const ScanGeom&, long long, long long, long long, int, int lane) {
        if (mode == 0) flush_lanes(lane);
        else if (mode == 1) flush_cache(lane);
        mode = A.S.nacc <= kLaneAcc ? 0 : 1;
        since = 0;
        thrash = 0;
    }

    __device__ void finish(const ScanGeom&, int, int) {}
};

// Host: fill the fast-path fields of A from its geometry (kfast = 0 when the
// keys or sums are not all staged, or the sums are not in closed form).
void lower_group_fast(GroupArgs* A);

// ---- joined plan: filter + probe + aggregate into dense group accumulators --------

struct PlanJoinArgs {
    ScanGeom G;
    EngineCtl ctl;
    int32_t ncond;
    int32_t fast;
    Cond cond[TQP_MAX_PREDS];
    CondFast cf[TQP_MAX_PREDS];
    int32_t fk_col;
    int32_t has_sum;
    DExpr sum;
    JoinHT H;
    const uint32_t* next;      // chained build: next dim row of the same key
    const uint32_t* dgs;       // dim row -> dense group id; nullptr: no aggregation
    GroupSpec S;
    unsigned long long* acc;   // [0] joined, [1] sum, [2] passing fact rows, [3] completions (zeroed)
    int64_t* d_num_joined;
    int64_t* d_sum;
    int64_t* d_num_rows;
    // full-tile fast path: foreign key and sums read straight from the stage
    int32_t pjfast;
    int32_t fk_soff;
    int32_t fk_type;
    int32_t nsum;              // accumulators after the count (S.nacc - 1)
    ProdForm psum;             // the ungrouped sum
    ProdForm pacc[kFastSums];  // accumulator a + 1
    // Aggregation by join key first (direct-mapped tables, full tiles): each
    // fact row adds to its key's entry kacc[(fk - min) * nk + i] (count, the
    // group sums, then the ungrouped sum), and a second kernel folds every
    // dimension row's key entry into its group.  nullptr: off.
    unsigned long long* kacc;
    int32_t nk;
};

struct PlanJoinBody {
    // One CTA per SM: the probe keeps its rows' slot loads, keys and sums in
    // registers, more than two 9-warp CTAs per SM leave (96 per thread).
    static constexpr int kMinBlocks = 1;
    static constexpr int kSmemBytes = 0;
    static constexpr int kJoinSums = 2; // sums of the fast path
    const PlanJoinArgs& A;
    unsigned long long joined = 0, passed = 0;
    long long sum = 0;

    __device__ PlanJoinBody(const PlanJoinArgs& a, unsigned char*) : A(a) {}

    // Accumulator i + 1 of a group: a sum, or the atomic maximum of a MIN/MAX code.
    __device__ __forceinline__ void acc_update(unsigned long long* a, int i, int64_t x) const {
        const int kind = A.S.acc_kind[i];
        if (kind == kAccSum) red_add_u64(&a[i + 1], static_cast<unsigned long long>(x));
        else atomicMax(&a[i + 1], acc_encode(kind, x));
    }

    // Add one joined row (count `cnt` matches, values x[]) to the group(s) of its slot.
    __device__ __forceinline__ void add_groups(const uint4& sl, const int64_t (&x)[kFastSums], int nsum) {
        const GroupSpec& S = A.S;
        if (sl.z & kDirectGroup) {  // a unique key whose dense group id sits in the slot
            unsigned long long* a = S.acc + static_cast<long long>(sl.z & ~kDirectGroup) * S.nacc;
            red_add_u64(&a[0], 1ULL);
#pragma unroll
            for (int i = 0; i < kFastSums; ++i)
                if (i < nsum) acc_update(a, i, x[i]);
            return;
        }
        uint32_t d = sl.z;
        for (uint32_t k = 0; k < sl.w; ++k) {
            unsigned long long* a = S.acc + static_cast<long long>(__ldg(&A.dgs[d])) * S.nacc;
            red_add_u64(&a[0], 1ULL);
#pragma unroll
            for (int i = 0; i < kFastSums; ++i)
                if (i < nsum) acc_update(a, i, x[i]);
            if (k + 1 < sl.w) d = __ldg(&A.next[d]);
        }
    }

    // Aggregate one joined fact row r into its slot's group(s) (general path).
    __device__ __forceinline__ void aggregate(const ScanGeom& G, const TileView& v, int r, const uint4& sl) {
        const uint32_t cnt = sl.w;
        joined += cnt;
        if (A.has_sum) sum += eval_expr(G, v, A.sum, r) * static_cast<long long>(cnt);
        if (!A.dgs) return;
        const GroupSpec& S = A.S;
        if (S.nacc - 1 <= kFastSums) {
            int64_t x[kFastSums];
#pragma unroll
            for (int i = 0; i < kFastSums; ++i) x[i] = i < S.nacc - 1 ? eval_expr(G, v, S.acc_expr[i], r) : 0;
            add_groups(sl, x, S.nacc - 1);
            return;
        }
        uint32_t d = sl.z;
        const bool direct_group = (sl.z & kDirectGroup) != 0;
        for (uint32_t k = 0; k < cnt; ++k) {
            const long long g = direct_group ? static_cast<long long>(sl.z & ~kDirectGroup) : __ldg(&A.dgs[d]);
            unsigned long long* a = S.acc + g * S.nacc;
            red_add_u64(&a[0], 1ULL);
            for (int i = 1; i < S.nacc; ++i) acc_update(a, i - 1, eval_expr(G, v, S.acc_expr[i - 1], r));
            if (!direct_group && k + 1 < cnt) d = __ldg(&A.next[d]);
        }
    }

    // Slot index of key (hashed tables: the home slot; the caller probes on).
    __device__ __forceinline__ unsigned long long home(uint64_t key, bool direct, long long kmin, bool& in) const {
        if (direct) {
            const unsigned long long s = key - static_cast<uint64_t>(kmin);
            in = s < static_cast<unsigned long long>(A.H.cap);
            return in ? s : 0;
        }
        in = true;
        return key == ~0ULL ? static_cast<unsigned long long>(A.H.cap)
                            : (mix64(key) & static_cast<unsigned long long>(A.H.cap - 1));
    }

    // The matching slot of `key` given its home slot's contents (w = 0: no match).
    __device__ __forceinline__ uint4 resolve(uint64_t key, bool direct, unsigned long long hh, uint4 s) const {
        if (direct || key == ~0ULL) return s;  // direct: the slot is the key's; ~0 lives in the extra slot
        const unsigned long long mask = static_cast<unsigned long long>(A.H.cap - 1);
        for (long long i = 0; i < A.H.cap; ++i) {
            const uint64_t k = slot_key(s);
            if (k == key) return s;
            if (k == ~0ULL) break;
            hh = (hh + 1) & mask;
            s = __ldg(&A.H.slots[hh]);
        }
        return make_uint4(0u, 0u, 0u, 0u);
    }

    // Full tile: kU rows per lane, foreign keys and sums from the stage, the
    // rows' slot loads in flight together.  Hot arguments are read into
    // registers once per tile (the argument block lives in shared memory).
    template <int kU>
    __device__ __forceinline__ void step_fast(const TileView& v, int rbase, bool direct, long long kmin,
                                              const uint4* __restrict__ slots, long long cap,
                                              unsigned long long* __restrict__ gacc, int nacc, bool has_sum,
                                              bool grouped, unsigned long long* __restrict__ kacc,
                                              unsigned long long krange) {
        const int r0 = rbase + (threadIdx.x % kWarp);
        const uint32_t ok = conds_full<kU>(v.stage, A.cf, A.ncond, r0);
        if (!__any_sync(0xffffffffu, ok)) return;
        int64_t fk[kU];
        load_rows<kU>(v.stage + A.fk_soff, A.fk_type, r0, fk);
        if (kacc) {  // by join key: no slot load; the fold adds the matches to their groups
            passed += __popc(ok);
            int64_t sv[kU];
            if (has_sum) prod_eval<kU>(A.psum, v.stage, r0, sv);
            int64_t xv[kJoinSums][kU];
#pragma unroll
            for (int i = 0; i < kJoinSums; ++i)
                if (i < nacc - 1) prod_eval<kU>(A.pacc[i], v.stage, r0, xv[i]);
            const int nk = A.nk;
#pragma unroll
            for (int j = 0; j < kU; ++j) {
                const unsigned long long e = static_cast<uint64_t>(fk[j]) - static_cast<uint64_t>(kmin);
                if (!((ok >> j) & 1u) || e >= krange) continue;
                unsigned long long* a = kacc + e * nk;
                red_add_u64(&a[0], 1ULL);
#pragma unroll
                for (int i = 0; i < kJoinSums; ++i)
                    if (i < nacc - 1) red_add_u64(&a[i + 1], static_cast<unsigned long long>(xv[i][j]));
                if (has_sum) red_add_u64(&a[nacc], static_cast<unsigned long long>(sv[j]));
            }
            return;
        }
        unsigned long long hh[kU];
        uint4 sl[kU];
#pragma unroll
        for (int j = 0; j < kU; ++j) {
            const uint64_t key = static_cast<uint64_t>(fk[j]);
            bool in;
            if (direct) {
                hh[j] = key - static_cast<uint64_t>(kmin);
                in = hh[j] < static_cast<unsigned long long>(cap);
            } else {
                hh[j] = key == ~0ULL ? static_cast<unsigned long long>(cap)
                                     : (mix64(key) & static_cast<unsigned long long>(cap - 1));
                in = true;
            }
            sl[j] = make_uint4(0u, 0u, 0u, 0u);
            if (((ok >> j) & 1u) && in) sl[j] = __ldg(&slots[hh[j]]);
        }
        passed += __popc(ok);
        int64_t sv[kU];
        if (has_sum) prod_eval<kU>(A.psum, v.stage, r0, sv);
        int64_t xv[kJoinSums][kU];
#pragma unroll
        for (int i = 0; i < kJoinSums; ++i)
            if (grouped && i < nacc - 1) prod_eval<kU>(A.pacc[i], v.stage, r0, xv[i]);
#pragma unroll
        for (int j = 0; j < kU; ++j) {
            if (!((ok >> j) & 1u)) continue;
            const uint4 s = resolve(static_cast<uint64_t>(fk[j]), direct, hh[j], sl[j]);
            if (!s.w) continue;
            joined += s.w;
            if (has_sum) sum += sv[j] * static_cast<long long>(s.w);
            if (!grouped) continue;
            if (s.z & kDirectGroup) {
                unsigned long long* a = gacc + static_cast<long long>(s.z & ~kDirectGroup) * nacc;
                red_add_u64(&a[0], 1ULL);
#pragma unroll
                for (int i = 0; i < kJoinSums; ++i)
                    if (i < nacc - 1) red_add_u64(&a[i + 1], static_cast<unsigned long long>(xv[i][j]));
            } else {
                int64_t x[kFastSums];
#pragma unroll
                for (int i = 0; i < kFastSums; ++i) x[i] = i < kJoinSums ? xv[i < kJoinSums ? i : 0][j] : 0;
                add_groups(s, x, nacc - 1);
            }
        }
    }

    __device__ void pass1(const ScanGeom& G, const TileView& v, int cw, int lane) {
        const int rw = G.T / kConsumerWarps;
        long long kmin = 0;
        const bool direct = ht_is_direct(A.H, &kmin);
        if (A.pjfast && A.fast && v.full) {
            const uint4* slots = A.H.slots;
            const long long cap = A.H.cap;
            unsigned long long* gacc = A.S.acc;
            const int nacc = A.S.nacc;
            const bool has_sum = A.has_sum != 0, grouped = A.dgs != nullptr;
            unsigned long long* kacc = direct ? A.kacc : nullptr;
            const unsigned long long krange = kacc ? static_cast<unsigned long long>(__ldg(&A.H.meta[1]) - kmin) + 1 : 0;
            // rw is a multiple of 128 = kUnroll * 32
            for (int r = 0; r < rw; r += kUnroll * kWarp)
                step_fast<kUnroll>(v, cw * rw + r, direct, kmin, slots, cap, gacc, nacc, has_sum, grouped, kacc,
                                   krange);
            return;
        }
        for (int r = 0; r < rw; r += kUnroll * kWarp) {
            const int rbase = cw * rw + r;
            if (rbase >= v.rows) break;
            const uint32_t ok = eval_rows<kUnroll>(G, v, A.cf, A.cond, A.ncond, A.fast != 0, rbase + lane);
            uint64_t key[kUnroll];
            unsigned long long h[kUnroll];
            uint4 sl[kUnroll];
#pragma unroll
            for (int j = 0; j < kUnroll; ++j) {
                key[j] = 0;
                h[j] = 0;
                sl[j] = make_uint4(0u, 0u, 0u, 0u);
                if ((ok >> j) & 1u) {
                    key[j] = static_cast<uint64_t>(col_val(G, v, A.fk_col, rbase + kWarp * j + lane));
                    bool in = false;
                    h[j] = home(key[j], direct, kmin, in);
                    if (in) sl[j] = __ldg(&A.H.slots[h[j]]);
                }
            }
#pragma unroll
            for (int j = 0; j < kUnroll; ++j) {
                if (!((ok >> j) & 1u)) continue;
                ++passed;
                const uint4 s = resolve(key[j], direct, h[j], sl[j]);
                if (s.w) aggregate(G, v, rbase + kWarp * j + lane, s);
            }
        }
    }

    __device__ void chunk_end(const ScanGeom&, long long, long long, long long, int, int lane) {
        unsigned long long j = joined, p = passed;
        long long s = sum;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            j += __shfl_xor_sync(0xffffffffu, j, o);
            p += __shfl_xor_sync(0xffffffffu, p, o);
            s += __shfl_xor_sync(0xffffffffu, s, o);
        }
        joined = passed = 0;
        sum = 0;
        if (lane == 0) {
            if (j) atomicAdd(&A.acc[0], j);
            if (s) atomicAdd(&A.acc[1], static_cast<unsigned long long>(s));
            if (p) atomicAdd(&A.acc[2], p);
            if (last_completion(&A.acc[3], A.ctl.nchunks)) {
                long long kmin;
                const bool folded = A.kacc && ht_is_direct(A.H, &kmin);  // the fold writes joined and sum
                if (A.d_num_joined && !folded) *A.d_num_joined = static_cast<int64_t>(atomicAdd(&A.acc[0], 0ULL));
                if (A.d_sum && !folded) *A.d_sum = static_cast<int64_t>(atomicAdd(&A.acc[1], 0ULL));
                if (A.d_num_rows) *A.d_num_rows = static_cast<int64_t>(atomicAdd(&A.acc[2], 0ULL));
            }
        }
    }

    __device__ void finish(const ScanGeom&, int, int) {}
};

// Host: fill the fast-path fields of A from its geometry (pjfast = 0 when the
// foreign key or a summed column is not staged or a sum is not in closed form).
void lower_join_fast(PlanJoinArgs* A);

// Fold the key-first accumulators into the groups: every dimension row adds
// its key's entry (the fact rows that matched it) to its group, and to the
// joined-pair count and the ungrouped sum (acc[0], acc[1]).  Block vb of vg;
// the last block to finish (counted in acc[4]) writes those two results.
// Nothing to do for a hashed table: the probe aggregated by group.
constexpr int kFoldThreads = 256;
__device__ __forceinline__ void keyfirst_fold_block(const JoinHT& H, const unsigned char* dkey, int dkey_type,
                                                    long long nd, const uint32_t* dgs, const GroupSpec& S,
                                                    const unsigned long long* kacc, int nk, int has_sum,
                                                    unsigned long long* acc, int64_t* d_num_joined, int64_t* d_sum,
                                                    long long vb, long long vg) {
    long long kmin;
    if (!ht_is_direct(H, &kmin)) return;
    const unsigned long long krange = static_cast<unsigned long long>(__ldg(&H.meta[1]) - kmin) + 1;
    unsigned long long joined = 0;
    long long sum = 0;
    for (long long d = vb * kFoldThreads + threadIdx.x; d < nd; d += vg * kFoldThreads) {
        const unsigned long long e =
            static_cast<uint64_t>(ldg_typed(dkey, dkey_type, d)) - static_cast<uint64_t>(kmin);
        if (e >= krange) continue;
        const unsigned long long* a = kacc + e * nk;
        const unsigned long long c = __ldg(&a[0]);
        if (!c) continue;
        unsigned long long* ga = S.acc + static_cast<long long>(__ldg(&dgs[d])) * S.nacc;
        red_add_u64(&ga[0], c);
        for (int i = 1; i < S.nacc; ++i) red_add_u64(&ga[i], __ldg(&a[i]));
        joined += c;
        if (has_sum) sum += static_cast<long long>(__ldg(&a[S.nacc]));
    }
    __shared__ unsigned long long rj[kFoldThreads / 32];
    __shared__ long long rs[kFoldThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        joined += __shfl_xor_sync(0xffffffffu, joined, o);
        sum += __shfl_xor_sync(0xffffffffu, sum, o);
    }
    if (threadIdx.x % 32 == 0) {
        rj[threadIdx.x / 32] = joined;
        rs[threadIdx.x / 32] = sum;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int w = 1; w < kFoldThreads / 32; ++w) {
        joined += rj[w];
        sum += rs[w];
    }
    if (joined) atomicAdd(&acc[0], joined);
    if (sum) atomicAdd(&acc[1], static_cast<unsigned long long>(sum));
    __threadfence();
    if (atomicAdd(&acc[4], 1ULL) != static_cast<unsigned long long>(vg) - 1ULL) return;
    __threadfence();
    if (d_num_joined) *d_num_joined = static_cast<int64_t>(atomicAdd(&acc[0], 0ULL));
    if (d_sum) *d_sum = static_cast<int64_t>(atomicAdd(&acc[1], 0ULL));
}

// ---- selection-mask expansion (second filter kernel) ------------------------------

// Expand the selection mask of rows [b * kCompactRows, ...) into row ids.
// Called by a whole block of kCompactThreads threads for mask block b: each
// thread takes two consecutive mask words (64 rows), one block-wide exclusive
// scan of their bit counts gives every thread its output offset, and each
// thread writes the ids of its own set bits (ascending, so the output is).
__device__ __forceinline__ void compact_block(const uint32_t* __restrict__ mask, const uint32_t* __restrict__ block_tot,
                                              long long n, int32_t* __restrict__ row_ids, long long capacity,
                                              long long b) {
    static_assert(kCompactWords == 2 * kCompactThreads, "two mask words per thread");
    constexpr int W = kCompactThreads / kWarp;
    __shared__ unsigned long long red[W];
    __shared__ uint32_t wsum[W];
    const int lane = threadIdx.x % kWarp, w = threadIdx.x / kWarp;
    // offset of this block: every earlier block's total
    unsigned long long before_blocks = 0;
    for (long long i = threadIdx.x; i < b; i += kCompactThreads) before_blocks += block_tot[i];
    // this thread's two words
    const long long nwords = (n + kWarp - 1) / kWarp;
    const long long wi = b * kCompactWords + 2 * threadIdx.x;
    const uint32_t m0 = wi < nwords ? mask[wi] : 0u;
    const uint32_t m1 = wi + 1 < nwords ? mask[wi + 1] : 0u;
    const uint32_t c = __popc(m0) + __popc(m1);
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < kWarp; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) before_blocks += __shfl_xor_sync(0xffffffffu, before_blocks, o);
    if (lane == kWarp - 1) wsum[w] = incl;
    if (lane == 0) red[w] = before_blocks;
    __syncthreads();
    unsigned long long base = 0;
    uint32_t before_warps = 0;
#pragma unroll
    for (int i = 0; i < W; ++i) {
        base += red[i];
        before_warps += i < w ? wsum[i] : 0u;
    }
    unsigned long long pos = base + before_warps + (incl - c);
    const long long row0 = wi * kWarp;
    uint32_t m = m0;
    while (m) {
        const int bit = __ffs(m) - 1;
        m &= m - 1;
        if (pos < static_cast<unsigned long long>(capacity)) row_ids[pos] = static_cast<int32_t>(row0 + bit);
        ++pos;
    }
    m = m1;
    while (m) {
        const int bit = __ffs(m) - 1;
        m &= m - 1;
        if (pos < static_cast<unsigned long long>(capacity)) row_ids[pos] = static_cast<int32_t>(row0 + kWarp + bit);
        ++pos;
    }
}

}  // namespace tqp
