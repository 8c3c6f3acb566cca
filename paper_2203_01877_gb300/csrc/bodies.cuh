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
constexpr int kCompactThreads = 256;

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

// ---- group-by: shared-memory pre-aggregation into the global table ---------------

struct GroupArgs {
    ScanGeom G;
    EngineCtl ctl;
    int32_t ncond;
    int32_t fast;
    Cond cond[TQP_MAX_PREDS];
    CondFast cf[TQP_MAX_PREDS];
    GroupSpec S;
};

struct GroupBody {
    static constexpr int kSmemBytes = kSmemSlots * 8 + kSmemSlots * kMaxAcc * 8;

    const GroupArgs& A;
    unsigned long long* skeys;
    unsigned long long* sacc;

    __device__ GroupBody(const GroupArgs& a, unsigned char* sm) : A(a) {
        skeys = reinterpret_cast<unsigned long long*>(sm);
        sacc = skeys + kSmemSlots;
        for (int i = threadIdx.x; i < kSmemSlots; i += blockDim.x) skeys[i] = kEmptyKey;
        for (int i = threadIdx.x; i < kSmemSlots * kMaxAcc; i += blockDim.x) sacc[i] = 0;
    }

    __device__ __forceinline__ int smem_slot(uint64_t key) {
        if (key == kEmptyKey) return -1;
        unsigned h = static_cast<unsigned>(mix64(key)) & (kSmemSlots - 1);
#pragma unroll 1
        for (int p = 0; p < kSmemProbe; ++p) {
            const unsigned long long k = *reinterpret_cast<volatile unsigned long long*>(&skeys[h]);
            if (k == key) return static_cast<int>(h);
            if (k == kEmptyKey) {
                const unsigned long long prev = atomicCAS(&skeys[h], kEmptyKey, key);
                if (prev == kEmptyKey || prev == key) return static_cast<int>(h);
            }
            h = (h + 1) & (kSmemSlots - 1);
        }
        return -1;
    }

    // One row per lane (act: the row passed).  Lanes whose rows share a
    // shared-memory slot are combined first (__match_any_sync), so each slot
    // takes one atomic per accumulator per warp instead of one per row: with
    // few groups (the Q1 shape) most of a warp's rows hit the same slots.
    __device__ __forceinline__ void add_rows(const ScanGeom& G, const TileView& v, int r, bool act) {
        const GroupSpec& S = A.S;
        uint64_t key = 0;
        int s = -2;  // -2: no row, -1: not in the shared table
        if (act) {
            key = pack_key(S, G, v, r);
            s = smem_slot(key);
        }
        const uint32_t peers = __match_any_sync(0xffffffffu, s);
        if (s >= 0) {
            const bool leader = (threadIdx.x % kWarp) == static_cast<unsigned>(__ffs(peers) - 1);
            unsigned long long* a = sacc + s * kMaxAcc;
            if (leader) atomicAdd(&a[0], static_cast<unsigned long long>(__popc(peers)));
            for (int i = 1; i < S.nacc; ++i) {
                const long long x = group_sum_i64(peers, eval_expr(G, v, S.acc_expr[i - 1], r));
                if (leader && x) atomicAdd(&a[i], static_cast<unsigned long long>(x));
            }
        } else if (s == -1) {
            const long long g = gtab_slot(S, key, A.ctl.err);
            if (g < 0) return;
            unsigned long long* a = S.acc + g * S.nacc;
            atomicAdd(&a[0], 1ULL);
            for (int i = 1; i < S.nacc; ++i)
                atomicAdd(&a[i], static_cast<unsigned long long>(eval_expr(G, v, S.acc_expr[i - 1], r)));
        }
    }

    __device__ void pass1(const ScanGeom& G, const TileView& v, int cw, int lane) {
        const int rw = G.T / kConsumerWarps;  // a multiple of 128
        for (int r = 0; r < rw; r += kUnroll * kWarp) {
            const int rbase = cw * rw + r;
            if (rbase >= v.rows) break;
            const uint32_t ok = eval_rows<kUnroll>(G, v, A.cf, A.cond, A.ncond, A.fast != 0, rbase + lane);
#pragma unroll
            for (int j = 0; j < kUnroll; ++j)
                if (__any_sync(0xffffffffu, (ok >> j) & 1u)) add_rows(G, v, rbase + kWarp * j + lane, (ok >> j) & 1u);
        }
    }

    // Flush the shared table into the global one and clear it for the next chunk.
    __device__ void chunk_end(const ScanGeom&, long long, long long, long long, int cw, int lane) {
        named_sync(kBarConsumers, kConsumers);
        const GroupSpec& S = A.S;
        for (int i = cw * kWarp + lane; i < kSmemSlots; i += kConsumers) {
            const unsigned long long key = skeys[i];
            if (key == kEmptyKey) continue;
            const long long g = gtab_slot(S, key, A.ctl.err);
            for (int a = 0; a < S.nacc; ++a) {
                const unsigned long long x = sacc[i * kMaxAcc + a];
                if (x && g >= 0) atomicAdd(&S.acc[g * S.nacc + a], x);
                sacc[i * kMaxAcc + a] = 0;
            }
            skeys[i] = kEmptyKey;
        }
        named_sync(kBarConsumers, kConsumers);
    }

    __device__ void finish(const ScanGeom&, int, int) {}
};

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
};

struct PlanJoinBody {
    static constexpr int kSmemBytes = 0;
    const PlanJoinArgs& A;
    unsigned long long joined = 0, passed = 0;
    long long sum = 0;

    __device__ PlanJoinBody(const PlanJoinArgs& a, unsigned char*) : A(a) {}

    // Aggregate one joined fact row r into its slot's group(s).
    __device__ __forceinline__ void aggregate(const ScanGeom& G, const TileView& v, int r, const uint4& sl) {
        const uint32_t cnt = sl.w;
        joined += cnt;
        if (A.has_sum) sum += eval_expr(G, v, A.sum, r) * static_cast<long long>(cnt);
        if (!A.dgs) return;
        const GroupSpec& S = A.S;
        if (sl.z & kDirectGroup) {  // a unique key whose dense group id sits in the slot
            unsigned long long* a = S.acc + static_cast<long long>(sl.z & ~kDirectGroup) * S.nacc;
            atomicAdd(&a[0], 1ULL);
            for (int i = 1; i < S.nacc; ++i)
                atomicAdd(&a[i], static_cast<unsigned long long>(eval_expr(G, v, S.acc_expr[i - 1], r)));
            return;
        }
        uint32_t d = sl.z;
        for (uint32_t k = 0; k < cnt; ++k) {
            unsigned long long* a = S.acc + static_cast<long long>(__ldg(&A.dgs[d])) * S.nacc;
            atomicAdd(&a[0], 1ULL);
            for (int i = 1; i < S.nacc; ++i)
                atomicAdd(&a[i], static_cast<unsigned long long>(eval_expr(G, v, S.acc_expr[i - 1], r)));
            if (k + 1 < cnt) d = __ldg(&A.next[d]);
        }
    }

    // kUnroll rows per lane are probed together: their first slot loads are
    // independent and in flight at once (the probe is latency-bound otherwise).
    __device__ void pass1(const ScanGeom& G, const TileView& v, int cw, int lane) {
        const int rw = G.T / kConsumerWarps;
        const unsigned long long mask = static_cast<unsigned long long>(A.H.cap - 1);
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
                if ((ok >> j) & 1u) {
                    key[j] = static_cast<uint64_t>(col_val(G, v, A.fk_col, rbase + kWarp * j + lane));
                    h[j] = key[j] == ~0ULL ? static_cast<unsigned long long>(A.H.cap) : (mix64(key[j]) & mask);
                }
            }
#pragma unroll
            for (int j = 0; j < kUnroll; ++j)
                if ((ok >> j) & 1u) sl[j] = __ldg(&A.H.slots[h[j]]);
#pragma unroll
            for (int j = 0; j < kUnroll; ++j) {
                if (!((ok >> j) & 1u)) continue;
                ++passed;
                if (key[j] == ~0ULL) {  // the value -1 lives in the extra slot
                    if (sl[j].w) aggregate(G, v, rbase + kWarp * j + lane, sl[j]);
                    continue;
                }
                uint4 s = sl[j];
                unsigned long long hh = h[j];
                for (long long i = 0; i < A.H.cap; ++i) {
                    const uint64_t k = slot_key(s);
                    if (k == key[j]) {
                        aggregate(G, v, rbase + kWarp * j + lane, s);
                        break;
                    }
                    if (k == ~0ULL) break;
                    hh = (hh + 1) & mask;
                    s = __ldg(&A.H.slots[hh]);
                }
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
                if (A.d_num_joined) *A.d_num_joined = static_cast<int64_t>(atomicAdd(&A.acc[0], 0ULL));
                if (A.d_sum) *A.d_sum = static_cast<int64_t>(atomicAdd(&A.acc[1], 0ULL));
                if (A.d_num_rows) *A.d_num_rows = static_cast<int64_t>(atomicAdd(&A.acc[2], 0ULL));
            }
        }
    }

    __device__ void finish(const ScanGeom&, int, int) {}
};

// ---- selection-mask expansion (second filter kernel) ------------------------------

// Expand the selection mask of rows [b * kCompactRows, ...) into row ids.
// Called by a whole block of kCompactThreads threads for mask block b.
__device__ __forceinline__ void compact_block(const uint32_t* __restrict__ mask, const uint32_t* __restrict__ block_tot,
                                              long long n, int32_t* __restrict__ row_ids, long long capacity,
                                              long long b) {
    constexpr int W = kCompactThreads / kWarp;
    __shared__ unsigned long long red[W];
    __shared__ uint32_t wtot[2][W];
    const int lane = threadIdx.x % kWarp, w = threadIdx.x / kWarp;
    // offset of this block: every earlier block's total
    unsigned long long before_blocks = 0;
    for (long long i = threadIdx.x; i < b; i += kCompactThreads) before_blocks += block_tot[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) before_blocks += __shfl_xor_sync(0xffffffffu, before_blocks, o);
    if (lane == 0) red[w] = before_blocks;
    __syncthreads();
    unsigned long long running = 0;
#pragma unroll
    for (int i = 0; i < W; ++i) running += red[i];

    const long long nwords = (n + kWarp - 1) / kWarp;
    const long long w0 = b * kCompactWords;
    const long long w1 = (w0 + kCompactWords < nwords) ? w0 + kCompactWords : nwords;
    const uint32_t lt = lanemask_lt();
    int par = 0;
    for (long long base = w0; base < w1; base += kCompactThreads) {
        const long long wi = base + threadIdx.x;
        const uint32_t word = wi < w1 ? mask[wi] : 0u;
        const uint32_t c = __popc(word);
        uint32_t incl = c;
#pragma unroll
        for (int o = 1; o < kWarp; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == kWarp - 1) wtot[par][w] = incl;
        __syncthreads();
        unsigned long long before = 0, round_total = 0;
#pragma unroll
        for (int i = 0; i < W; ++i) {
            const uint32_t x = wtot[par][i];
            before += (i < w) ? x : 0u;
            round_total += x;
        }
        const unsigned long long my_off = running + before + (incl - c);
        uint32_t nz = __ballot_sync(0xffffffffu, word != 0u);
        while (nz) {
            const int j = __ffs(nz) - 1;
            nz &= nz - 1;
            const uint32_t wj = __shfl_sync(0xffffffffu, word, j);
            const unsigned long long oj = __shfl_sync(0xffffffffu, my_off, j);
            if ((wj >> lane) & 1u) {
                const unsigned long long pos = oj + __popc(wj & lt);
                if (pos < static_cast<unsigned long long>(capacity))
                    row_ids[pos] = static_cast<int32_t>((base + w * kWarp + j) * kWarp + lane);
            }
        }
        running += round_total;
        par ^= 1;
    }
}

}  // namespace tqp
