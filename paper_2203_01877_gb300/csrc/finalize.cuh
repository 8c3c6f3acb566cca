// Group-table finalisation shared by the group-by operator, the plan runner
// and the batched executor: one-CTA sorted output for small tables and the
// top-k tournament.  Functions take the block index they work on, so a
// kernel may serve many tables.
#pragma once

#include "group.cuh"

namespace tqp {

// One CTA: collect occupied slots, bitonic-sort (key, slot), emit.
// fsm: kFinSmemBytes of dynamic shared memory.
static __device__ void finalize_small_block(const GroupSpec& S, const GroupOut& O, unsigned char* fsm) {
    const int P = 2 * kSmallCap;  // slots + special, padded to a power of two
    unsigned long long* sk = reinterpret_cast<unsigned long long*>(fsm);
    uint32_t* ss = reinterpret_cast<uint32_t*>(sk + P);
    __shared__ int count;
    if (threadIdx.x == 0) count = 0;
    __syncthreads();
    const bool overflow = static_cast<long long>(*S.ndistinct) > S.max_groups;
    for (long long i = threadIdx.x; i <= S.cap; i += blockDim.x) {
        if (slot_used(S, i)) {
            const int p = atomicAdd(&count, 1);
            if (p < P) {
                sk[p] = slot_key(S, i);
                ss[p] = static_cast<uint32_t>(i);
            }
        }
    }
    __syncthreads();
    const int G = min(count, P);
    int n2 = 1;
    while (n2 < G) n2 <<= 1;
    for (int i = G + threadIdx.x; i < n2; i += blockDim.x) {
        sk[i] = kEmptyKey;
        ss[i] = 0xFFFFFFFFu;
    }
    __syncthreads();
    for (int k = 2; k <= n2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n2; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) {
                    const bool up = (i & k) == 0;
                    const unsigned long long ki = sk[i], kl = sk[l];
                    const uint32_t si = ss[i], sl = ss[l];
                    const bool gt = (ki > kl) || (ki == kl && si > sl);
                    if (gt == up) {
                        sk[i] = kl; sk[l] = ki;
                        ss[i] = sl; ss[l] = si;
                    }
                }
            }
            __syncthreads();
        }
    }
    if (overflow || G > O.capacity) {
        if (threadIdx.x == 0) {
            *O.num_groups = -1;
            latch_error(O.err, TQP_ERR_CAPACITY);
        }
        return;
    }
    if (S.ngc == 0 && G == 0) {  // ungrouped aggregate over no rows: one row, COUNT 0, AVG NaN
        if (threadIdx.x == 0) {
            emit_group(S, O, 0, 0, -1);
            if (O.fvals)
                for (int j = 0; j < S.naggs; ++j)
                    if (S.agg_fn[j] == TQP_AVG) O.fvals[j] = __longlong_as_double(0x7ff8000000000000LL);
            *O.num_groups = 1;
        }
        return;
    }
    for (int g = threadIdx.x; g < G; g += blockDim.x) emit_group(S, O, g, sk[g], ss[g]);
    if (threadIdx.x == 0) *O.num_groups = G;
}

// ---- top-k ------------------------------------------------------------------------
// Groups ordered by one accumulator descending, ties by packed key ascending
// (then slot, which orders padding last).  A tournament of block-local
// bitonic sorts: each block sorts kTopBlock candidates in shared memory and
// keeps its first k, until one block remains.

constexpr int kTopBlock = 2048;
constexpr int kTopThreads = 1024;

struct TopBuf {
    long long* rank;
    uint64_t* key;
    uint32_t* slot;
};

static __device__ __forceinline__ bool top_before(long long r1, uint64_t k1, uint32_t s1, long long r2, uint64_t k2,
                                           uint32_t s2) {
    if (r1 != r2) return r1 > r2;
    if (k1 != k2) return k1 < k2;
    return s1 < s2;
}

// Bitonic sort of the first n entries (n a power of two, at most kTopBlock).
static __device__ void top_sort_block(long long* r, uint64_t* k, uint32_t* s, int n = kTopBlock) {
    for (int kk = 2; kk <= n; kk <<= 1) {
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) {
                    const bool asc = (i & kk) == 0;  // "ascending" in before-order
                    const bool lb = top_before(r[l], k[l], s[l], r[i], k[i], s[i]);
                    if (lb == asc) {
                        const long long tr = r[i]; r[i] = r[l]; r[l] = tr;
                        const uint64_t tk = k[i]; k[i] = k[l]; k[l] = tk;
                        const uint32_t ts = s[i]; s[i] = s[l]; s[l] = ts;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// The value a group is ranked by: its accumulator `rank_acc`, with a MIN/MAX
// accumulator's order-preserving code decoded to the int64 value it keeps.
__device__ __forceinline__ long long rank_value(const GroupSpec& S, int rank_acc, long long slot) {
    const unsigned long long x = S.acc[slot * S.nacc + rank_acc];
    const int kind = rank_acc > 0 ? S.acc_kind[rank_acc - 1] : kAccSum;
    return kind == kAccSum ? static_cast<long long>(x) : acc_decode(kind, x);
}

static __device__ void topk_level0_block(const GroupSpec& S, int rank_acc, int k, TopBuf out, unsigned long long* total,
                                  long long block, const unsigned int* run = nullptr) {
    if (run && *reinterpret_cast<const volatile unsigned int*>(run) == 0) return;  // the radix select succeeded
    __shared__ long long r[kTopBlock];
    __shared__ uint64_t kk[kTopBlock];
    __shared__ uint32_t ss[kTopBlock];
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    for (int i = threadIdx.x; i < kTopBlock; i += blockDim.x) {
        r[i] = LLONG_MIN;
        kk[i] = ~0ULL;
        ss[i] = 0xFFFFFFFFu;
    }
    __syncthreads();
    const long long s0 = block * kTopBlock;
    for (int i = threadIdx.x; i < kTopBlock; i += blockDim.x) {
        const long long slot = s0 + i;
        if (slot <= S.cap && slot_used(S, slot)) {
            const int p = atomicAdd(&cnt, 1);
            r[p] = rank_value(S, rank_acc, slot);
            kk[p] = slot_key(S, slot);
            ss[p] = static_cast<uint32_t>(slot);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && cnt) atomicAdd(total, static_cast<unsigned long long>(cnt));
    // empty blocks (beyond a dense table's groups) skip the sort; a handful of
    // candidates is ordered by one thread
    if (cnt > 32) top_sort_block(r, kk, ss);
    else if (cnt > 1) {
        if (threadIdx.x == 0)
            for (int a = 1; a < cnt; ++a)
                for (int b = a; b > 0 && top_before(r[b], kk[b], ss[b], r[b - 1], kk[b - 1], ss[b - 1]); --b) {
                    const long long tr = r[b]; r[b] = r[b - 1]; r[b - 1] = tr;
                    const uint64_t tk = kk[b]; kk[b] = kk[b - 1]; kk[b - 1] = tk;
                    const uint32_t ts = ss[b]; ss[b] = ss[b - 1]; ss[b - 1] = ts;
                }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        const long long o = block * k + i;
        out.rank[o] = r[i];
        out.key[o] = kk[i];
        out.slot[o] = ss[i];
    }
}

// One reduction level; with `emit` set (a single block) the winners are written out.
static __device__ void topk_reduce_block(const GroupSpec& S, TopBuf in, long long n_in, int k, TopBuf out, int emit,
                                  const GroupOut& O, const unsigned long long* total, int64_t* total_out, long long block,
                                  const unsigned int* run = nullptr) {
    if (run && *reinterpret_cast<const volatile unsigned int*>(run) == 0) return;
    __shared__ long long r[kTopBlock];
    __shared__ uint64_t kk[kTopBlock];
    __shared__ uint32_t ss[kTopBlock];
    const long long c0 = block * kTopBlock;
    for (int i = threadIdx.x; i < kTopBlock; i += blockDim.x) {
        const long long c = c0 + i;
        if (c < n_in) {
            r[i] = in.rank[c];
            kk[i] = in.key[c];
            ss[i] = in.slot[c];
        } else {
            r[i] = LLONG_MIN;
            kk[i] = ~0ULL;
            ss[i] = 0xFFFFFFFFu;
        }
    }
    __syncthreads();
    top_sort_block(r, kk, ss);
    if (!emit) {
        for (int i = threadIdx.x; i < k; i += blockDim.x) {
            const long long o = block * k + i;
            out.rank[o] = r[i];
            out.key[o] = kk[i];
            out.slot[o] = ss[i];
        }
        return;
    }
    const long long G = static_cast<long long>(*total);
    const long long m = G < k ? G : k;
    if (m > O.capacity) {
        if (threadIdx.x == 0) {
            *O.num_groups = -1;
            latch_error(O.err, TQP_ERR_CAPACITY);
        }
        return;
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x) emit_group(S, O, i, kk[i], ss[i]);
    if (threadIdx.x == 0) {
        *O.num_groups = m;
        if (total_out) *total_out = G;
    }
}

// ---- top-k by radix select -------------------------------------------------------
// The k-th largest rank is located by histogram passes over the order-
// preserving transform u = rank ^ 2^63.  The first pass bins ranks on a log
// scale (sign, position of the highest bit, the next five bits: 4096 bins
// that each cover one aligned interval of u), so that ranks of any magnitude
// spread over many bins; every later pass bins the next (at most) 12 bits
// below what is already known.  The last block of each pass picks the bin
// holding the k-th largest.  As soon as every group at or above the chosen
// interval fits kSelCand candidates they are collected and one block sorts
// them (rank descending, key ascending, slot ascending) and emits the first k.
// If the interval narrows to one value with more ties than that, `fallback`
// is set and the tournament above runs instead (its blocks return early
// otherwise).  Passes after the deciding one return at once.

constexpr int kSelBins = 4096;
constexpr int kSelPasses = 6;     // 7 bits from the first pass, then 12 per pass: 64 bits
constexpr int kSelCand = kTopBlock;
constexpr int kSelThreads = 256;
constexpr int kSelSlots = 2048;  // slots per block of a pass

struct TopSel {
    unsigned long long thresh;     // u of the chosen interval's lower end (bits below `known` zero)
    long long need;                // rank of the k-th largest within the chosen interval
    long long total;               // groups (used slots)
    long long above;               // groups above the chosen interval
    unsigned int done;             // candidates are final
    unsigned int fallback;         // run the tournament
    unsigned int blocks_done;      // last-block detection of the running pass
    unsigned int ncand;
    int known;                     // bits of u at and above this position are fixed by the interval
    int empty;                     // no group to emit
    int pad[2];
    unsigned int hist[kSelBins];
};
static_assert(sizeof(TopSel) % 16 == 0, "TopSel is zeroed in 16-byte words");

__host__ __device__ __forceinline__ unsigned long long rank_u(long long rank) {
    return static_cast<unsigned long long>(rank) ^ (1ULL << 63);
}

// log-scale code of x >= 0 in [0, 2048): exact below 32, else 32 per octave
__host__ __device__ __forceinline__ int log_code(unsigned long long x) {
    if (x < 32) return static_cast<int>(x);
#ifdef __CUDA_ARCH__
    const int e = 63 - __clzll(static_cast<long long>(x));
#else
    const int e = 63 - __builtin_clzll(x);
#endif
    return 32 + (e - 5) * 32 + static_cast<int>((x >> (e - 5)) & 31);
}

// first-pass bin: increasing in rank
__host__ __device__ __forceinline__ int first_bin(long long rank) {
    return rank >= 0 ? 2048 + log_code(static_cast<unsigned long long>(rank))
                     : 2047 - log_code(static_cast<unsigned long long>(~rank));
}

// the interval of u a first-pass bin covers: its lower end and the low bits left open
__host__ __device__ __forceinline__ void first_bin_interval(int b, unsigned long long* lo, int* open) {
    const int g = b >= 2048 ? b - 2048 : 2047 - b;
    unsigned long long x;
    int p;
    if (g < 32) {
        x = static_cast<unsigned long long>(g);
        p = 0;
    } else {
        const int e = (g - 32) / 32 + 5;
        p = e - 5;
        x = (1ULL << e) | (static_cast<unsigned long long>((g - 32) % 32) << p);
    }
    // rank = x (b >= 2048) or ~x; u = rank ^ 2^63, bits below p cleared
    const unsigned long long u = b >= 2048 ? x ^ (1ULL << 63) : (~x) & ~(1ULL << 63);
    *lo = p ? (u >> p) << p : u;
    *open = p;
}

__device__ __forceinline__ long long slot_rank(const GroupSpec& S, int rank_acc, long long slot) {
    return rank_value(S, rank_acc, slot);
}

// One block of pass `pass` over slots [block * kSelSlots, ...).
static __device__ void topsel_pass_block(const GroupSpec& S, int rank_acc, int k, TopSel* sel, int pass,
                                         long long block, long long nblocks) {
    __shared__ unsigned int h[kSelBins];
    __shared__ int last;
    __shared__ long long red[kSelThreads / 32];
    __shared__ int found_b;
    __shared__ long long found_above;
    int known = 64, shift = 0;
    unsigned long long pre = 0;
    if (pass > 0) {
        const volatile TopSel* vs = sel;
        if (vs->done || vs->fallback) return;
        known = vs->known;  // > 0: a pass that leaves one value decides
        shift = known > 12 ? known - 12 : 0;
        pre = vs->thresh >> known;
    }
    for (int i = threadIdx.x; i < kSelBins; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const long long s0 = block * kSelSlots;
    for (long long i = s0 + threadIdx.x; i < s0 + kSelSlots && i <= S.cap; i += blockDim.x) {
        if (!slot_used(S, i)) continue;
        const long long rank = slot_rank(S, rank_acc, i);
        int b;
        if (pass == 0) {
            b = first_bin(rank);
        } else {
            const unsigned long long u = rank_u(rank);
            if ((u >> known) != pre) continue;
            b = static_cast<int>((u >> shift) & ((1ULL << (known - shift)) - 1));
        }
        atomicAdd(&h[b], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kSelBins; i += blockDim.x)
        if (h[i]) atomicAdd(&sel->hist[i], h[i]);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&sel->blocks_done, 1u) == static_cast<unsigned int>(nblocks - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    // the last block: bins from the top, each thread a run of kSelBins / kSelThreads
    constexpr int R = kSelBins / kSelThreads;
    const volatile unsigned int* gh = sel->hist;
    const int hi = kSelBins - 1 - threadIdx.x * R;  // this thread's bins: hi, hi - 1, ..., hi - R + 1
    long long mine = 0;
    for (int j = 0; j < R; ++j) mine += gh[hi - j];
    long long incl = mine;  // inclusive prefix over runs, top bins first
    const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) red[w] = incl;
    if (threadIdx.x == 0) found_b = -1;
    __syncthreads();
    long long before = 0, all = 0;
    for (int i = 0; i < kSelThreads / 32; ++i) {
        before += i < w ? red[i] : 0;
        all += red[i];
    }
    before += incl - mine;
    if (pass == 0 && threadIdx.x == 0) {
        sel->total = all;
        sel->need = all < k ? all : k;
    }
    __syncthreads();
    const long long need = *reinterpret_cast<volatile long long*>(&sel->need);
    if (need > 0 && before < need && before + mine >= need) {
        long long c = before;
        for (int j = 0; j < R; ++j) {
            const long long hb = gh[hi - j];
            if (c + hb >= need) {
                found_b = hi - j;
                found_above = c;
                break;
            }
            c += hb;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (need <= 0) {
            sel->done = 1;
            sel->empty = 1;
        } else {
            const int b = found_b;
            const long long hb = gh[b];
            int open;
            if (pass == 0) {
                unsigned long long lo;
                first_bin_interval(b, &lo, &open);
                sel->thresh = lo;
            } else {
                open = shift;
                sel->thresh |= static_cast<unsigned long long>(b) << shift;
            }
            sel->known = open;
            sel->above += found_above;
            sel->need = need - found_above;
            if (sel->above + hb <= kSelCand) sel->done = 1;
            else if (open == 0) sel->fallback = 1;  // one value, too many ties
        }
        sel->blocks_done = 0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kSelBins; i += blockDim.x) sel->hist[i] = 0;
}

// Collect the candidates: every group whose u is at or above the chosen interval's lower end.
static __device__ void topsel_collect_block(const GroupSpec& S, int rank_acc, TopSel* sel, TopBuf cand, long long block) {
    const volatile TopSel* vs = sel;
    if (!vs->done || vs->empty) return;
    const unsigned long long lo = vs->thresh;
    const long long s0 = block * kSelSlots;
    for (long long i = s0 + threadIdx.x; i < s0 + kSelSlots && i <= S.cap; i += blockDim.x) {
        if (!slot_used(S, i)) continue;
        const long long rank = slot_rank(S, rank_acc, i);
        if (rank_u(rank) < lo) continue;
        const unsigned int p = atomicAdd(&sel->ncand, 1u);
        if (p < static_cast<unsigned int>(kSelCand)) {
            cand.rank[p] = rank;
            cand.key[p] = slot_key(S, i);
            cand.slot[p] = static_cast<uint32_t>(i);
        }
    }
}

// One block (kTopThreads threads): sort the candidates, emit the first k.
static __device__ void topsel_emit_block(const GroupSpec& S, int k, const TopSel* sel, TopBuf cand, const GroupOut& O,
                                         int64_t* total_out) {
    __shared__ long long r[kTopBlock];
    __shared__ uint64_t kk[kTopBlock];
    __shared__ uint32_t ss[kTopBlock];
    const volatile TopSel* vs = sel;
    if (!vs->done) return;
    const long long total = vs->total;
    const int n = vs->empty ? 0 : static_cast<int>(vs->ncand < static_cast<unsigned int>(kSelCand) ? vs->ncand
                                                                                                  : kSelCand);
    int n2 = 1;
    while (n2 < n) n2 <<= 1;
    for (int i = threadIdx.x; i < n2; i += blockDim.x) {
        if (i < n) {
            r[i] = cand.rank[i];
            kk[i] = cand.key[i];
            ss[i] = cand.slot[i];
        } else {
            r[i] = LLONG_MIN;
            kk[i] = ~0ULL;
            ss[i] = 0xFFFFFFFFu;
        }
    }
    __syncthreads();
    top_sort_block(r, kk, ss, n2);
    const long long m = total < k ? total : k;
    if (m > O.capacity) {
        if (threadIdx.x == 0) {
            *O.num_groups = -1;
            latch_error(O.err, TQP_ERR_CAPACITY);
        }
        return;
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x) emit_group(S, O, i, kk[i], ss[i]);
    if (threadIdx.x == 0) {
        *O.num_groups = m;
        if (total_out) *total_out = total;
    }
}

}  // namespace tqp
