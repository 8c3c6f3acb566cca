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

static __device__ void top_sort_block(long long* r, uint64_t* k, uint32_t* s) {
    for (int kk = 2; kk <= kTopBlock; kk <<= 1) {
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < kTopBlock; i += blockDim.x) {
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

static __device__ void topk_level0_block(const GroupSpec& S, int rank_acc, int k, TopBuf out, unsigned long long* total,
                                  long long block) {
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
            r[p] = static_cast<long long>(S.acc[slot * S.nacc + rank_acc]);
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
                                  const GroupOut& O, const unsigned long long* total, int64_t* total_out, long long block) {
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

}  // namespace tqp
