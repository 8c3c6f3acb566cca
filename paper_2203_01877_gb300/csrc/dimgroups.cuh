// Dimension-side preparation shared by the plan runner and the batched
// executor: dense group ids of the dimension rows (claim, number, remap) and
// direct group ids in unique-key hash slots.  Each function handles one
// element (or, for numbering, one block's range); kernels wrap them.
#pragma once

#include "group.cuh"
#include "join.cuh"

namespace tqp {

struct DimCols {
    const unsigned char* ptr[TQP_MAX_COLS];
    int32_t type[TQP_MAX_COLS];
};

// Claim dim row d's packed group key in the claim table; remember the slot.
__device__ __forceinline__ void dim_claim_row(const GroupSpec& S, const DimCols& D, long long d, uint32_t* dslot,
                                              int* err) {
    uint64_t k = 0;
    for (int i = 0; i < S.ngc; ++i) {
        const int b = S.key_bits[i];
        const int c = S.key_col[i];
        const uint64_t e = enc_key(ldg_typed(D.ptr[c], D.type[c], d), b);
        k = (b == 64) ? e : ((k << b) | e);
    }
    const long long s = gtab_slot(S, k, err);
    if (s == S.cap) S.keys[S.cap] = 0;  // mark the all-ones key's slot as claimed
    dslot[d] = s < 0 ? 0u : static_cast<uint32_t>(s);
}

constexpr int kNumberThreads = 256;

// A block of kNumberThreads numbers the claimed slots of [s0, s1) in order,
// taking its ids with a single atomic (one counter hit per claimed slot or per
// warp serialises at the L2 when groups are many); clears their accumulators.
__device__ __forceinline__ void dense_number_range(const GroupSpec& S, uint32_t* slot2dense,
                                                   unsigned long long* keys_out, unsigned long long* acc_out,
                                                   long long* d_n, long long s0, long long s1) {
    constexpr int W = kNumberThreads / kWarp;
    __shared__ uint32_t wc[2][W];
    __shared__ unsigned long long base_sm;
    const int lane = threadIdx.x % kWarp, w = threadIdx.x / kWarp;
    uint32_t c = 0;
    for (long long i = s0 + threadIdx.x; i < s1; i += kNumberThreads) c += S.keys[i] != kEmptyKey;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) wc[0][w] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int i = 0; i < W; ++i) t += wc[0][i];
        base_sm = t ? atomicAdd(reinterpret_cast<unsigned long long*>(d_n), t) : 0ULL;
    }
    __syncthreads();
    unsigned long long running = base_sm;
    int par = 1;
    for (long long rb = s0; rb < s1; rb += kNumberThreads) {
        const long long i = rb + threadIdx.x;
        const unsigned long long k = i < s1 ? S.keys[i] : kEmptyKey;
        const bool used = k != kEmptyKey;
        const uint32_t m = __ballot_sync(0xffffffffu, used);
        if (lane == 0) wc[par][w] = __popc(m);
        __syncthreads();
        unsigned long long before = 0, total = 0;
#pragma unroll
        for (int j = 0; j < W; ++j) {
            before += j < w ? wc[par][j] : 0u;
            total += wc[par][j];
        }
        if (used) {
            const long long id = static_cast<long long>(running + before + __popc(m & lanemask_lt()));
            slot2dense[i] = static_cast<uint32_t>(id);
            keys_out[id] = i < S.cap ? k : kEmptyKey;
            for (int a = 0; a < S.nacc; ++a) acc_out[id * S.nacc + a] = 0;
        }
        running += total;
        par ^= 1;
    }
}

// A unique key's slot takes its dim row's dense group id (flagged), so a
// probe that hits it needs no further dependent load.
__device__ __forceinline__ void ht_direct_slot(const JoinHT& H, const uint32_t* dgs, long long s) {
    const uint4 sl = H.slots[s];
    if (sl.w == 1u && sl.z != kNoRow) H.slots[s].z = dgs[sl.z] | kDirectGroup;
}

// Build-key range of a chained table: rows i0, i0 + stride, ... < i1 into
// H.meta (min, max).  Called by every thread of a block (block-wide sync).
__device__ __forceinline__ void ht_key_range(const JoinHT& H, const unsigned char* key_col, int key_type,
                                             long long i0, long long i1, long long stride) {
    long long lo = LLONG_MAX, hi = LLONG_MIN;
    for (long long i = i0; i < i1; i += stride) {
        const long long k = ldg_typed(key_col, key_type, i);
        lo = k < lo ? k : lo;
        hi = k > hi ? k : hi;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long l2 = __shfl_xor_sync(0xffffffffu, lo, o), h2 = __shfl_xor_sync(0xffffffffu, hi, o);
        lo = l2 < lo ? l2 : lo;
        hi = h2 > hi ? h2 : hi;
    }
    // one atomic pair per block (every warp of the block calls this)
    __shared__ long long blo[32], bhi[32];
    const int w = threadIdx.x / kWarp, nw = (blockDim.x + kWarp - 1) / kWarp;
    if ((threadIdx.x % kWarp) == 0) {
        blo[w] = lo;
        bhi[w] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < nw; ++i) {
            lo = blo[i] < lo ? blo[i] : lo;
            hi = bhi[i] > hi ? bhi[i] : hi;
        }
        if (lo <= hi) {
            long long* m = const_cast<long long*>(H.meta);
            atomicMin(&m[0], lo);
            atomicMax(&m[1], hi);
        }
    }
}

// Chained build: row i claims its key's slot, pushes itself on the slot's
// list (z = head row, next[] links) and counts itself.
__device__ __forceinline__ void ht_chain_insert_row(const JoinHT& H, const unsigned char* key_col, int key_type,
                                                    long long i, uint32_t* next, int* err) {
    const uint64_t key = static_cast<uint64_t>(ldg_typed(key_col, key_type, i));
    long long kmin = 0;
    long long s;
    if (ht_is_direct(H, &kmin)) {
        s = static_cast<long long>(key - static_cast<uint64_t>(kmin));
        H.slots[s].x = static_cast<uint32_t>(key);
        H.slots[s].y = static_cast<uint32_t>(key >> 32);
    } else {
        s = ht_claim(H, key, err);
    }
    if (s < 0) return;
    next[i] = atomicExch(&H.slots[s].z, static_cast<uint32_t>(i));
    atomicAdd(&H.slots[s].w, 1u);
}

}  // namespace tqp
