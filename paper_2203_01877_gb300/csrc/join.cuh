// Open-addressing join hash table shared by tqp_hash_join and the plan runner.
//
// One 16-byte slot per distinct build key: {key lo, key hi, run start, run
// length}; the key is the column value as int64 bits, ~0 marks a free slot and
// the key ~0 itself (the value -1) lives in the extra slot `cap`.  Linear
// probing over a power-of-two table at load factor <= 1/2, one 16-byte load per
// probe step.  `bidx[start .. start+len)` are the build rows of the key in
// ascending order.
#pragma once

#include "common.cuh"

namespace tqp {

struct JoinHT {
    uint4* slots;      // [cap + 1]
    long long cap;     // power of two
    const uint32_t* bidx;
    // Chained tables only: the build keys' [min, max] (meta[0], meta[1]),
    // reduced on the device before the inserts.  When max - min < cap the
    // table is direct-mapped: key k lives in slot k - min, one probe, no
    // collisions (dense surrogate keys, the usual star-schema build side).
    // nullptr: hashed.
    const long long* meta;
    // Sort-based form (paper Section 5.2, Algorithm 1: sort, then bucketize):
    // the build keys minus min, sorted ascending (skeys; bidx holds their rows
    // in the same order, ascending within a key), and a directory over the
    // key range: bucket b = (key - min) >> meta[2] starts at sorted index
    // sdir[b] (sdir has nbuckets + 1 entries).  skeys == nullptr: a hash table.
    const uint64_t* skeys;
    const uint32_t* sdir;
    long long nbuild;
    long long nbuckets;
};

// Direct-mapped?  (and the key offset).  Uniform across the grid.
__device__ __forceinline__ bool ht_is_direct(const JoinHT& H, long long* kmin) {
    if (!H.meta) return false;
    const long long lo = __ldg(&H.meta[0]), hi = __ldg(&H.meta[1]);
    *kmin = lo;
    return hi >= lo && static_cast<unsigned long long>(hi) - static_cast<unsigned long long>(lo) <
                           static_cast<unsigned long long>(H.cap);
}

constexpr uint32_t kNoRow = 0xFFFFFFFFu;
// In a chained table prepared for aggregation, a slot whose key has exactly
// one build row may hold that row's dense group id (flagged) instead of the row.
constexpr uint32_t kDirectGroup = 0x80000000u;

inline long long ht_cap(long long n_build) {
    long long cap = 64;
    while (cap < 2 * n_build) cap <<= 1;
    return cap;
}

// Chained tables (plans) run at load factor <= 3/4 so that a large build
// side still leaves room in L2 for the aggregation state.
inline long long ht_cap_dense(long long n_build) {
    long long cap = 64;
    while (cap * 3 < 4 * n_build) cap <<= 1;
    return cap;
}

__device__ __forceinline__ uint64_t slot_key(const uint4& s) {
    return static_cast<uint64_t>(s.x) | (static_cast<uint64_t>(s.y) << 32);
}

// Find or claim the slot of `key` (build side).
__device__ __forceinline__ long long ht_claim(const JoinHT& H, uint64_t key, int* err) {
    if (key == ~0ULL) return H.cap;
    unsigned long long h = mix64(key) & static_cast<unsigned long long>(H.cap - 1);
    for (long long i = 0; i < H.cap; ++i) {
        unsigned long long* kp = reinterpret_cast<unsigned long long*>(&H.slots[h]);
        const unsigned long long k = *reinterpret_cast<volatile unsigned long long*>(kp);
        if (k == key) return static_cast<long long>(h);
        if (k == ~0ULL) {
            const unsigned long long prev = atomicCAS(kp, ~0ULL, key);
            if (prev == ~0ULL || prev == key) return static_cast<long long>(h);
        }
        h = (h + 1) & static_cast<unsigned long long>(H.cap - 1);
    }
    latch_error(err, TQP_ERR_CAPACITY);
    return -1;
}

// Slot of `key` or -1 (probe side; the table is read-only by then).
__device__ __forceinline__ long long ht_find(const JoinHT& H, uint64_t key) {
    if (key == ~0ULL) return H.slots[H.cap].w ? H.cap : -1;
    unsigned long long h = mix64(key) & static_cast<unsigned long long>(H.cap - 1);
    for (long long i = 0; i < H.cap; ++i) {
        const uint4 s = __ldg(&H.slots[h]);
        const uint64_t k = slot_key(s);
        if (k == key) return static_cast<long long>(h);
        if (k == ~0ULL) return -1;
        h = (h + 1) & static_cast<unsigned long long>(H.cap - 1);
    }
    return -1;
}

// The run of `key` in a sort-based table: (first sorted index, length); length
// 0 when absent.  Equal keys share a bucket, so the run lies within it.
__device__ __forceinline__ uint2 sj_lookup(const JoinHT& H, uint64_t key) {
    if (H.nbuild == 0) return make_uint2(0u, 0u);
    const long long lo_k = __ldg(&H.meta[0]), hi_k = __ldg(&H.meta[1]);
    const uint64_t e = key - static_cast<uint64_t>(lo_k);
    if (e > static_cast<uint64_t>(hi_k) - static_cast<uint64_t>(lo_k)) return make_uint2(0u, 0u);
    const uint64_t b = e >> __ldg(&H.meta[2]);
    uint32_t lo = __ldg(&H.sdir[b]), hi = __ldg(&H.sdir[b + 1]);
    const uint32_t end = hi;
    while (lo < hi) {  // first key >= e
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(&H.skeys[mid]) < e) lo = mid + 1;
        else hi = mid;
    }
    uint32_t last = lo;
    hi = end;
    while (last < hi) {  // first key > e
        const uint32_t mid = (last + hi) >> 1;
        if (__ldg(&H.skeys[mid]) <= e) last = mid + 1;
        else hi = mid;
    }
    return make_uint2(lo, last - lo);
}

// The slot of `key` in a probe-ready table (w = 0: no match): the key's own
// slot when direct-mapped, else the linear probe from its home slot.
__device__ __forceinline__ uint4 ht_match(const JoinHT& H, bool direct, long long kmin, uint64_t key) {
    if (direct) {
        const unsigned long long s = key - static_cast<uint64_t>(kmin);
        return s < static_cast<unsigned long long>(H.cap) ? __ldg(&H.slots[s]) : make_uint4(0u, 0u, 0u, 0u);
    }
    if (key == ~0ULL) return __ldg(&H.slots[H.cap]);  // the all-ones key lives in the extra slot
    const unsigned long long mask = static_cast<unsigned long long>(H.cap - 1);
    unsigned long long h = mix64(key) & mask;
    for (long long i = 0; i < H.cap; ++i) {
        const uint4 s = __ldg(&H.slots[h]);
        const uint64_t k = slot_key(s);
        if (k == key) return s;
        if (k == ~0ULL) break;
        h = (h + 1) & mask;
    }
    return make_uint4(0u, 0u, 0u, 0u);
}

}  // namespace tqp
