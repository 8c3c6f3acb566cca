// Aggregation-table pieces shared by the group-by scan and the plan runner:
// packed order-preserving group keys, the global open-addressing table of
// exact int64 accumulators, and the per-group output writer.
#pragma once

#include "engine.cuh"

namespace tqp {

constexpr unsigned long long kEmptyKey = ~0ULL;
constexpr int kMaxAcc = 1 + TQP_MAX_AGGS;  // count + one sum per distinct expression
constexpr int kSmallCap = 4096;            // finalize in one CTA up to this many table slots
constexpr int kFinThreads = 1024;

struct GroupSpec {
    int32_t ngc;
    int32_t width;                 // packed key bits (0..64)
    int32_t key_col[TQP_MAX_GROUP_COLS];
    int32_t key_bits[TQP_MAX_GROUP_COLS];
    int32_t nacc;                  // accumulators; [0] is the row count
    int32_t naggs;
    int32_t agg_fn[TQP_MAX_AGGS];
    int32_t agg_acc[TQP_MAX_AGGS];
    DExpr acc_expr[TQP_MAX_AGGS];  // expression of accumulator a + 1
    // How accumulator a + 1 combines (kAccSum: the sum; kAccMax / kAccMin: the
    // unsigned maximum of an order-preserving code, so every accumulator still
    // starts at zero); `minmax` is set when any is not a sum.
    int32_t acc_kind[TQP_MAX_AGGS];
    int32_t minmax;
    int32_t pad_kind;
    unsigned long long* keys;      // [cap + 1], kEmptyKey = free; slot cap holds the all-ones key
    unsigned long long* acc;       // [(cap + 1) * nacc]
    long long cap;                 // power of two (dense mode: entry bound)
    unsigned long long* ndistinct;
    long long max_groups;
    const long long* d_dense_n;    // dense mode: entries [0, *d_dense_n) are groups with any key
};

constexpr int32_t kAccSum = 0, kAccMax = 1, kAccMin = 2;

// MAX keeps the largest x ^ 2^63 (unsigned order = signed order of x); MIN
// the largest ~(x ^ 2^63).  Both codes of a row are above the zero start
// except that of the extreme value, which decodes correctly from zero.
__host__ __device__ __forceinline__ unsigned long long acc_encode(int kind, int64_t x) {
    const unsigned long long u = static_cast<unsigned long long>(x) ^ 0x8000000000000000ull;
    return kind == kAccMin ? ~u : u;
}
__host__ __device__ __forceinline__ int64_t acc_decode(int kind, unsigned long long u) {
    return static_cast<int64_t>((kind == kAccMin ? ~u : u) ^ 0x8000000000000000ull);
}

__device__ __forceinline__ uint64_t enc_key(int64_t x, int bits) {
    if (bits == 8) return static_cast<uint64_t>(x) & 0xFFull;
    if (bits == 32) return static_cast<uint64_t>(static_cast<uint32_t>(x) ^ 0x80000000u);
    return static_cast<uint64_t>(x) ^ 0x8000000000000000ull;
}

__device__ __forceinline__ int64_t dec_key(uint64_t e, int bits) {
    if (bits == 8) return static_cast<int64_t>(e & 0xFFull);
    if (bits == 32) return static_cast<int64_t>(static_cast<int32_t>(static_cast<uint32_t>(e) ^ 0x80000000u));
    return static_cast<int64_t>(e ^ 0x8000000000000000ull);
}

__device__ __forceinline__ uint64_t pack_key(const GroupSpec& S, const ScanGeom& G, const TileView& v, int r) {
    uint64_t k = 0;
    for (int i = 0; i < S.ngc; ++i) {
        const int b = S.key_bits[i];
        const uint64_t e = enc_key(col_val(G, v, S.key_col[i], r), b);
        k = (b == 64) ? e : ((k << b) | e);
    }
    return k;
}

// Find or claim the global slot of `key`; -1 (and CAPACITY latched) if full.
__device__ __forceinline__ long long gtab_slot(const GroupSpec& S, uint64_t key, int* err) {
    if (key == kEmptyKey) return S.cap;
    unsigned long long h = mix64(key) & static_cast<unsigned long long>(S.cap - 1);
    long long slot = -1;
    bool inserted = false;
    for (long long i = 0; i < S.cap; ++i) {
        const unsigned long long k = *reinterpret_cast<volatile unsigned long long*>(&S.keys[h]);
        if (k == key) {
            slot = static_cast<long long>(h);
            break;
        }
        if (k == kEmptyKey) {
            const unsigned long long prev = atomicCAS(&S.keys[h], kEmptyKey, key);
            if (prev == kEmptyKey || prev == key) {
                slot = static_cast<long long>(h);
                inserted = prev == kEmptyKey;
                break;
            }
        }
        h = (h + 1) & static_cast<unsigned long long>(S.cap - 1);
    }
    // new keys counted with one atomic per converged group of lanes (the
    // counter is a single address: one add per insert serialises at L2); each
    // inserting lane's index is the count before it, as with its own add
    const unsigned am = __activemask();
    const unsigned im = __ballot_sync(am, inserted);
    if (im) {
        const int lane = static_cast<int>(threadIdx.x % 32);
        const int first = __ffs(im) - 1;
        unsigned long long base = 0;
        if (lane == first) base = atomicAdd(S.ndistinct, static_cast<unsigned long long>(__popc(im)));
        base = __shfl_sync(am, base, first);
        if (inserted && static_cast<long long>(base + __popc(im & ((1u << lane) - 1u))) >= S.max_groups)
            latch_error(err, TQP_ERR_CAPACITY);
    }
    if (slot < 0) latch_error(err, TQP_ERR_CAPACITY);
    return slot;
}

struct GroupOut {
    int64_t* keys;     // [G][ngc]
    int64_t* ivals;    // [G][naggs]
    double* fvals;     // [G][naggs]
    long long capacity;
    int64_t* num_groups;
    int* err;
};

__device__ __forceinline__ void emit_group(const GroupSpec& S, const GroupOut& O, long long g, uint64_t key,
                                           long long slot) {
    if (O.keys) {
        uint64_t k = key;
        for (int i = S.ngc - 1; i >= 0; --i) {
            const int b = S.key_bits[i];
            const uint64_t e = (b == 64) ? k : (k & ((1ULL << b) - 1));
            O.keys[g * S.ngc + i] = dec_key(e, b);
            k = (b == 64) ? 0 : (k >> b);
        }
    }
    const unsigned long long* a = slot >= 0 ? S.acc + slot * S.nacc : nullptr;
    const long long cnt = a ? static_cast<long long>(a[0]) : 0;
    for (int j = 0; j < S.naggs; ++j) {
        const int fn = S.agg_fn[j];
        const bool mm = fn == TQP_MIN || fn == TQP_MAX;
        long long x = a ? static_cast<long long>(a[S.agg_acc[j]]) : 0;
        if (mm) x = cnt ? acc_decode(S.acc_kind[S.agg_acc[j] - 1], static_cast<unsigned long long>(x)) : 0;
        if (O.ivals) O.ivals[g * S.naggs + j] = x;
        if (O.fvals) {
            double f = 0.0;
            if (fn == TQP_AVG) f = __ddiv_rn(__ll2double_rn(x), __ll2double_rn(cnt));
            else if (mm && cnt == 0) f = __longlong_as_double(0x7ff8000000000000LL);  // no rows: NaN flag
            O.fvals[g * S.naggs + j] = f;
        }
    }
}

// A slot is a group iff at least one row was counted into it (a slot may
// be claimed in advance, e.g. for every dimension-table group of a join).
__device__ __forceinline__ bool slot_used(const GroupSpec& S, long long i) {
    if (S.d_dense_n && i >= *S.d_dense_n) return false;
    return S.acc[i * S.nacc] != 0ULL;
}

// Packed key of a used slot.
__device__ __forceinline__ uint64_t slot_key(const GroupSpec& S, long long i) {
    if (S.d_dense_n) return S.keys[i];
    return i < S.cap ? S.keys[i] : kEmptyKey;
}


// host side (groupby.cu)
tqp_status lower_group(const int32_t* key_cols, const int32_t* key_types, int32_t ngc, const tqp_agg* aggs,
                       int32_t naggs, int ncols, GroupSpec* S);
long long group_table_cap(long long max_groups);
size_t group_table_bytes(long long cap, int nacc);
tqp_status group_table_init(GroupSpec* S, void* mem, long long cap, long long max_groups, cudaStream_t stream,
                            bool clear = true);
tqp_status group_finalize(tqp_ctx* ctx, const GroupSpec& S, const GroupOut& O, cudaStream_t stream);
// Top-k groups by accumulator of aggregate `agg` (descending; ties: key
// ascending); writes min(k, G) rows in rank order and *total_groups = G.
tqp_status group_topk(tqp_ctx* ctx, const GroupSpec& S, const GroupOut& O, int k, int agg,
                      int64_t* total_groups, cudaStream_t stream);

}  // namespace tqp
