// tqp_hash_join: inner equi-join returning index pairs (late materialisation).
//
// Semantics of paper Sections 5.2-5.3 (Algorithm 2's hash join and Algorithm
// 1's sort join both produce every (left, right) index pair with equal keys);
// the result here is emitted in canonical (probe ascending, build ascending)
// order.  Instead of Algorithm 2's repeated scatter/probe rounds (one round
// per colliding build row), the build side goes into one open-addressing
// table:
//   build  1. each build row finds or claims its key's slot (64-bit CAS on the
//             key, linear probing, load factor <= 1/2) and counts itself;
//          2. a stable radix sort of (slot, build row) groups the build rows
//             of each key into one run, in ascending row order;
//          3. each run's start is written into its slot.
//   probe  staged scan of the probe keys: every row's slot is looked up and
//          remembered, matches are counted per chunk, a decoupled look-back
//          over chunks gives each chunk's output offset, and each row's run
//          is copied out as (build, probe) pairs.
// Keys compare by their int64 value; int32, int64 and uint8 key columns mix.
#include <cstdio>

#include "host.h"
#include "join.cuh"
#include "dimgroups.cuh"

namespace tqp {

tqp_status radix_sort_pairs(uint64_t* k0, uint32_t* v0, uint64_t* k1, uint32_t* v1, const long long* d_n,
                            long long n_max, int begin_bit, int end_bit, void* scratch, cudaStream_t stream,
                            bool* result_in_1);
size_t radix_sort_scratch(long long n_max);

__global__ void k_ht_init(JoinHT H) {
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i <= H.cap;
         i += static_cast<long long>(gridDim.x) * blockDim.x)
        H.slots[i] = make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, kNoRow, 0u);
}

// Chained build (plans): each build row claims its key's slot, pushes itself
// on the slot's list (z = head row, next[] links) and counts itself.  The
// rows of a key come out in no particular order, which aggregation does not
// mind; no sort is needed.
__global__ void k_ht_meta_init(long long* meta) {
    meta[0] = LLONG_MAX;
    meta[1] = LLONG_MIN;
}

__global__ void k_ht_key_range(JoinHT H, const unsigned char* key_col, int key_type, long long n) {
    const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
    ht_key_range(H, key_col, key_type, blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x, n, stride);
}

__global__ void k_ht_insert_chain(JoinHT H, const unsigned char* key_col, int key_type, long long n,
                                  uint32_t* next, int* err) {
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x)
        ht_chain_insert_row(H, key_col, key_type, i, next, err);
}

// Key range of a chained table's build side into meta[0..1] (device).
tqp_status ht_key_range_launch(const tqp_ctx* ctx, const tqp_table* build, int32_t key_col, long long* meta,
                               cudaStream_t stream) {
    k_ht_meta_init<<<1, 1, 0, stream>>>(meta);
    TQP_CUDA(cudaGetLastError());
    const long long n = build->num_rows;
    if (n == 0) return TQP_OK;
    JoinHT R;
    memset(&R, 0, sizeof(R));
    R.meta = meta;
    const tqp_column& kc = build->cols[key_col];
    const int threads = 256;
    const int blocks = static_cast<int>(std::min<long long>((n + threads - 1) / threads, ctx->num_sms * 16LL));
    k_ht_key_range<<<blocks, threads, 0, stream>>>(R, static_cast<const unsigned char*>(kc.data), kc.type, n);
    TQP_CUDA(cudaGetLastError());
    return TQP_OK;
}

// Chained inserts into H (slots [cap + 1] and next [n] provided; H.meta holds
// the key range already).
tqp_status ht_chain_insert_launch(const tqp_ctx* ctx, const tqp_table* build, int32_t key_col, const JoinHT& H,
                                  uint32_t* next, cudaStream_t stream) {
    const int threads = 256;
    const int blocks = static_cast<int>(std::min<long long>((H.cap + threads) / threads, ctx->num_sms * 16LL));
    k_ht_init<<<blocks, threads, 0, stream>>>(H);
    TQP_CUDA(cudaGetLastError());
    const long long n = build->num_rows;
    if (n == 0) return TQP_OK;
    const tqp_column& kc = build->cols[key_col];
    const int iblocks = static_cast<int>(std::min<long long>((n + threads - 1) / threads, ctx->num_sms * 16LL));
    k_ht_insert_chain<<<iblocks, threads, 0, stream>>>(H, static_cast<const unsigned char*>(kc.data), kc.type, n, next,
                                                       ctx->d_err);
    TQP_CUDA(cudaGetLastError());
    return TQP_OK;
}

tqp_status ht_build_chain(tqp_ctx* ctx, const tqp_table* build, int32_t key_col, JoinHT* H, uint32_t** next,
                          cudaStream_t stream) {
    const long long n = build->num_rows;
    H->cap = ht_cap_dense(n) * ht_scale(ctx);
    H->slots = static_cast<uint4*>(arena_alloc(ctx, static_cast<size_t>(H->cap + 1) * sizeof(uint4)));
    *next = static_cast<uint32_t*>(arena_alloc(ctx, static_cast<size_t>(n > 0 ? n : 1) * 4));
    long long* meta = static_cast<long long*>(arena_alloc(ctx, 64));
    if (!H->slots || !*next || !meta) return arena_oom(ctx, static_cast<size_t>(H->cap + 1) * 16 + n * 4);
    H->bidx = nullptr;
    H->meta = meta;
    TQP_TRY(ht_key_range_launch(ctx, build, key_col, meta, stream));
    return ht_chain_insert_launch(ctx, build, key_col, *H, *next, stream);
}

// A direct-mapped table (dense build keys: max - min < cap) puts key k in
// slot k - min, and every key, the all-ones one included, in the main slots.
__global__ void k_ht_insert(JoinHT H, const unsigned char* key_col, int key_type, long long n, uint64_t* sort_key,
                            uint32_t* sort_val, int* err) {
    long long kmin = 0;
    const bool direct = ht_is_direct(H, &kmin);
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const uint64_t key = static_cast<uint64_t>(ldg_typed(key_col, key_type, i));
        long long s;
        if (direct) {
            s = static_cast<long long>(key - static_cast<uint64_t>(kmin));
            H.slots[s].x = static_cast<uint32_t>(key);  // (several rows may write the same key)
            H.slots[s].y = static_cast<uint32_t>(key >> 32);
        } else {
            s = ht_claim(H, key, err);
        }
        if (s >= 0) atomicAdd(&H.slots[s].w, 1u);
        sort_key[i] = static_cast<uint64_t>(s < 0 ? H.cap : s);
        sort_val[i] = static_cast<uint32_t>(i);
    }
}

// After the sort: run starts into the slots; the sorted values are the
// build rows of each run in ascending order.  A run of one build row (a
// unique key) stores that row itself, flagged kRunRow, so the probe writes
// its pairs without loading it from the sorted rows.
constexpr uint32_t kRunRow = 0x80000000u;
// The run of a probe row paired with no build row (left outer without a
// match, semi and anti joins): one pair with build index -1.  (Build rows are
// below 2^31 - 1, so no flagged row collides with it.)
constexpr uint32_t kRunNone = 0xFFFFFFFFu;

__global__ void k_ht_runs(JoinHT H, const uint64_t* skey, const uint32_t* sval, long long n) {
    for (long long p = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; p < n;
         p += static_cast<long long>(gridDim.x) * blockDim.x) {
        const uint64_t s = skey[p];
        if (p == 0 || skey[p - 1] != s) {
            const bool single = p + 1 == n || skey[p + 1] != s;
            H.slots[s].z = single ? (sval[p] | kRunRow) : static_cast<uint32_t>(p);
        }
    }
}

size_t ht_bytes(long long n_build) {
    const long long cap = ht_cap(n_build);
    return static_cast<size_t>(cap + 1) * sizeof(uint4) + 256 +                 // slots
           2 * (static_cast<size_t>(n_build) * 12 + 256) + 256 +                // sort buffers
           radix_sort_scratch(n_build > 0 ? n_build : 1) + 256;
}

tqp_status ht_build(tqp_ctx* ctx, const tqp_table* build, int32_t key_col, JoinHT* H, cudaStream_t stream) {
    const long long n = build->num_rows;
    H->cap = ht_cap(n) * ht_scale(ctx);
    H->slots = static_cast<uint4*>(arena_alloc(ctx, static_cast<size_t>(H->cap + 1) * sizeof(uint4)));
    const long long nn = n > 0 ? n : 1;
    unsigned char* sb = static_cast<unsigned char*>(arena_alloc(ctx, 2 * (static_cast<size_t>(nn) * 12 + 256)));
    void* rs = arena_alloc(ctx, radix_sort_scratch(nn));
    long long* d_n = static_cast<long long*>(arena_alloc(ctx, 256));
    long long* meta = static_cast<long long*>(arena_alloc(ctx, 64));
    if (!H->slots || !sb || !rs || !d_n || !meta) return arena_oom(ctx, ht_bytes(n));
    // the build keys' range first: dense keys make the table direct-mapped
    H->meta = meta;
    TQP_TRY(ht_key_range_launch(ctx, build, key_col, meta, stream));
    uint64_t* k0 = reinterpret_cast<uint64_t*>(sb);
    uint64_t* k1 = k0 + nn;
    uint32_t* v0 = reinterpret_cast<uint32_t*>(k1 + nn);
    uint32_t* v1 = v0 + nn;
    const int threads = 256;
    const int blocks = static_cast<int>(std::min<long long>((H->cap + threads) / threads, ctx->num_sms * 16LL));
    k_ht_init<<<blocks, threads, 0, stream>>>(*H);
    TQP_CUDA(cudaGetLastError());
    H->bidx = v0;
    if (n == 0) return TQP_OK;
    const tqp_column& kc = build->cols[key_col];
    const int iblocks = static_cast<int>(std::min<long long>((n + threads - 1) / threads, ctx->num_sms * 16LL));
    k_ht_insert<<<iblocks, threads, 0, stream>>>(*H, static_cast<const unsigned char*>(kc.data), kc.type, n, k0, v0,
                                                 ctx->d_err);
    TQP_TRY(set_device_i64(d_n, n, stream));
    int bits = 1;
    while ((1LL << bits) <= H->cap) ++bits;
    bool in1 = false;
    TQP_TRY(radix_sort_pairs(k0, v0, k1, v1, d_n, n, 0, (bits + 7) / 8 * 8, rs, stream, &in1));
    const uint64_t* sk = in1 ? k1 : k0;
    H->bidx = in1 ? v1 : v0;
    k_ht_runs<<<iblocks, threads, 0, stream>>>(*H, sk, H->bidx, n);
    TQP_CUDA(cudaGetLastError());
    return TQP_OK;
}

// ---- sort-based build (paper Section 5.2, Algorithm 1) ---------------------------
// The build keys (minus their minimum) are radix-sorted with their rows; the
// probe bucketizes each key into the sorted keys through a radix directory
// over the key range (the top bits of key - min select a bucket, a binary
// search within the bucket finds the run).  The sorted rows are the build
// rows of each key in ascending order, as the canonical output wants.

__global__ void k_sj_keys(const long long* meta, const unsigned char* key_col, int key_type, long long n,
                          uint64_t* skey, uint32_t* sval) {
    const long long kmin = __ldg(&meta[0]);
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        skey[i] = static_cast<uint64_t>(ldg_typed(key_col, key_type, i)) - static_cast<uint64_t>(kmin);
        sval[i] = static_cast<uint32_t>(i);
    }
}

// meta[2] = bucket shift: the key range's bit length beyond log2(nbuckets).
__global__ void k_sj_shift(long long* meta, int dir_bits) {
    const unsigned long long range = static_cast<unsigned long long>(meta[1]) - static_cast<unsigned long long>(meta[0]);
    const int bits = range ? 64 - __clzll(static_cast<long long>(range)) : 0;
    meta[2] = bits > dir_bits ? bits - dir_bits : 0;
}

// sdir[b] = the first sorted index whose key lies in bucket >= b.
__global__ void k_sj_dir(const long long* meta, const uint64_t* skey, long long n, uint32_t* sdir, long long nb) {
    const int sh = static_cast<int>(__ldg(&meta[2]));
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i <= n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long b_i = i < n ? static_cast<long long>(skey[i] >> sh) : nb;
        const long long b_p = i > 0 ? static_cast<long long>(skey[i - 1] >> sh) : -1;
        for (long long b = b_p + 1; b <= b_i && b <= nb; ++b) sdir[b] = static_cast<uint32_t>(i);
    }
}

tqp_status ht_build_sorted(tqp_ctx* ctx, const tqp_table* build, int32_t key_col, JoinHT* H, cudaStream_t stream) {
    const long long n = build->num_rows;
    const long long nn = n > 0 ? n : 1;
    int dir_bits = 1;
    while ((1LL << dir_bits) < nn) ++dir_bits;
    const long long nb = 1LL << dir_bits;
    unsigned char* sb = static_cast<unsigned char*>(arena_alloc(ctx, 2 * (static_cast<size_t>(nn) * 12 + 256)));
    void* rs = arena_alloc(ctx, radix_sort_scratch(nn));
    long long* d_n = static_cast<long long*>(arena_alloc(ctx, 256));
    long long* meta = static_cast<long long*>(arena_alloc(ctx, 64));
    uint32_t* sdir = static_cast<uint32_t*>(arena_alloc(ctx, static_cast<size_t>(nb + 1) * 4));
    if (!sb || !rs || !d_n || !meta || !sdir)
        return arena_oom(ctx, 2 * (static_cast<size_t>(nn) * 12 + 256) + radix_sort_scratch(nn) + (nb + 1) * 4 + 512);
    memset(H, 0, sizeof(*H));
    H->cap = 0;
    H->meta = meta;
    H->nbuild = n;
    H->nbuckets = nb;
    H->sdir = sdir;
    TQP_TRY(ht_key_range_launch(ctx, build, key_col, meta, stream));
    uint64_t* k0 = reinterpret_cast<uint64_t*>(sb);
    uint64_t* k1 = k0 + nn;
    uint32_t* v0 = reinterpret_cast<uint32_t*>(k1 + nn);
    uint32_t* v1 = v0 + nn;
    H->skeys = k0;
    H->bidx = v0;
    if (n == 0) return TQP_OK;
    const tqp_column& kc = build->cols[key_col];
    const int threads = 256;
    const int blocks = static_cast<int>(std::min<long long>((n + threads - 1) / threads, ctx->num_sms * 16LL));
    k_sj_keys<<<blocks, threads, 0, stream>>>(meta, static_cast<const unsigned char*>(kc.data), kc.type, n, k0, v0);
    k_sj_shift<<<1, 1, 0, stream>>>(meta, dir_bits);
    TQP_CUDA(cudaGetLastError());
    TQP_TRY(set_device_i64(d_n, n, stream));
    bool in1 = false;
    // key - min fits 32 bits for 32- and 8-bit key columns
    TQP_TRY(radix_sort_pairs(k0, v0, k1, v1, d_n, n, 0, kc.type == TQP_I64 ? 64 : 32, rs, stream, &in1));
    H->skeys = in1 ? k1 : k0;
    H->bidx = in1 ? v1 : v0;
    const int dblocks = static_cast<int>(std::min<long long>((n + threads) / threads, ctx->num_sms * 16LL));
    k_sj_dir<<<dblocks, threads, 0, stream>>>(meta, H->skeys, n, sdir, nb);
    TQP_CUDA(cudaGetLastError());
    return TQP_OK;
}

// ---- probe with pair output ----------------------------------------------------

struct ProbeArgs {
    ScanGeom G;
    EngineCtl ctl;
    JoinHT H{};
    int32_t key_col;
    int32_t kind;                // tqp_join_kind
    uint2* row_run;              // per probe row: its key's run (first bidx index, length); length 0: no match
    int32_t* out_build;
    int32_t* out_probe;
    int64_t capacity;
    int64_t* d_count;
    unsigned long long* status;  // per-chunk look-back words
    unsigned long long* acc;     // [0] pairs, [1] finished warps
};

struct ProbeBody {
    static constexpr int kSmemBytes = 256;
    const ProbeArgs& A;
    unsigned long long* wtot;     // [2][warps]
    unsigned long long* excl_sm;
    int* skipped_sm;              // some consumer warp of this CTA skipped a tile (a wait gave up)
    unsigned long long chunk_pairs = 0;  // lane 0
    unsigned long long my_pairs = 0;     // lane 0
    long long tiles_seen = 0;            // tiles of the current chunk this warp processed

    __device__ ProbeBody(const ProbeArgs& a, unsigned char* sm) : A(a) {
        wtot = reinterpret_cast<unsigned long long*>(sm);
        excl_sm = wtot + 2 * kConsumerWarps;
        skipped_sm = reinterpret_cast<int*>(excl_sm + 1);
        if (threadIdx.x == 0) *skipped_sm = 0;  // ordered before use by the engine's first __syncthreads
    }

    // Four rows per lane: their home slots are loaded together, then each
    // row walks its probe sequence (rarely past the home slot at load factor
    // <= 1/2) and records its key's run for the second pass.
    __device__ void pass1(const ScanGeom& G, const TileView& v, int cw, int lane) {
        ++tiles_seen;
        const int rw = G.T / kConsumerWarps;  // a multiple of 128
        const JoinHT& H = A.H;
        const unsigned long long mask = static_cast<unsigned long long>(H.cap - 1);
        long long kmin = 0;
        const bool direct = ht_is_direct(H, &kmin);
        unsigned long long pairs = 0;
        if (H.skeys) {  // sort-based table: bucketize each key into the sorted build keys
            for (int base = cw * rw; base < cw * rw + rw; base += kWarp) {
                const int r = base + lane;
                if (base >= v.rows) break;
                if (r >= v.rows) continue;
                uint2 run = sj_lookup(H, static_cast<uint64_t>(col_val(G, v, A.key_col, r)));
                if (A.kind != TQP_JOIN_INNER) {
                    const bool keep = A.kind == TQP_JOIN_LEFT_SEMI ? run.y != 0 : run.y == 0;
                    if (keep) run = make_uint2(kRunNone, 1u);
                    else if (A.kind != TQP_JOIN_LEFT_OUTER) run = make_uint2(0u, 0u);
                }
                pairs += run.y;
                A.row_run[v.row0 + r] = run;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
            if (lane == 0) chunk_pairs += pairs;
            return;
        }
        for (int base = cw * rw; base < cw * rw + rw; base += 4 * kWarp) {
            if (base >= v.rows) break;
            uint64_t key[4];
            unsigned long long h[4];
            uint4 sl[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int r = base + kWarp * j + lane;
                key[j] = 0;
                h[j] = 0;
                sl[j] = make_uint4(0u, 0u, 0u, 0u);
                if (r < v.rows) {
                    key[j] = static_cast<uint64_t>(col_val(G, v, A.key_col, r));
                    if (direct) {
                        h[j] = key[j] - static_cast<uint64_t>(kmin);
                        if (h[j] < static_cast<unsigned long long>(H.cap)) sl[j] = __ldg(&H.slots[h[j]]);
                    } else {
                        h[j] = key[j] == ~0ULL ? static_cast<unsigned long long>(H.cap) : (mix64(key[j]) & mask);
                        sl[j] = __ldg(&H.slots[h[j]]);
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int r = base + kWarp * j + lane;
                if (r >= v.rows) continue;
                uint4 s = sl[j];
                bool hit;
                if (direct) {  // the key's own slot (zero when out of range): any rows are matches
                    hit = s.w != 0;
                } else if (key[j] == ~0ULL) {  // the all-ones key lives in the extra slot
                    hit = s.w != 0;
                } else {
                    unsigned long long hh = h[j];
                    for (long long i = 0; i < H.cap; ++i) {
                        const uint64_t k = slot_key(s);
                        if (k == key[j] || k == ~0ULL) break;
                        hh = (hh + 1) & mask;
                        s = __ldg(&H.slots[hh]);
                    }
                    hit = slot_key(s) == key[j];
                }
                uint2 run = hit ? make_uint2(s.z, s.w) : make_uint2(0u, 0u);
                if (A.kind != TQP_JOIN_INNER) {  // one pair (r, -1), or none, for this row
                    const bool keep = A.kind == TQP_JOIN_LEFT_SEMI ? run.y != 0 : run.y == 0;
                    if (keep) run = make_uint2(kRunNone, 1u);
                    else if (A.kind != TQP_JOIN_LEFT_OUTER) run = make_uint2(0u, 0u);
                }
                pairs += run.y;
                A.row_run[v.row0 + r] = run;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
        if (lane == 0) chunk_pairs += pairs;
    }

    __device__ void chunk_end(const ScanGeom& G, long long chunk, long long t0, long long t1, int cw, int lane) {
        if (lane == 0) {
            my_pairs += chunk_pairs;
            wtot[cw] = chunk_pairs;
            // a skipped tile left its rows' runs unwritten: the second pass
            // below must not read them (the call reports TQP_ERR_TIMEOUT)
            if (tiles_seen != t1 - t0) *skipped_sm = 1;
        }
        chunk_pairs = 0;
        tiles_seen = 0;
        named_sync(kBarConsumers, kConsumers);
        if (cw == 0) {
            unsigned long long c = lane < kConsumerWarps ? wtot[lane] : 0ULL;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
            const unsigned long long ex = lookback(A.status, chunk, c, lane, A.ctl.err, A.ctl.wait_cap);
            if (lane == 0) *excl_sm = ex;
        }
        named_sync(kBarConsumers, kConsumers);
        if (*skipped_sm) return;  // CTA-uniform: every consumer warp reads it after the same barrier
        unsigned long long running = *excl_sm;
        const long long r_begin = t0 * G.T;  // a multiple of 1024: every lane's four rows start 32-byte aligned
        const long long r_end = (t1 * G.T < G.n) ? t1 * G.T : G.n;
        int par = 0;
        // rounds of 4 * kConsumers rows, four consecutive rows per lane (row order = lane order)
        for (long long base = r_begin; base < r_end; base += 4 * kConsumers) {
            const long long r0 = base + 4LL * (cw * kWarp + lane);
            uint2 run[4];
            if (r0 + 4 <= r_end) {
                const uint4* p = reinterpret_cast<const uint4*>(A.row_run + r0);
                const uint4 a = p[0], b = p[1];
                run[0] = make_uint2(a.x, a.y);
                run[1] = make_uint2(a.z, a.w);
                run[2] = make_uint2(b.x, b.y);
                run[3] = make_uint2(b.z, b.w);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) run[j] = r0 + j < r_end ? A.row_run[r0 + j] : make_uint2(0u, 0u);
            }
            const unsigned long long c = static_cast<unsigned long long>(run[0].y) + run[1].y + run[2].y + run[3].y;
            unsigned long long incl = c;
#pragma unroll
            for (int o = 1; o < kWarp; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane == kWarp - 1) wtot[par * kConsumerWarps + cw] = incl;
            named_sync(kBarConsumers, kConsumers);
            unsigned long long before = 0, round_total = 0;
#pragma unroll
            for (int w = 0; w < kConsumerWarps; ++w) {
                const unsigned long long x = wtot[par * kConsumerWarps + w];
                before += (w < cw) ? x : 0ULL;
                round_total += x;
            }
            unsigned long long pos = running + before + (incl - c);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (run[j].x & kRunRow) {  // a unique key: the run is the build row itself (or none: -1)
                    if (run[j].y && pos < static_cast<unsigned long long>(A.capacity)) {
                        A.out_build[pos] = run[j].x == kRunNone ? -1 : static_cast<int32_t>(run[j].x & ~kRunRow);
                        A.out_probe[pos] = static_cast<int32_t>(r0 + j);
                    }
                    pos += run[j].y;
                    continue;
                }
                for (uint32_t k = 0; k < run[j].y; ++k, ++pos) {
                    if (pos < static_cast<unsigned long long>(A.capacity)) {
                        A.out_build[pos] = static_cast<int32_t>(A.H.bidx[run[j].x + k]);
                        A.out_probe[pos] = static_cast<int32_t>(r0 + j);
                    }
                }
            }
            running += round_total;
            par ^= 1;
        }
    }

    __device__ void finish(const ScanGeom&, int cw, int lane) {
        if (lane == 0) {
            if (my_pairs) atomicAdd(&A.acc[0], my_pairs);
            __threadfence();
            const unsigned long long done = atomicAdd(&A.acc[1], 1ULL);
            if (done == static_cast<unsigned long long>(gridDim.x) * kConsumerWarps - 1) {
                __threadfence();
                const unsigned long long tot = atomicAdd(&A.acc[0], 0ULL);
                *A.d_count = static_cast<int64_t>(tot);
                if (static_cast<long long>(tot) > A.capacity) latch_error(A.ctl.err, TQP_ERR_CAPACITY);
            }
        }
    }
};

__global__ void __launch_bounds__(kEngineThreads, 2) k_join_probe(const __grid_constant__ ProbeArgs P) {
    extern __shared__ __align__(128) unsigned char smem[];
    const ProbeArgs& A = stage_args(P, smem + kHeaderBytes);
    ProbeBody body(A, smem + kHeaderBytes + args_bytes<ProbeArgs>());
    run_engine(A.G, A.ctl, body, smem, args_bytes<ProbeArgs>());
}

tqp_status launch_hash_join(tqp_ctx* ctx, const tqp_table* build, int32_t build_key, const tqp_table* probe,
                            int32_t probe_key, int32_t kind, int32_t* d_build_idx, int32_t* d_probe_idx,
                            int64_t capacity, int64_t* d_count, cudaStream_t stream) {
    JoinHT H{};
    // variant 1: the sort-based join; 0: the hash table (the autotuner times both)
    if (tuned_variant(ctx) == 1) TQP_TRY(ht_build_sorted(ctx, build, build_key, &H, stream));
    else TQP_TRY(ht_build(ctx, build, build_key, &H, stream));
    if (probe->num_rows == 0) {
        TQP_CUDA(cudaMemsetAsync(d_count, 0, sizeof(int64_t), stream));
        return TQP_OK;
    }
    ProbeArgs A;
    memset(&A, 0, sizeof(A));
    A.H = H;
    A.key_col = probe_key;
    A.kind = kind;
    const int es = probe->cols[probe_key].type == TQP_I64 ? 8 : (probe->cols[probe_key].type == TQP_I32 ? 4 : 1);
    const tqp_tuning tu = default_tuning(ctx, es, ProbeBody::kSmemBytes + args_bytes<ProbeArgs>());
    size_t smem = 0;
    TQP_TRY(make_geom(ctx, probe, std::vector<int>{probe_key}, tu, ProbeBody::kSmemBytes + args_bytes<ProbeArgs>(), &A.G, &smem));
    static SmemFlags attr_done;
    TQP_TRY(allow_smem(ctx, reinterpret_cast<const void*>(k_join_probe), attr_done));
    const int g = engine_grid(ctx, reinterpret_cast<const void*>(k_join_probe), smem, A.G.ntiles, tu.ctas_per_sm);
    A.ctl.chunk_tiles = (A.G.ntiles + g - 1) / g;
    A.ctl.nchunks = (A.G.ntiles + A.ctl.chunk_tiles - 1) / A.ctl.chunk_tiles;
    const size_t words = 3 + static_cast<size_t>(A.ctl.nchunks);
    unsigned long long* sc = static_cast<unsigned long long*>(arena_alloc(ctx, words * 8));
    A.row_run = static_cast<uint2*>(arena_alloc(ctx, static_cast<size_t>(probe->num_rows) * 8));
    if (!sc || !A.row_run) return arena_oom(ctx, words * 8 + static_cast<size_t>(probe->num_rows) * 8);
    TQP_CUDA(cudaMemsetAsync(sc, 0, words * 8, stream));
    A.ctl.ticket = sc;
    A.ctl.err = ctx->d_err;
    A.ctl.wait_cap = ctx->wait_cap;
    A.acc = sc + 1;
    A.status = sc + 3;
    A.out_build = d_build_idx;
    A.out_probe = d_probe_idx;
    A.capacity = capacity;
    A.d_count = d_count;
    k_join_probe<<<static_cast<int>(A.ctl.nchunks), kEngineThreads, smem, stream>>>(A);
    TQP_CUDA(cudaGetLastError());
    return TQP_OK;
}

}  // namespace tqp

using namespace tqp;

extern "C" tqp_status tqp_hash_join(tqp_ctx* ctx, const tqp_table* build, int32_t build_key, const tqp_table* probe,
                                    int32_t probe_key, int32_t* d_build_idx, int32_t* d_probe_idx, int64_t capacity,
                                    int64_t* d_count, void* stream) {
    return tqp_hash_join_kind(ctx, build, build_key, probe, probe_key, TQP_JOIN_INNER, d_build_idx, d_probe_idx,
                              capacity, d_count, stream);
}

extern "C" tqp_status tqp_hash_join_kind(tqp_ctx* ctx, const tqp_table* build, int32_t build_key,
                                         const tqp_table* probe, int32_t probe_key, int32_t join_kind,
                                         int32_t* d_build_idx, int32_t* d_probe_idx, int64_t capacity,
                                         int64_t* d_count, void* stream) {
    clear_error();
    if (join_kind < TQP_JOIN_INNER || join_kind > TQP_JOIN_LEFT_OUTER)
        return fail(TQP_ERR_INVALID_ARG, "join_kind %d is not a tqp_join_kind", join_kind);
    TQP_TRY(check_ctx(ctx));
    TQP_TRY(check_table(build, "tqp_hash_join(build)"));
    TQP_TRY(check_table(probe, "tqp_hash_join(probe)"));
    TQP_TRY(check_device_cols(build, {build_key}, "tqp_hash_join(build)"));
    TQP_TRY(check_device_cols(probe, {probe_key}, "tqp_hash_join(probe)"));
    if (build_key < 0 || build_key >= build->num_cols) return fail(TQP_ERR_INVALID_ARG, "build_key out of range");
    if (probe_key < 0 || probe_key >= probe->num_cols) return fail(TQP_ERR_INVALID_ARG, "probe_key out of range");
    TQP_TRY(check_numeric_cols(build, {build_key}, "tqp_hash_join(build)"));
    TQP_TRY(check_numeric_cols(probe, {probe_key}, "tqp_hash_join(probe)"));
    if (!d_count) return fail(TQP_ERR_INVALID_ARG, "d_count is NULL");
    if (capacity < 0) return fail(TQP_ERR_INVALID_ARG, "capacity < 0");
    if (capacity > 0 && (!d_build_idx || !d_probe_idx))
        return fail(TQP_ERR_INVALID_ARG, "output arrays are NULL");
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(TQP_ERR_CUDA, "cannot select device %d", ctx->device);
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    char key[96];
    snprintf(key, sizeof(key), "hashjoin%d r%d b%d n%d", join_kind, rows_class(probe->num_rows),
             row_bytes(probe, std::vector<int>{probe_key}), rows_class(build->num_rows));
    auto run = [&]() {
        arena_reset(ctx);
        return launch_hash_join(ctx, build, build_key, probe, probe_key, join_kind, d_build_idx, d_probe_idx,
                                capacity, d_count, st);
    };
    return tuned(ctx, key, st, kTuneHt | kTuneVariant, run);
}
