// Sort-based group-by aggregation (paper Section 5.4, Algorithm 3: sort the
// rows by their group key, cut the sorted keys into runs of equal keys,
// evaluate the aggregates per run) -- the group-by's variant 1, next to the
// hash aggregation; the autotuner times both.
//
//   k_sa_keys    rows passing the predicates append (packed group key, row)
//                pairs (warp-aggregated, so their order is arbitrary: a
//                group's aggregates do not depend on the order of its rows);
//   radix sort   of the pairs by the packed key (order-preserving packing, so
//                sorted keys are the groups in ascending key order);
//   k_sa_heads / k_sa_scan / k_sa_assign
//                run heads -> dense group ids (an exclusive scan of the head
//                flags), the packed key of each group;
//   k_sa_agg     each sorted row's aggregate values (gathered by row id) into
//                its group's accumulators.
// The dense table then goes through the same finalization / top-k as every
// other group-by (dense mode: entries [0, G) are the groups).
#include "host.h"
#include "group.cuh"

namespace tqp {

tqp_status radix_sort_pairs(uint64_t* k0, uint32_t* v0, uint64_t* k1, uint32_t* v1, const long long* d_n,
                            long long n_max, int begin_bit, int end_bit, void* scratch, cudaStream_t stream,
                            bool* result_in_1);
size_t radix_sort_scratch(long long n_max);

constexpr int kSaThreads = 256;
constexpr int kSaTile = 2048;  // sorted elements per scan tile

struct SortAggArgs {
    ScanGeom G;        // column pointers (nothing staged)
    int32_t ncond;
    int32_t pad;
    Cond cond[TQP_MAX_PREDS];
    GroupSpec S;       // dense mode: keys[G], acc[G * nacc], d_dense_n
    uint64_t* skey;    // appended pairs (then sorted in place by the radix sort)
    uint32_t* srow;
    long long* d_np;   // appended pairs (device)
    uint32_t* tile_sum;  // heads per scan tile
    uint32_t* gid;     // dense group of each sorted pair
    long long cap_groups;
    int* err;
};

__device__ __forceinline__ bool sa_pass(const SortAggArgs& A, long long r) {
    for (int q = 0; q < A.ncond; ++q) {
        const Cond& cd = A.cond[q];
        const ColRef& c = A.G.col[cd.col];
        const uint64_t x = static_cast<uint64_t>(ldg_typed(c.ptr, c.type, r));
        if (((x - static_cast<uint64_t>(cd.lo)) <= cd.span) == (cd.negate != 0)) return false;
    }
    return true;
}

__global__ void __launch_bounds__(kSaThreads) k_sa_keys(const __grid_constant__ SortAggArgs A) {
    const int lane = threadIdx.x % kWarp;
    const long long n = A.G.n;
    const long long stride = static_cast<long long>(gridDim.x) * kSaThreads;
    // every lane of a warp runs the same number of iterations (warp-uniform bound)
    const long long wbase = (blockIdx.x * static_cast<long long>(kSaThreads) + threadIdx.x) - lane;
    for (long long r0 = wbase; r0 < n; r0 += stride) {
        const long long r = r0 + lane;
        const bool ok = r < n && sa_pass(A, r);
        uint64_t key = 0;
        if (ok)
            for (int i = 0; i < A.S.ngc; ++i) {
                const int b = A.S.key_bits[i];
                const ColRef& c = A.G.col[A.S.key_col[i]];
                const uint64_t e = enc_key(ldg_typed(c.ptr, c.type, r), b);
                key = (b == 64) ? e : ((key << b) | e);
            }
        const uint32_t m = __ballot_sync(0xffffffffu, ok);
        unsigned long long base = 0;
        if (lane == 0 && m) base = atomicAdd(reinterpret_cast<unsigned long long*>(A.d_np), static_cast<unsigned long long>(__popc(m)));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (ok) {
            const unsigned long long pos = base + __popc(m & lanemask_lt());
            A.skey[pos] = key;
            A.srow[pos] = static_cast<uint32_t>(r);
        }
    }
}

// Heads (first pair of each run of equal keys) per tile of kSaTile pairs.
__global__ void __launch_bounds__(kSaThreads) k_sa_heads(const __grid_constant__ SortAggArgs A) {
    __shared__ uint32_t part[kSaThreads / kWarp];
    const long long np = *A.d_np;
    const long long t0 = blockIdx.x * static_cast<long long>(kSaTile);
    uint32_t c = 0;
    for (long long i = t0 + threadIdx.x; i < t0 + kSaTile && i < np; i += kSaThreads)
        c += (i == 0 || A.skey[i] != A.skey[i - 1]) ? 1u : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (threadIdx.x % kWarp == 0) part[threadIdx.x / kWarp] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kSaThreads / kWarp; ++w) t += part[w];
        A.tile_sum[blockIdx.x] = t;
    }
}

// One block: exclusive scan of the tile head counts; the total is the group count.
__global__ void __launch_bounds__(1024) k_sa_scan(const __grid_constant__ SortAggArgs A, long long ntiles) {
    __shared__ unsigned long long wsum[32];
    __shared__ unsigned long long carry;
    const int lane = threadIdx.x % kWarp, w = threadIdx.x / kWarp;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (long long b = 0; b < ntiles; b += 1024) {
        const long long i = b + threadIdx.x;
        const unsigned long long x = i < ntiles ? A.tile_sum[i] : 0;
        unsigned long long incl = x;
#pragma unroll
        for (int o = 1; o < kWarp; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == kWarp - 1) wsum[w] = incl;
        __syncthreads();
        unsigned long long before = 0, total = 0;
        for (int k = 0; k < 32; ++k) {
            before += k < w ? wsum[k] : 0;
            total += wsum[k];
        }
        const unsigned long long c0 = carry;
        __syncthreads();
        if (i < ntiles) A.tile_sum[i] = static_cast<uint32_t>(c0 + before + incl - x);
        if (threadIdx.x == 0) carry = c0 + total;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const long long G = static_cast<long long>(carry);
        if (G > A.cap_groups) latch_error(A.err, TQP_ERR_CAPACITY);
        *A.S.ndistinct = static_cast<unsigned long long>(G);  // the finalization reports G > bound as -1
        *const_cast<long long*>(A.S.d_dense_n) = G > A.cap_groups ? A.cap_groups : G;
    }
}

// Dense group id of every sorted pair; each head stores its group's packed key.
__global__ void __launch_bounds__(kSaThreads) k_sa_assign(const __grid_constant__ SortAggArgs A) {
    __shared__ uint32_t wsum[kSaThreads / kWarp];
    const long long np = *A.d_np;
    const long long t0 = blockIdx.x * static_cast<long long>(kSaTile);
    if (t0 >= np) return;
    constexpr int kPer = kSaTile / kSaThreads;  // consecutive pairs per thread
    const int lane = threadIdx.x % kWarp, w = threadIdx.x / kWarp;
    const long long i0 = t0 + static_cast<long long>(threadIdx.x) * kPer;
    uint32_t h[kPer], c = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const long long i = i0 + k;
        h[k] = (i < np && (i == 0 || A.skey[i] != A.skey[i - 1])) ? 1u : 0u;
        c += h[k];
    }
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < kWarp; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == kWarp - 1) wsum[w] = incl;
    __syncthreads();
    uint32_t before = 0;
    for (int k = 0; k < kSaThreads / kWarp; ++k) before += k < w ? wsum[k] : 0u;
    // inclusive count of heads through each pair, minus one: its dense group
    long long g = static_cast<long long>(A.tile_sum[blockIdx.x]) + before + (incl - c) - 1;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const long long i = i0 + k;
        if (i >= np) break;
        g += h[k];
        A.gid[i] = static_cast<uint32_t>(g);
        if (h[k] && g < A.cap_groups) A.S.keys[g] = A.skey[i];
    }
}

// Each sorted pair's aggregate values into its group's accumulators.
__global__ void __launch_bounds__(kSaThreads) k_sa_agg(const __grid_constant__ SortAggArgs A) {
    const long long np = *A.d_np;
    const GroupSpec& S = A.S;
    for (long long i = blockIdx.x * static_cast<long long>(kSaThreads) + threadIdx.x; i < np;
         i += static_cast<long long>(gridDim.x) * kSaThreads) {
        const long long g = A.gid[i];
        if (g >= A.cap_groups) continue;
        const long long r = A.srow[i];
        unsigned long long* a = S.acc + g * S.nacc;
        red_add_u64(&a[0], 1ULL);
        for (int k = 1; k < S.nacc; ++k) {
            const int64_t x = eval_expr_global(A.G, S.acc_expr[k - 1], r);
            const int kind = S.acc_kind[k - 1];
            if (kind == kAccSum) red_add_u64(&a[k], static_cast<unsigned long long>(x));
            else atomicMax(&a[k], acc_encode(kind, x));
        }
    }
}

size_t sort_agg_scratch_bytes(long long n, long long cap_groups, int nacc) {
    const long long nn = n > 0 ? n : 1;
    const long long ntiles = (nn + kSaTile - 1) / kSaTile;
    return 2 * static_cast<size_t>(nn) * 12 + 4 * 256 + radix_sort_scratch(nn) + static_cast<size_t>(ntiles) * 4 +
           static_cast<size_t>(nn) * 4 + static_cast<size_t>(cap_groups + 1) * (8 + 8 * nacc) + 1024;
}

// Variant 1 of launch_groupby: the sort-based aggregation into a dense table
// (S lowered by the caller; S.keys / S.acc / S.d_dense_n are set here).
tqp_status launch_sort_agg(tqp_ctx* ctx, const tqp_table* t, const Cond* cond, int ncond, GroupSpec* S,
                           long long cap_groups, cudaStream_t stream) {
    const long long n = t->num_rows;
    const long long nn = n > 0 ? n : 1;
    const long long ntiles = (nn + kSaTile - 1) / kSaTile;
    SortAggArgs A;
    memset(&A, 0, sizeof(A));
    A.G.n = n;
    A.G.ncols = t->num_cols;
    for (int c = 0; c < t->num_cols; ++c) {
        A.G.col[c].ptr = static_cast<const unsigned char*>(t->cols[c].data);
        A.G.col[c].type = t->cols[c].type;
        A.G.col[c].slot = -1;
    }
    A.ncond = ncond;
    for (int q = 0; q < ncond; ++q) A.cond[q] = cond[q];
    uint64_t* k0 = static_cast<uint64_t*>(arena_alloc(ctx, static_cast<size_t>(nn) * 8));
    uint64_t* k1 = static_cast<uint64_t*>(arena_alloc(ctx, static_cast<size_t>(nn) * 8));
    uint32_t* v0 = static_cast<uint32_t*>(arena_alloc(ctx, static_cast<size_t>(nn) * 4));
    uint32_t* v1 = static_cast<uint32_t*>(arena_alloc(ctx, static_cast<size_t>(nn) * 4));
    void* rs = arena_alloc(ctx, radix_sort_scratch(nn));
    long long* words = static_cast<long long*>(arena_alloc(ctx, 256));  // [0] pairs, [1] groups kept, [2] groups
    uint32_t* tsum = static_cast<uint32_t*>(arena_alloc(ctx, static_cast<size_t>(ntiles) * 4));
    uint32_t* gid = static_cast<uint32_t*>(arena_alloc(ctx, static_cast<size_t>(nn) * 4));
    unsigned long long* keys = static_cast<unsigned long long*>(arena_alloc(ctx, static_cast<size_t>(cap_groups + 1) * 8));
    unsigned long long* acc =
        static_cast<unsigned long long*>(arena_alloc(ctx, static_cast<size_t>(cap_groups + 1) * S->nacc * 8));
    if (!k0 || !k1 || !v0 || !v1 || !rs || !words || !tsum || !gid || !keys || !acc)
        return arena_oom(ctx, sort_agg_scratch_bytes(n, cap_groups, S->nacc));
    TQP_CUDA(cudaMemsetAsync(words, 0, 24, stream));
    TQP_CUDA(cudaMemsetAsync(acc, 0, static_cast<size_t>(cap_groups + 1) * S->nacc * 8, stream));
    S->keys = keys;
    S->acc = acc;
    S->cap = cap_groups;
    S->max_groups = cap_groups;
    S->ndistinct = reinterpret_cast<unsigned long long*>(words + 2);
    S->d_dense_n = words + 1;
    A.S = *S;
    A.skey = k0;
    A.srow = v0;
    A.d_np = words;
    A.tile_sum = tsum;
    A.gid = gid;
    A.cap_groups = cap_groups;
    A.err = ctx->d_err;
    const int blocks = static_cast<int>(std::min<long long>((nn + kSaThreads - 1) / kSaThreads, 8LL * ctx->num_sms));
    k_sa_keys<<<blocks, kSaThreads, 0, stream>>>(A);
    TQP_CUDA(cudaGetLastError());
    bool in1 = false;
    const int end_bit = std::max(8, (S->width + 7) / 8 * 8);
    TQP_TRY(radix_sort_pairs(k0, v0, k1, v1, words, nn, 0, end_bit, rs, stream, &in1));
    A.skey = in1 ? k1 : k0;
    A.srow = in1 ? v1 : v0;
    k_sa_heads<<<static_cast<unsigned>(ntiles), kSaThreads, 0, stream>>>(A);
    k_sa_scan<<<1, 1024, 0, stream>>>(A, ntiles);
    k_sa_assign<<<static_cast<unsigned>(ntiles), kSaThreads, 0, stream>>>(A);
    k_sa_agg<<<blocks, kSaThreads, 0, stream>>>(A);
    TQP_CUDA(cudaGetLastError());
    return TQP_OK;
}

}  // namespace tqp
