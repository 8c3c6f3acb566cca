// tqp_filter: predicate evaluation + stream compaction + fused projection-sum.
//
// Paper Section 3.1 (Listing 1: comparison mask then masked_select; the
// selection-vector variant uses nonzero + index_select) and Section 5.1
// (expressions).  Two kernels, no host synchronisation and no inter-CTA
// waiting on the streaming path:
//   k_filter   the staged scan: the producer warp stages the predicate
//              columns in shared memory with bulk asynchronous copies; consumer
//              warps evaluate the conjunction lane-per-row, take one warp
//              ballot per 32 rows and store it (a 1-bit-per-row selection
//              mask, 1/128 of a 16-byte row), count with popc into per-block
//              totals, and evaluate the sum expression for passing rows only
//              (columns that are not staged are read lazily);
//   k_compact  expands the mask (written moments before, so read from L2)
//              into ascending int32 row ids: each block takes the total of all
//              earlier blocks as its offset, then scans its own words with
//              warp ballots/shuffles and writes ids with coalesced stores.
// Count and sum are reduced per warp and added once per warp to scratch; the
// last warp to finish publishes them.
//
// An earlier single-kernel form that chained tiles with a decoupled look-back
// (per tile, then per chunk) was measured slower on GB300: per-tile look-back
// advances the published-prefix frontier only ~32 tiles per L2 round trip, and
// a per-chunk look-back leaves the expansion as a serial tail.  The offsets
// here come straight from counts that are complete when k_compact starts.
#include <mutex>

#include <cstdio>

#include "host.h"
#include "bodies.cuh"

namespace tqp {



// Scratch layout (bytes): ticket + acc[3], block totals, then the mask.
struct FilterScratch {
    size_t tot_off, mask_off, bytes;
    long long nblocks;
};

static FilterScratch filter_scratch_layout(const ScanGeom& G, bool ids) {
    FilterScratch s;
    s.nblocks = ids ? (G.n + kCompactRows - 1) / kCompactRows : 0;
    s.tot_off = 4 * sizeof(unsigned long long);
    s.mask_off = (s.tot_off + s.nblocks * sizeof(uint32_t) + 255) / 256 * 256;
    s.bytes = s.mask_off + (ids ? static_cast<size_t>(G.ntiles) * (G.T / kWarp) * sizeof(uint32_t) : 0);
    return s;
}


__global__ void __launch_bounds__(kEngineThreads, 2) k_filter(const __grid_constant__ FilterArgs P) {
    extern __shared__ __align__(128) unsigned char smem[];
    const FilterArgs& A = stage_args(P, smem + kHeaderBytes);
    FilterBody body(A, smem + kHeaderBytes + args_bytes<FilterArgs>());
    run_engine(A.G, A.ctl, body, smem, args_bytes<FilterArgs>());
}

// ---- direct form (variant 1): no staging ------------------------------------------
// Every thread reads quads (four consecutive rows) of each predicate column
// with one 16-byte load per 32-bit column (two per 64-bit column, one 4-byte
// load per 8-bit column), kFdQuads quads at a time, at full occupancy: plain
// loads with many in flight instead of bulk copies through a stage ring.  A
// warp's 32 quads are 128 consecutive rows, so its pass bits form four mask
// words in the layout the compaction kernel reads; the sum expression is
// evaluated for passing rows only, from global memory.
constexpr int kFdThreads = 256;
constexpr int kFdQuads = 1;  // warp steps (32 quads each) per iteration of a warp

constexpr int kFdConds = 4;  // conditions of the direct form (more: the staged scan)

// The raw values of one quad of one condition column: 64-bit columns in
// a.x, a.y, b.x, b.y; 32-bit ones in the four words of a; 8-bit ones in a.x.
struct FdRaw {
    longlong2 a, b;
};

__device__ __forceinline__ FdRaw fd_load(const unsigned char* p, int type, long long q, long long n) {
    FdRaw r;
    r.a = make_longlong2(0, 0);
    r.b = make_longlong2(0, 0);
    if (4 * q + 3 < n) {
        if (type == TQP_I64) {
            r.a = __ldg(reinterpret_cast<const longlong2*>(p) + 2 * q);
            r.b = __ldg(reinterpret_cast<const longlong2*>(p) + 2 * q + 1);
        } else if (type == TQP_I32) {
            r.a = __ldg(reinterpret_cast<const longlong2*>(p) + q);
        } else {
            r.a.x = __ldg(reinterpret_cast<const unsigned int*>(p) + q);
        }
        return r;
    }
    // a partial last quad: row by row, the missing rows read as 0 (they fail anyway)
    long long x[4] = {0, 0, 0, 0};
    for (int j = 0; j < 4; ++j)
        if (4 * q + j < n) x[j] = ldg_typed(p, type, 4 * q + j);
    if (type == TQP_I64) {
        r.a = make_longlong2(x[0], x[1]);
        r.b = make_longlong2(x[2], x[3]);
    } else if (type == TQP_I32) {
        r.a.x = static_cast<long long>(static_cast<uint32_t>(x[0]) | (static_cast<uint64_t>(static_cast<uint32_t>(x[1])) << 32));
        r.a.y = static_cast<long long>(static_cast<uint32_t>(x[2]) | (static_cast<uint64_t>(static_cast<uint32_t>(x[3])) << 32));
    } else {
        r.a.x = static_cast<long long>((x[0] & 0xFF) | ((x[1] & 0xFF) << 8) | ((x[2] & 0xFF) << 16) | ((x[3] & 0xFF) << 24));
    }
    return r;
}

__device__ __forceinline__ uint32_t fd_test(const CondFast& f, const FdRaw& r) {
    uint32_t m = 0;
    if (f.type == TQP_I64) {
        const uint64_t x[4] = {static_cast<uint64_t>(r.a.x), static_cast<uint64_t>(r.a.y), static_cast<uint64_t>(r.b.x),
                               static_cast<uint64_t>(r.b.y)};
#pragma unroll
        for (int j = 0; j < 4; ++j) m |= static_cast<uint32_t>(x[j] - static_cast<uint64_t>(f.lo) <= f.span) << j;
    } else {
        uint32_t x[4];
        if (f.type == TQP_I32) {
            x[0] = static_cast<uint32_t>(r.a.x);
            x[1] = static_cast<uint32_t>(static_cast<uint64_t>(r.a.x) >> 32);
            x[2] = static_cast<uint32_t>(r.a.y);
            x[3] = static_cast<uint32_t>(static_cast<uint64_t>(r.a.y) >> 32);
        } else {
            const uint32_t w = static_cast<uint32_t>(r.a.x);
#pragma unroll
            for (int j = 0; j < 4; ++j) x[j] = (w >> (8 * j)) & 0xFFu;
        }
        const uint32_t lo = static_cast<uint32_t>(f.lo), sp = static_cast<uint32_t>(f.span);
#pragma unroll
        for (int j = 0; j < 4; ++j) m |= static_cast<uint32_t>(x[j] - lo <= sp) << j;
    }
    return f.negate ? ~m & 0xFu : m;
}

// Per warp: passing row ids whose sum is still to be evaluated (two steps of
// at most 128 rows each plus a partial round of fewer than 32).
constexpr int kFdQueue = kFdQuads * 4 * kWarp + kWarp;

__global__ void __launch_bounds__(kFdThreads, 4) k_filter_direct(const __grid_constant__ FilterArgs A) {
    __shared__ unsigned long long red[2][kFdThreads / kWarp];
    __shared__ uint32_t queue[kFdThreads / kWarp][kFdQueue];
    const int lane = threadIdx.x % kWarp, w = threadIdx.x / kWarp;
    uint32_t* q = queue[w];
    int qn = 0;  // queued rows (warp-uniform)
    const long long n = A.G.n;
    const long long nq = (n + 3) / 4;
    const long long nsteps = (nq + kWarp - 1) / kWarp;  // warp steps of 32 quads
    const long long warps = static_cast<long long>(gridDim.x) * (kFdThreads / kWarp);
    const long long gw = blockIdx.x * static_cast<long long>(kFdThreads / kWarp) + w;
    unsigned long long cnt = 0;
    long long sum = 0;
    for (long long s0 = gw; s0 < nsteps; s0 += kFdQuads * warps) {
        uint32_t bits[kFdQuads];
        FdRaw raw[kFdQuads][kFdConds];
#pragma unroll
        for (int u = 0; u < kFdQuads; ++u) {  // every load of the iteration in flight together
            const long long st = s0 + u * warps;
            const long long q = st * kWarp + lane;
#pragma unroll
            for (int c = 0; c < kFdConds; ++c)
                if (c < A.ncond && st < nsteps) raw[u][c] = fd_load(A.G.col[A.cond[c].col].ptr, A.cf[c].type, q, n);
        }
#pragma unroll
        for (int u = 0; u < kFdQuads; ++u) {
            const long long st = s0 + u * warps;
            const long long q = st * kWarp + lane;
            uint32_t ok = 0;
            if (st < nsteps) {
                ok = 0xFu;
                if (4 * q + 3 >= n)
                    for (int j = 0; j < 4; ++j) ok &= ~(static_cast<uint32_t>(4 * q + j >= n) << j);
#pragma unroll
                for (int c = 0; c < kFdConds; ++c)
                    if (c < A.ncond) ok &= fd_test(A.cf[c], raw[u][c]);
            }
            bits[u] = ok;
        }
#pragma unroll
        for (int u = 0; u < kFdQuads; ++u) {
            const long long st = s0 + u * warps;
            if (st >= nsteps) break;  // (warp-uniform)
            // word k of the step: the nibbles of lanes 8k .. 8k+7
            uint32_t v = bits[u] << (4 * (lane & 7));
            v |= __shfl_xor_sync(0xffffffffu, v, 1);
            v |= __shfl_xor_sync(0xffffffffu, v, 2);
            v |= __shfl_xor_sync(0xffffffffu, v, 4);
            const uint32_t w0 = __shfl_sync(0xffffffffu, v, 0), w1 = __shfl_sync(0xffffffffu, v, 8),
                           w2 = __shfl_sync(0xffffffffu, v, 16), w3 = __shfl_sync(0xffffffffu, v, 24);
            const uint32_t c = __popc(w0) + __popc(w1) + __popc(w2) + __popc(w3);  // (warp-uniform)
            const long long row0 = st * kWarp * 4;
            if (lane == 0) {
                cnt += c;
                if (A.mask && c) atomicAdd(&A.block_tot[row0 / kCompactRows], c);
                if (A.mask) *reinterpret_cast<uint4*>(A.mask + row0 / kWarp) = make_uint4(w0, w1, w2, w3);
            }
            if (A.has_sum && c) {  // queue the passing rows; evaluate them 32 at a time
                const uint32_t lt = lanemask_lt();
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint32_t m = __ballot_sync(0xffffffffu, (bits[u] >> j) & 1u);
                    if ((bits[u] >> j) & 1u) q[qn + __popc(m & lt)] = static_cast<uint32_t>(row0 + 4 * lane + j);
                    qn += __popc(m);
                }
                __syncwarp();
            }
        }
        if (A.has_sum && qn >= kWarp) {
            int h = 0;
            for (; qn - h >= kWarp; h += kWarp) sum += eval_expr_global(A.G, A.sum, q[h + lane]);
            const uint32_t keep = lane < qn - h ? q[h + lane] : 0u;
            __syncwarp();
            if (lane < qn - h) q[lane] = keep;
            qn -= h;
            __syncwarp();
        }
    }
    if (A.has_sum && lane < qn) sum += eval_expr_global(A.G, A.sum, q[lane]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) {
        red[0][w] = cnt;
        red[1][w] = static_cast<unsigned long long>(sum);
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    unsigned long long tc = 0, ts = 0;
    for (int i = 0; i < kFdThreads / kWarp; ++i) {
        tc += red[0][i];
        ts += red[1][i];
    }
    if (ts) atomicAdd(&A.acc[0], ts);
    if (tc) atomicAdd(&A.acc[1], tc);
    __threadfence();
    if (atomicAdd(&A.acc[2], 1ULL) != static_cast<unsigned long long>(gridDim.x) - 1ULL) return;
    __threadfence();
    const unsigned long long tot_sum = atomicAdd(&A.acc[0], 0ULL);
    const unsigned long long tot_cnt = atomicAdd(&A.acc[1], 0ULL);
    *A.d_count = static_cast<int64_t>(tot_cnt);
    if (A.d_count2) *A.d_count2 = static_cast<int64_t>(tot_cnt);
    if (A.d_sum) *A.d_sum = static_cast<int64_t>(tot_sum);
    if (A.mask && static_cast<long long>(tot_cnt) > A.capacity) latch_error(A.ctl.err, TQP_ERR_CAPACITY);
}

__global__ void __launch_bounds__(kCompactThreads) k_compact(const uint32_t* __restrict__ mask,
                                                             const uint32_t* __restrict__ block_tot, long long n,
                                                             int32_t* __restrict__ row_ids, long long capacity) {
    compact_block(mask, block_tot, n, row_ids, capacity, blockIdx.x);
}

// Lower a filter call into kernel arguments and a launch shape.
static tqp_status plan_filter(const tqp_ctx* ctx, const tqp_table* t, const tqp_pred* preds, int32_t npreds,
                              const tqp_expr* sum_expr, bool ids, const tqp_tuning* force, FilterArgs* A,
                              size_t* smem, int* grid, FilterScratch* lay) {
    memset(A, 0, sizeof(*A));
    int ncond = 0;
    TQP_TRY(lower_preds(t, preds, npreds, A->cond, &ncond));
    A->ncond = ncond;
    std::vector<int> staged;
    for (int i = 0; i < ncond; ++i) staged.push_back(A->cond[i].col);
    if (sum_expr) {
        TQP_TRY(lower_expr(sum_expr, t->num_cols, &A->sum));
        A->has_sum = 1;
        if (ncond == 0) expr_cols(A->sum, staged);  // every row passes: stage the summed columns
    }
    std::vector<int> u = staged;
    std::sort(u.begin(), u.end());
    u.erase(std::unique(u.begin(), u.end()), u.end());
    TQP_TRY(check_device_cols(t, u, "tqp_filter"));
    if (A->has_sum) {  // the rest are read in place at passing rows only
        std::vector<int> lazy;
        expr_cols(A->sum, lazy);
        TQP_TRY(check_numeric_cols(t, lazy, "tqp_filter sum_expr"));
        TQP_TRY(check_visible_cols(t, lazy, "tqp_filter"));
    }
    int bpr = 0;
    for (int c : u) bpr += t->cols[c].type == TQP_I64 ? 8 : (t->cols[c].type == TQP_I32 ? 4 : 1);
    const tqp_tuning tu = force ? *force : default_tuning(ctx, bpr, FilterBody::kSmemBytes + args_bytes<FilterArgs>());
    TQP_TRY(make_geom(ctx, t, staged, tu, FilterBody::kSmemBytes + args_bytes<FilterArgs>(), &A->G, smem));
    lower_fast(A->cond, A->ncond, A->G, A->cf, &A->fast);
    static SmemFlags attr_done;
    TQP_TRY(allow_smem(ctx, reinterpret_cast<const void*>(k_filter), attr_done));
    const int g = engine_grid(ctx, reinterpret_cast<const void*>(k_filter), *smem, A->G.ntiles, tu.ctas_per_sm);
    A->ctl.chunk_tiles = (A->G.ntiles + g - 1) / g;
    A->ctl.nchunks = (A->G.ntiles + A->ctl.chunk_tiles - 1) / A->ctl.chunk_tiles;
    *grid = static_cast<int>(A->ctl.nchunks);
    *lay = filter_scratch_layout(A->G, ids);
    return TQP_OK;
}

// Launch with caller-provided scratch of at least lay.bytes (cleared here).
static tqp_status launch_filter_with(FilterArgs& A, int grid, size_t smem, const FilterScratch& lay,
                                     void* scratch, int* d_err, long long wait_cap, int32_t* d_row_ids,
                                     int64_t capacity, int64_t* d_count, int64_t* d_sum, cudaStream_t stream,
                                     int direct_grid = 0) {
    unsigned char* sc = static_cast<unsigned char*>(scratch);
    TQP_CUDA(cudaMemsetAsync(sc, 0, lay.mask_off, stream));
    A.ctl.ticket = reinterpret_cast<unsigned long long*>(sc);
    A.ctl.err = d_err;
    A.ctl.wait_cap = wait_cap;
    A.acc = reinterpret_cast<unsigned long long*>(sc) + 1;
    A.block_tot = reinterpret_cast<uint32_t*>(sc + lay.tot_off);
    A.mask = d_row_ids ? reinterpret_cast<uint32_t*>(sc + lay.mask_off) : nullptr;
    A.capacity = capacity;
    A.d_count = d_count;
    A.d_sum = d_sum;
    if (direct_grid > 0) k_filter_direct<<<direct_grid, kFdThreads, 0, stream>>>(A);
    else k_filter<<<grid, kEngineThreads, smem, stream>>>(A);
    TQP_CUDA(cudaGetLastError());
    if (d_row_ids) {
        k_compact<<<static_cast<unsigned>(lay.nblocks), kCompactThreads, 0, stream>>>(A.mask, A.block_tot, A.G.n,
                                                                                       d_row_ids, capacity);
        TQP_CUDA(cudaGetLastError());
    }
    return TQP_OK;
}

tqp_status launch_filter(tqp_ctx* ctx, const tqp_table* t, const tqp_pred* preds, int32_t npreds,
                         const tqp_expr* sum_expr, int64_t* d_sum, int32_t* d_row_ids, int64_t capacity,
                         int64_t* d_count, cudaStream_t stream, const tqp_tuning* force) {
    // IN / LIKE / NOT LIKE: one pre-pass writes a pass column that the scan then filters on
    StrLowered SL;
    TQP_TRY(str_prepass(ctx, t, preds, npreds, stream, &SL));
    if (SL.active) {
        t = &SL.t;
        preds = SL.preds;
        npreds = SL.npreds;
    }
    FilterArgs A;
    size_t smem = 0;
    int grid = 0;
    FilterScratch lay;
    TQP_TRY(plan_filter(ctx, t, preds, npreds, sum_expr, d_row_ids != nullptr, force, &A, &smem, &grid, &lay));
    if (t->num_rows == 0) {
        TQP_CUDA(cudaMemsetAsync(d_count, 0, sizeof(int64_t), stream));
        if (d_sum) TQP_CUDA(cudaMemsetAsync(d_sum, 0, sizeof(int64_t), stream));
        return TQP_OK;
    }
    void* scratch = arena_alloc(ctx, lay.bytes);
    if (!scratch) return arena_oom(ctx, lay.bytes);
    // variant 1: the direct form (every predicate column read with plain vector loads)
    int dgrid = 0;
    if (tuned_variant(ctx) == 1 && A.ncond > 0 && A.ncond <= kFdConds) {
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_filter_direct, kFdThreads, 0) != cudaSuccess || occ < 1)
            occ = 1;
        const long long steps = ((t->num_rows + 3) / 4 + kWarp - 1) / kWarp;
        const long long want = (steps + kFdThreads / kWarp - 1) / (kFdThreads / kWarp);
        dgrid = static_cast<int>(std::max<long long>(1, std::min<long long>(want, static_cast<long long>(occ) * ctx->num_sms)));
    }
    return launch_filter_with(A, grid, smem, lay, scratch, ctx->d_err, ctx->wait_cap, d_row_ids, capacity, d_count,
                              d_sum, stream, dgrid);
}

}  // namespace tqp

using namespace tqp;

extern "C" tqp_status tqp_filter(tqp_ctx* ctx, const tqp_table* t, const tqp_pred* preds, int32_t npreds,
                                 const tqp_expr* sum_expr, int64_t* d_sum, int32_t* d_row_ids, int64_t capacity,
                                 int64_t* d_count, void* stream) {
    clear_error();
    TQP_TRY(check_ctx(ctx));
    TQP_TRY(check_table(t, "tqp_filter"));
    if (!d_count) return fail(TQP_ERR_INVALID_ARG, "d_count is NULL");
    if ((sum_expr == nullptr) != (d_sum == nullptr))
        return fail(TQP_ERR_INVALID_ARG, "sum_expr and d_sum must both be set or both be NULL");
    if (d_row_ids && capacity < 0) return fail(TQP_ERR_INVALID_ARG, "capacity < 0");
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(TQP_ERR_CUDA, "cannot select device %d", ctx->device);
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::vector<int> cols;
    for (int i = 0; i < npreds && i < TQP_MAX_PREDS && preds; ++i) cols.push_back(preds[i].col);
    if (npreds == 0) expr_col_ids(sum_expr, cols);
    char key[96];
    snprintf(key, sizeof(key), "filter r%d b%d i%d s%d", rows_class(t->num_rows), row_bytes(t, cols),
             d_row_ids ? 1 : 0, sum_expr ? 1 : 0);
    auto run = [&]() {
        arena_reset(ctx);
        return launch_filter(ctx, t, preds, npreds, sum_expr, d_sum, d_row_ids, capacity, d_count, st, nullptr);
    };
    return tuned(ctx, key, st, npreds > 0 ? (kTuneVariant | kTuneV1Shapeless) : 0, run);
}

// ---- allocation-free variant (tqp_filter_noalloc) ------------------------------
// For callers that may not allocate device memory.  Its scratch is the
// file-scope array below (every device that loads the library holds it until
// exit): 256 bytes for the device error word, then the filter's own scratch
// layout (ticket, partial sums, block totals, selection mask) for at most
// TQP_NOALLOC_MAX_ROWS rows.  In host code `g_noalloc_scratch` names a host
// stand-in, not device memory, so its device address is looked up once per
// device (with that device current) and passed to the kernels.

namespace tqp {
constexpr size_t kNoallocErrBytes = 256;
constexpr size_t kNoallocScratchBytes = TQP_NOALLOC_SCRATCH_BYTES - kNoallocErrBytes;
}  // namespace tqp

static __device__ __align__(256) unsigned char g_noalloc_scratch[TQP_NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_noalloc_mu;
unsigned char* g_noalloc_addr[tqp::kMaxDevices] = {};

__global__ void k_noalloc_status(const int* err, int32_t* d_status) { *d_status = *err; }

// Device address of the scratch array on `device` (the caller made it current).
tqp_status noalloc_scratch(int device, unsigned char** out) {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_noalloc_addr[device] = static_cast<unsigned char*>(p);
    }
    *out = g_noalloc_addr[device];
    return TQP_OK;
}
}  // namespace

extern "C" tqp_status tqp_filter_noalloc(int device, const tqp_table* t, const tqp_pred* preds, int32_t npreds,
                                         const tqp_expr* sum_expr, int64_t* d_sum, int32_t* d_row_ids,
                                         int64_t capacity, int64_t* d_count, int32_t* d_status, void* stream) {
    clear_error();
    TQP_TRY(check_table(t, "tqp_filter_noalloc"));
    if (!d_count) return fail(TQP_ERR_INVALID_ARG, "d_count is NULL");
    if ((sum_expr == nullptr) != (d_sum == nullptr))
        return fail(TQP_ERR_INVALID_ARG, "sum_expr and d_sum must both be set or both be NULL");
    if (d_row_ids && capacity < 0) return fail(TQP_ERR_INVALID_ARG, "capacity < 0");
    if (t->num_rows > TQP_NOALLOC_MAX_ROWS)
        return fail(TQP_ERR_INVALID_ARG, "tqp_filter_noalloc handles at most %lld rows (got %lld); use tqp_filter",
                    (long long)TQP_NOALLOC_MAX_ROWS, (long long)t->num_rows);
    int ndev = 0;
    TQP_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev || device >= kMaxDevices)
        return fail(TQP_ERR_INVALID_ARG, "device %d out of range", device);
    DeviceGuard g(device);
    if (!g.ok) return fail(TQP_ERR_CUDA, "cannot select device %d", device);
    unsigned char* base = nullptr;
    TQP_TRY(noalloc_scratch(device, &base));

    // a context-shaped description of the device; nothing here is allocated
    tqp_ctx dev_info{};
    dev_info.device = device;
    TQP_CUDA(cudaDeviceGetAttribute(&dev_info.num_sms, cudaDevAttrMultiProcessorCount, device));
    TQP_CUDA(cudaDeviceGetAttribute(&dev_info.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
    dev_info.wait_cap = kDefaultWaitCap;

    FilterArgs A;
    size_t smem = 0;
    int grid = 0;
    FilterScratch lay;
    TQP_TRY(plan_filter(&dev_info, t, preds, npreds, sum_expr, d_row_ids != nullptr, nullptr, &A, &smem, &grid,
                        &lay));
    if (lay.bytes > kNoallocScratchBytes)
        return fail(TQP_ERR_INVALID_ARG, "tqp_filter_noalloc needs %zu scratch bytes, holds %zu", lay.bytes,
                    kNoallocScratchBytes);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int* err = reinterpret_cast<int*>(base);
    TQP_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));  // the array keeps the previous call's contents
    if (t->num_rows == 0) {
        TQP_CUDA(cudaMemsetAsync(d_count, 0, sizeof(int64_t), st));
        if (d_sum) TQP_CUDA(cudaMemsetAsync(d_sum, 0, sizeof(int64_t), st));
    } else {
        TQP_TRY(launch_filter_with(A, grid, smem, lay, base + kNoallocErrBytes, err, kDefaultWaitCap, d_row_ids,
                                   capacity, d_count, d_sum, st));
    }
    if (d_status) {
        k_noalloc_status<<<1, 1, 0, st>>>(err, d_status);
        TQP_CUDA(cudaGetLastError());
    }
    return TQP_OK;
}
