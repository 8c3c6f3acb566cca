// tqp_filter: predicate evaluation + stream compaction + fused projection-sum.
//
// Paper Section 3.1 (Listing 1: comparison mask then masked_select; the
// selection-vector variant uses nonzero + index_select) and Section 5.1
// (expressions).  One kernel does all of it:
//   * pass 1, per tile: the producer warp stages the predicate columns in
//     shared memory with bulk asynchronous copies; consumer warps evaluate the
//     conjunction lane-per-row, take one warp ballot per 32 rows, store the
//     ballot words (a 1-bit-per-row selection mask, 1/128 of a 16-byte row in
//     size) and count with popc; the sum expression is evaluated for passing
//     rows only (columns that are not staged are read lazily);
//   * once per chunk: a decoupled look-back over chunk counts gives the
//     chunk's output offset;
//   * pass 2, per chunk: the chunk's mask words (still in L2) are expanded into
//     ascending row ids with warp-cooperative, coalesced stores.
// Count and sum are reduced per warp and added once per warp to scratch; the
// last warp to finish publishes them, so no host synchronisation is needed.
#include "host.h"

namespace tqp {

struct FilterArgs {
    ScanGeom G;
    EngineCtl ctl;
    int32_t ncond;
    int32_t has_sum;
    Cond cond[TQP_MAX_PREDS];
    DExpr sum;
    int32_t* row_ids;            // nullable: count/sum only
    int64_t capacity;
    int64_t* d_count;
    int64_t* d_sum;              // nullable
    uint32_t* mask;              // one ballot word per 32 rows (with row_ids)
    unsigned long long* status;  // per-chunk look-back words (zeroed)
    unsigned long long* acc;     // [0] sum, [1] count, [2] finished warps (zeroed)
};

// Scratch layout (bytes): ticket + acc[3], chunk status words, then the mask.
struct FilterScratch {
    size_t status_off, mask_off, bytes;
};

static FilterScratch filter_scratch_layout(const ScanGeom& G, long long nchunks, bool ids) {
    FilterScratch s;
    s.status_off = 4 * sizeof(unsigned long long);
    s.mask_off = (s.status_off + (ids ? nchunks : 0) * sizeof(unsigned long long) + 255) / 256 * 256;
    s.bytes = s.mask_off + (ids ? static_cast<size_t>(G.ntiles) * (G.T / 32) * sizeof(uint32_t) : 0);
    return s;
}

struct FilterBody {
    static constexpr int kSmemBytes = 128;  // warp totals [2][warps] + chunk offset

    const FilterArgs& A;
    uint32_t* wtot;              // [2][kConsumerWarps]
    unsigned long long* excl_sm;
    long long my_sum = 0;
    unsigned long long my_cnt = 0;     // lane 0: rows passed by this warp (all chunks)
    unsigned long long chunk_cnt = 0;  // lane 0: rows passed by this warp in the current chunk

    __device__ FilterBody(const FilterArgs& a, unsigned char* sm) : A(a) {
        wtot = reinterpret_cast<uint32_t*>(sm);
        excl_sm = reinterpret_cast<unsigned long long*>(sm + 2 * kConsumerWarps * 4);
    }

    __device__ void pass1(const ScanGeom& G, const TileView& v, int cw, int lane) {
        const int rw = G.T / kConsumerWarps;
        const int chunks = rw / kWarp;
        uint32_t cnt = 0;
        for (int c = 0; c < chunks; c += kUnroll) {
            const int rbase = cw * rw + c * kWarp;
            if (rbase >= v.rows) break;  // words wholly past the table end are never read
            bool ok[kUnroll];
            eval_conds(G, v, A.cond, A.ncond, rbase + lane, ok);
            uint32_t b[kUnroll];
#pragma unroll
            for (int j = 0; j < kUnroll; ++j) {
                b[j] = __ballot_sync(0xffffffffu, ok[j]);
                cnt += __popc(b[j]);
                if (A.has_sum && ok[j]) my_sum += eval_expr(G, v, A.sum, rbase + kWarp * j + lane);
            }
            if (A.row_ids && lane == 0)
                *reinterpret_cast<uint4*>(A.mask + (v.row0 + rbase) / kWarp) = make_uint4(b[0], b[1], b[2], b[3]);
        }
        if (lane == 0) chunk_cnt += cnt;
    }

    __device__ void chunk_end(const ScanGeom& G, long long chunk, long long t0, long long t1, int cw, int lane) {
        if (lane == 0) my_cnt += chunk_cnt;
        if (!A.row_ids) {
            chunk_cnt = 0;
            return;
        }
        if (lane == 0) wtot[cw] = static_cast<uint32_t>(chunk_cnt);
        chunk_cnt = 0;
        named_sync(kBarConsumers, kConsumers);
        if (cw == 0) {
            unsigned long long c = lane < kConsumerWarps ? wtot[lane] : 0ULL;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
            const unsigned long long ex = lookback(A.status, chunk, c, lane, A.ctl.err, A.ctl.wait_cap);
            if (lane == 0) *excl_sm = ex;
        }
        named_sync(kBarConsumers, kConsumers);
        unsigned long long running = *excl_sm;

        // expand this chunk's mask words into row ids, 256 words per round
        const long long w_begin = t0 * (G.T / kWarp);
        const long long row_end = (t1 * G.T < G.n) ? t1 * G.T : G.n;
        const long long w_end = (row_end + kWarp - 1) / kWarp;
        const uint32_t lt = lanemask_lt();
        int par = 0;
        for (long long base = w_begin; base < w_end; base += kConsumers) {
            const long long wi = base + cw * kWarp + lane;
            const uint32_t word = wi < w_end ? A.mask[wi] : 0u;
            const uint32_t c = __popc(word);
            uint32_t incl = c;
#pragma unroll
            for (int o = 1; o < kWarp; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane == kWarp - 1) wtot[par * kConsumerWarps + cw] = incl;
            named_sync(kBarConsumers, kConsumers);
            unsigned long long before = 0, round_total = 0;
#pragma unroll
            for (int w = 0; w < kConsumerWarps; ++w) {
                const uint32_t x = wtot[par * kConsumerWarps + w];
                before += (w < cw) ? x : 0u;
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
                    if (pos < static_cast<unsigned long long>(A.capacity))
                        A.row_ids[pos] = static_cast<int32_t>((base + cw * kWarp + j) * kWarp + lane);
                }
            }
            running += round_total;
            par ^= 1;
        }
    }

    __device__ void finish(const ScanGeom&, int cw, int lane) {
        long long s = my_sum;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            if (s) atomicAdd(&A.acc[0], static_cast<unsigned long long>(s));
            if (my_cnt) atomicAdd(&A.acc[1], my_cnt);
            __threadfence();
            const unsigned long long done = atomicAdd(&A.acc[2], 1ULL);
            if (done == static_cast<unsigned long long>(gridDim.x) * kConsumerWarps - 1) {
                __threadfence();
                const unsigned long long tot_sum = atomicAdd(&A.acc[0], 0ULL);
                const unsigned long long tot_cnt = atomicAdd(&A.acc[1], 0ULL);
                *A.d_count = static_cast<int64_t>(tot_cnt);
                if (A.d_sum) *A.d_sum = static_cast<int64_t>(tot_sum);
                if (A.row_ids && static_cast<long long>(tot_cnt) > A.capacity)
                    latch_error(A.ctl.err, TQP_ERR_CAPACITY);
            }
        }
    }
};

__global__ void __launch_bounds__(kEngineThreads, 2) k_filter(const __grid_constant__ FilterArgs A) {
    extern __shared__ __align__(128) unsigned char smem[];
    FilterBody body(A, smem + kHeaderBytes);
    run_engine(A.G, A.ctl, body, smem);
}

// Lower a filter call into kernel arguments; *scratch_bytes receives the
// scratch it needs and *grid / *smem the launch shape.
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
    int bpr = 0;
    for (int c : u) bpr += t->cols[c].type == TQP_I64 ? 8 : (t->cols[c].type == TQP_I32 ? 4 : 1);
    const tqp_tuning tu = force ? *force : default_tuning(ctx, bpr, FilterBody::kSmemBytes);
    TQP_TRY(make_geom(ctx, t, staged, tu, FilterBody::kSmemBytes, &A->G, smem));
    static bool attr_done[kMaxDevices] = {};
    TQP_TRY(allow_smem(ctx, reinterpret_cast<const void*>(k_filter), attr_done));
    const int g = engine_grid(ctx, reinterpret_cast<const void*>(k_filter), *smem, A->G.ntiles, tu.ctas_per_sm);
    A->ctl.chunk_tiles = (A->G.ntiles + g - 1) / g;
    A->ctl.nchunks = (A->G.ntiles + A->ctl.chunk_tiles - 1) / A->ctl.chunk_tiles;
    *grid = static_cast<int>(A->ctl.nchunks);
    *lay = filter_scratch_layout(A->G, A->ctl.nchunks, ids);
    return TQP_OK;
}

// Launch with caller-provided scratch of at least lay.bytes (zeroed here).
static tqp_status launch_filter_with(FilterArgs& A, int grid, size_t smem, const FilterScratch& lay,
                                     void* scratch, int* d_err, long long wait_cap, int32_t* d_row_ids,
                                     int64_t capacity, int64_t* d_count, int64_t* d_sum, cudaStream_t stream) {
    unsigned char* sc = static_cast<unsigned char*>(scratch);
    TQP_CUDA(cudaMemsetAsync(sc, 0, lay.mask_off, stream));
    A.ctl.ticket = reinterpret_cast<unsigned long long*>(sc);
    A.ctl.err = d_err;
    A.ctl.wait_cap = wait_cap;
    A.acc = reinterpret_cast<unsigned long long*>(sc) + 1;
    A.status = reinterpret_cast<unsigned long long*>(sc + lay.status_off);
    A.mask = reinterpret_cast<uint32_t*>(sc + lay.mask_off);
    A.row_ids = d_row_ids;
    A.capacity = capacity;
    A.d_count = d_count;
    A.d_sum = d_sum;
    k_filter<<<grid, kEngineThreads, smem, stream>>>(A);
    TQP_CUDA(cudaGetLastError());
    return TQP_OK;
}

tqp_status launch_filter(tqp_ctx* ctx, const tqp_table* t, const tqp_pred* preds, int32_t npreds,
                         const tqp_expr* sum_expr, int64_t* d_sum, int32_t* d_row_ids, int64_t capacity,
                         int64_t* d_count, cudaStream_t stream, const tqp_tuning* force) {
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
    return launch_filter_with(A, grid, smem, lay, scratch, ctx->d_err, ctx->wait_cap, d_row_ids, capacity, d_count,
                              d_sum, stream);
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
    arena_reset(ctx);
    return launch_filter(ctx, t, preds, npreds, sum_expr, d_sum, d_row_ids, capacity, d_count,
                         static_cast<cudaStream_t>(stream), nullptr);
}
