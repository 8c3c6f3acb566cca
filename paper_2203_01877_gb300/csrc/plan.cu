// tqp_run_plan: a fixed operator plan (paper Section 4.2.5: the executor runs
// the plan's operators in topological order and wires outputs to inputs).
//
//   scan(fact) -> filter -> [hash join fact.fk = dim.key] -> [SUM] ->
//   [GROUP BY: aggregates] -> [top-k]
//
// Everything stays on the device and stream-ordered; no step waits for the
// host.  Without a join the plan is the filter kernel and/or the group-by
// scan.  With a join, one fused kernel filters the fact rows, probes the
// dimension table and aggregates every joined row straight into the group
// table: the join result is never materialised.  Group keys are dimension
// columns, so each dimension row's group slot is resolved once, before the
// probe (k_dim_groups), and a probe costs one table lookup plus atomics.
#include "host.h"
#include "group.cuh"
#include "join.cuh"

namespace tqp {

tqp_status launch_filter(tqp_ctx* ctx, const tqp_table* t, const tqp_pred* preds, int32_t npreds,
                         const tqp_expr* sum_expr, int64_t* d_sum, int32_t* d_row_ids, int64_t capacity,
                         int64_t* d_count, cudaStream_t stream, const tqp_tuning* force);
tqp_status launch_groupby(tqp_ctx* ctx, const tqp_table* t, const tqp_pred* preds, int32_t npreds,
                          const int32_t* group_cols, int32_t ngc, const tqp_agg* aggs, int32_t naggs,
                          int64_t* d_keys, int64_t* d_ivals, double* d_fvals, int64_t capacity_groups,
                          int64_t* d_num_groups, cudaStream_t stream, long long max_groups, int topk, int topk_agg,
                          int64_t* d_total_groups);
tqp_status ht_build(tqp_ctx* ctx, const tqp_table* build, int32_t key_col, JoinHT* H, cudaStream_t stream);

struct DimCols {
    const unsigned char* ptr[TQP_MAX_COLS];
    int32_t type[TQP_MAX_COLS];
};

// Group slot of every dimension row (its packed group key, inserted once).
__global__ void k_dim_groups(const __grid_constant__ GroupSpec S, const __grid_constant__ DimCols D, long long n,
                             uint32_t* dgs, int* err) {
    for (long long d = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; d < n;
         d += static_cast<long long>(gridDim.x) * blockDim.x) {
        uint64_t k = 0;
        for (int i = 0; i < S.ngc; ++i) {
            const int b = S.key_bits[i];
            const int c = S.key_col[i];
            const uint64_t e = enc_key(ldg_typed(D.ptr[c], D.type[c], d), b);
            k = (b == 64) ? e : ((k << b) | e);
        }
        const long long s = gtab_slot(S, k, err);
        dgs[d] = s < 0 ? 0u : static_cast<uint32_t>(s);
    }
}

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
    const uint32_t* dgs;       // dim row -> group slot; nullptr: no aggregation
    GroupSpec S;
    unsigned long long* acc;   // [0] joined, [1] sum, [2] passing fact rows, [3] finished warps (zeroed)
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

    __device__ __forceinline__ void row(const ScanGeom& G, const TileView& v, int r) {
        ++passed;
        const uint64_t key = static_cast<uint64_t>(col_val(G, v, A.fk_col, r));
        const long long s = ht_find(A.H, key);
        if (s < 0) return;
        const uint4 sl = A.H.slots[s];
        const uint32_t cnt = sl.w;
        joined += cnt;
        if (A.has_sum) sum += eval_expr(G, v, A.sum, r) * static_cast<long long>(cnt);
        if (!A.dgs) return;
        const GroupSpec& S = A.S;
        for (uint32_t k = 0; k < cnt; ++k) {
            const uint32_t d = A.H.bidx[sl.z + k];
            unsigned long long* a = S.acc + static_cast<long long>(__ldg(&A.dgs[d])) * S.nacc;
            atomicAdd(&a[0], 1ULL);
            for (int i = 1; i < S.nacc; ++i)
                atomicAdd(&a[i], static_cast<unsigned long long>(eval_expr(G, v, S.acc_expr[i - 1], r)));
        }
    }

    __device__ void pass1(const ScanGeom& G, const TileView& v, int cw, int lane) {
        const int rw = G.T / kConsumerWarps;
        for (int r = 0; r < rw; r += kUnroll * kWarp) {
            const int rbase = cw * rw + r;
            if (rbase >= v.rows) break;
            const uint32_t ok = eval_rows<kUnroll>(G, v, A.cf, A.cond, A.ncond, A.fast != 0, rbase + lane);
#pragma unroll
            for (int j = 0; j < kUnroll; ++j)
                if ((ok >> j) & 1u) row(G, v, rbase + kWarp * j + lane);
        }
    }

    __device__ void chunk_end(const ScanGeom&, long long, long long, long long, int, int) {}

    __device__ void finish(const ScanGeom&, int cw, int lane) {
        unsigned long long j = joined, p = passed;
        long long s = sum;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            j += __shfl_xor_sync(0xffffffffu, j, o);
            p += __shfl_xor_sync(0xffffffffu, p, o);
            s += __shfl_xor_sync(0xffffffffu, s, o);
        }
        if (lane == 0) {
            if (j) atomicAdd(&A.acc[0], j);
            if (s) atomicAdd(&A.acc[1], static_cast<unsigned long long>(s));
            if (p) atomicAdd(&A.acc[2], p);
            __threadfence();
            const unsigned long long done = atomicAdd(&A.acc[3], 1ULL);
            if (done == static_cast<unsigned long long>(gridDim.x) * kConsumerWarps - 1) {
                __threadfence();
                if (A.d_num_joined) *A.d_num_joined = static_cast<int64_t>(atomicAdd(&A.acc[0], 0ULL));
                if (A.d_sum) *A.d_sum = static_cast<int64_t>(atomicAdd(&A.acc[1], 0ULL));
                if (A.d_num_rows) *A.d_num_rows = static_cast<int64_t>(atomicAdd(&A.acc[2], 0ULL));
            }
        }
    }
};

__global__ void __launch_bounds__(kEngineThreads, 2) k_plan_join(const __grid_constant__ PlanJoinArgs A) {
    extern __shared__ __align__(128) unsigned char smem[];
    PlanJoinBody body(A, smem + kHeaderBytes);
    run_engine(A.G, A.ctl, body, smem);
}

static bool expr_uses_only(const tqp_expr& e, int lo, int hi) {
    for (int i = 0; i < e.n && i < TQP_MAX_EXPR; ++i)
        if (e.op[i] == TQP_X_COL && (e.v[i] < lo || e.v[i] >= hi)) return false;
    return true;
}

static tqp_status run_join_plan(tqp_ctx* ctx, const tqp_plan* p, const tqp_result* r, cudaStream_t stream) {
    const tqp_table* F = p->fact;
    const tqp_table* D = p->dim;
    TQP_TRY(check_table(D, "plan.dim"));
    const int nf = F->num_cols, nd = D->num_cols;
    if (p->fact_fk < 0 || p->fact_fk >= nf) return fail(TQP_ERR_INVALID_ARG, "fact_fk out of range");
    if (p->dim_key < 0 || p->dim_key >= nd) return fail(TQP_ERR_INVALID_ARG, "dim_key out of range");
    if (nf + nd > 2 * TQP_MAX_COLS) return fail(TQP_ERR_INVALID_ARG, "too many columns");
    for (int i = 0; i < p->ngc; ++i)
        if (p->group_cols[i] < nf || p->group_cols[i] >= nf + nd)
            return fail(TQP_ERR_UNSUPPORTED, "with a join, group columns must be dimension columns");
    for (int a = 0; a < p->naggs; ++a)
        if (p->aggs[a].fn != TQP_COUNT && !expr_uses_only(p->aggs[a].expr, 0, nf))
            return fail(TQP_ERR_UNSUPPORTED, "with a join, aggregate expressions must use fact columns only");
    if (p->has_sum && !expr_uses_only(p->sum_expr, 0, nf))
        return fail(TQP_ERR_UNSUPPORTED, "with a join, the sum expression must use fact columns only");

    // passing fact row ids (before the join) come from the filter kernel
    if (p->emit_row_ids && r->d_row_ids) {
        if (!r->d_num_rows) return fail(TQP_ERR_INVALID_ARG, "emit_row_ids needs d_num_rows");
        TQP_TRY(launch_filter(ctx, F, p->preds, p->npreds, nullptr, nullptr, r->d_row_ids, r->capacity_rows,
                              r->d_num_rows, stream, nullptr));
    }

    JoinHT H;
    TQP_TRY(ht_build(ctx, D, p->dim_key, &H, stream));

    PlanJoinArgs A;
    memset(&A, 0, sizeof(A));
    int ncond = 0;
    TQP_TRY(lower_preds(F, p->preds, p->npreds, A.cond, &ncond));
    A.ncond = ncond;
    A.fk_col = p->fact_fk;
    A.H = H;
    if (p->has_sum) {
        TQP_TRY(lower_expr(&p->sum_expr, nf, &A.sum));
        A.has_sum = 1;
    }
    const bool grouped = p->ngc > 0 || p->naggs > 0;
    if (grouped) {
        int32_t kc[TQP_MAX_GROUP_COLS], kt[TQP_MAX_GROUP_COLS];
        for (int i = 0; i < p->ngc; ++i) {
            kc[i] = p->group_cols[i] - nf;
            kt[i] = D->cols[kc[i]].type;
        }
        TQP_TRY(lower_group(kc, kt, p->ngc, p->aggs, p->naggs, nf, &A.S));
        // AVG needs d_fvals
        for (int a = 0; a < p->naggs; ++a)
            if (p->aggs[a].fn == TQP_AVG && !r->d_fvals) return fail(TQP_ERR_INVALID_ARG, "AVG needs d_fvals");
        if (!r->d_num_groups) return fail(TQP_ERR_INVALID_ARG, "d_num_groups is NULL");
        const long long maxg = p->max_groups > 0 ? p->max_groups : (p->ngc == 0 ? 1 : std::max<long long>(1, D->num_rows));
        const long long cap = group_table_cap(maxg);
        void* tab = arena_alloc(ctx, group_table_bytes(cap, A.S.nacc));
        uint32_t* dgs = static_cast<uint32_t*>(arena_alloc(ctx, static_cast<size_t>(std::max<long long>(1, D->num_rows)) * 4));
        if (!tab || !dgs) return arena_oom(ctx, group_table_bytes(cap, A.S.nacc));
        TQP_TRY(group_table_init(&A.S, tab, cap, maxg, stream));
        DimCols DC;
        memset(&DC, 0, sizeof(DC));
        for (int c = 0; c < nd; ++c) {
            DC.ptr[c] = static_cast<const unsigned char*>(D->cols[c].data);
            DC.type[c] = D->cols[c].type;
        }
        if (D->num_rows > 0) {
            const int threads = 256;
            const int blocks = static_cast<int>(std::min<long long>((D->num_rows + threads - 1) / threads, ctx->num_sms * 16LL));
            k_dim_groups<<<blocks, threads, 0, stream>>>(A.S, DC, D->num_rows, dgs, ctx->d_err);
            TQP_CUDA(cudaGetLastError());
        }
        A.dgs = dgs;
    }

    // stage the conditions, the foreign key and every aggregated fact column
    std::vector<int> staged;
    for (int i = 0; i < ncond; ++i) staged.push_back(A.cond[i].col);
    staged.push_back(p->fact_fk);
    if (A.has_sum) expr_cols(A.sum, staged);
    for (int a = 1; a < A.S.nacc; ++a) expr_cols(A.S.acc_expr[a - 1], staged);
    std::sort(staged.begin(), staged.end());
    staged.erase(std::unique(staged.begin(), staged.end()), staged.end());
    if (static_cast<int>(staged.size()) > kMaxStaged) staged.resize(kMaxStaged);
    int bpr = 0;
    for (int c : staged) bpr += F->cols[c].type == TQP_I64 ? 8 : (F->cols[c].type == TQP_I32 ? 4 : 1);
    const tqp_tuning tu = default_tuning(ctx, bpr, PlanJoinBody::kSmemBytes);
    size_t smem = 0;
    TQP_TRY(make_geom(ctx, F, staged, tu, PlanJoinBody::kSmemBytes, &A.G, &smem));
    lower_fast(A.cond, A.ncond, A.G, A.cf, &A.fast);

    unsigned long long* sc = static_cast<unsigned long long*>(arena_alloc(ctx, 8 * 8));
    if (!sc) return arena_oom(ctx, 64);
    TQP_CUDA(cudaMemsetAsync(sc, 0, 8 * 8, stream));
    A.acc = sc + 1;
    A.d_num_joined = r->d_num_joined;
    A.d_sum = p->has_sum ? r->d_sum : nullptr;
    A.d_num_rows = (p->emit_row_ids && r->d_row_ids) ? nullptr : r->d_num_rows;
    if (F->num_rows > 0) {
        static bool attr_done[kMaxDevices] = {};
        TQP_TRY(allow_smem(ctx, reinterpret_cast<const void*>(k_plan_join), attr_done));
        const int g = engine_grid(ctx, reinterpret_cast<const void*>(k_plan_join), smem, A.G.ntiles, tu.ctas_per_sm);
        A.ctl.chunk_tiles = (A.G.ntiles + g - 1) / g;
        A.ctl.nchunks = (A.G.ntiles + A.ctl.chunk_tiles - 1) / A.ctl.chunk_tiles;
        A.ctl.ticket = sc;
        A.ctl.err = ctx->d_err;
        A.ctl.wait_cap = ctx->wait_cap;
        k_plan_join<<<static_cast<int>(A.ctl.nchunks), kEngineThreads, smem, stream>>>(A);
        TQP_CUDA(cudaGetLastError());
    } else {
        if (A.d_num_joined) TQP_CUDA(cudaMemsetAsync(A.d_num_joined, 0, 8, stream));
        if (A.d_sum) TQP_CUDA(cudaMemsetAsync(A.d_sum, 0, 8, stream));
        if (A.d_num_rows) TQP_CUDA(cudaMemsetAsync(A.d_num_rows, 0, 8, stream));
    }
    if (!grouped) return TQP_OK;
    GroupOut O{r->d_keys, r->d_ivals, r->d_fvals, r->capacity_groups, r->d_num_groups, ctx->d_err};
    if (p->topk > 0) return group_topk(ctx, A.S, O, p->topk, p->topk_agg, r->d_total_groups, stream);
    TQP_TRY(group_finalize(ctx, A.S, O, stream));
    if (r->d_total_groups)
        TQP_CUDA(cudaMemcpyAsync(r->d_total_groups, r->d_num_groups, 8, cudaMemcpyDeviceToDevice, stream));
    return TQP_OK;
}

static tqp_status run_scan_plan(tqp_ctx* ctx, const tqp_plan* p, const tqp_result* r, cudaStream_t stream) {
    const tqp_table* F = p->fact;
    const bool grouped = p->ngc > 0 || p->naggs > 0;
    int64_t* d_cnt = r->d_num_rows ? r->d_num_rows : r->d_num_joined;
    const bool ids = p->emit_row_ids && r->d_row_ids;
    if (ids && !d_cnt) return fail(TQP_ERR_INVALID_ARG, "emit_row_ids needs d_num_rows");
    if (ids || (p->has_sum && r->d_sum) || d_cnt) {
        if (!d_cnt) {
            d_cnt = static_cast<int64_t*>(arena_alloc(ctx, 256));
            if (!d_cnt) return arena_oom(ctx, 256);
        }
        TQP_TRY(launch_filter(ctx, F, p->preds, p->npreds, (p->has_sum && r->d_sum) ? &p->sum_expr : nullptr,
                              (p->has_sum && r->d_sum) ? r->d_sum : nullptr, ids ? r->d_row_ids : nullptr,
                              ids ? r->capacity_rows : 0, d_cnt, stream, nullptr));
        if (r->d_num_rows && r->d_num_joined)
            TQP_CUDA(cudaMemcpyAsync(r->d_num_joined, r->d_num_rows, 8, cudaMemcpyDeviceToDevice, stream));
    }
    if (!grouped) return TQP_OK;
    if (!r->d_num_groups) return fail(TQP_ERR_INVALID_ARG, "d_num_groups is NULL");
    for (int i = 0; i < p->ngc; ++i)
        if (p->group_cols[i] < 0 || p->group_cols[i] >= F->num_cols)
            return fail(TQP_ERR_INVALID_ARG, "group column %d out of range", p->group_cols[i]);
    const long long cap_groups = r->capacity_groups;
    const long long maxg = p->max_groups > 0 ? p->max_groups : std::max<long long>(1, cap_groups);
    TQP_TRY(launch_groupby(ctx, F, p->preds, p->npreds, p->group_cols, p->ngc, p->aggs, p->naggs, r->d_keys,
                           r->d_ivals, r->d_fvals, cap_groups, r->d_num_groups, stream, maxg, p->topk, p->topk_agg,
                           r->d_total_groups));
    if (p->topk == 0 && r->d_total_groups)
        TQP_CUDA(cudaMemcpyAsync(r->d_total_groups, r->d_num_groups, 8, cudaMemcpyDeviceToDevice, stream));
    return TQP_OK;
}

tqp_status run_plan_one(tqp_ctx* ctx, const tqp_plan* p, const tqp_result* r, cudaStream_t stream) {
    if (!p || !r) return fail(TQP_ERR_INVALID_ARG, "plan or result is NULL");
    TQP_TRY(check_table(p->fact, "plan.fact"));
    if (p->ngc < 0 || p->ngc > TQP_MAX_GROUP_COLS) return fail(TQP_ERR_INVALID_ARG, "ngc out of range");
    if (p->naggs < 0 || p->naggs > TQP_MAX_AGGS) return fail(TQP_ERR_INVALID_ARG, "naggs out of range");
    if (p->topk < 0) return fail(TQP_ERR_INVALID_ARG, "topk < 0");
    if (p->ngc + p->naggs > 0 && r->capacity_groups < 1) return fail(TQP_ERR_INVALID_ARG, "capacity_groups < 1");
    arena_reset(ctx);
    if (p->dim) return run_join_plan(ctx, p, r, stream);
    return run_scan_plan(ctx, p, r, stream);
}

}  // namespace tqp

using namespace tqp;

extern "C" tqp_status tqp_run_plan(tqp_ctx* ctx, const tqp_plan* plan, const tqp_result* res, void* stream) {
    clear_error();
    TQP_TRY(check_ctx(ctx));
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(TQP_ERR_CUDA, "cannot select device %d", ctx->device);
    return run_plan_one(ctx, plan, res, static_cast<cudaStream_t>(stream));
}

extern "C" tqp_status tqp_run_plans(tqp_ctx* ctx, const tqp_plan* plans, const tqp_result* res, int32_t n,
                                    void* stream) {
    clear_error();
    TQP_TRY(check_ctx(ctx));
    if (n < 0 || (n > 0 && (!plans || !res))) return fail(TQP_ERR_INVALID_ARG, "bad plan array");
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(TQP_ERR_CUDA, "cannot select device %d", ctx->device);
    for (int32_t i = 0; i < n; ++i) TQP_TRY(run_plan_one(ctx, &plans[i], &res[i], static_cast<cudaStream_t>(stream)));
    return TQP_OK;
}
