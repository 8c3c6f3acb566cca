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
#include <cstdio>
#include <new>

#include "host.h"
#include "group.cuh"
#include "join.cuh"
#include "bodies.cuh"
#include "dimgroups.cuh"
#include "dim.cuh"
#include "partjoin.cuh"

namespace tqp {

tqp_status launch_groupby(tqp_ctx* ctx, const tqp_table* t, const tqp_pred* preds, int32_t npreds,
                          const int32_t* group_cols, int32_t ngc, const tqp_agg* aggs, int32_t naggs,
                          int64_t* d_keys, int64_t* d_ivals, double* d_fvals, int64_t capacity_groups,
                          int64_t* d_num_groups, cudaStream_t stream, long long max_groups, int topk, int topk_agg,
                          int64_t* d_total_groups);
tqp_status ht_build_chain(tqp_ctx* ctx, const tqp_table* build, int32_t key_col, JoinHT* H, uint32_t** next,
                          cudaStream_t stream);
tqp_status ht_key_range_launch(const tqp_ctx* ctx, const tqp_table* build, int32_t key_col, long long* meta,
                               cudaStream_t stream);
tqp_status ht_chain_insert_launch(const tqp_ctx* ctx, const tqp_table* build, int32_t key_col, const JoinHT& H,
                                  uint32_t* next, cudaStream_t stream);
tqp_status launch_part_join(tqp_ctx* ctx, const PlanJoinArgs& J, const tqp_table* F, long long maxg,
                            unsigned long long* acc_words, cudaStream_t stream);

// Fact rows from which a grouped join plan takes the radix-partitioned
// aggregation by default (variant 0; variant 1 is the fused probe).  Below,
// the extra kernel and the record traffic do not pay for themselves.
constexpr long long kPartJoinMinRows = 1LL << 20;

// Dense group ids of the dimension rows, in three small passes:
//   claim  each dim row inserts its packed group key into a claim table
//          (open addressing, keys only) and remembers the slot;
//   number every claimed slot gets a dense id 0..G-1; its key is stored and its
//          accumulators are cleared (so nothing of size max_groups is memset);
//   remap  dim row -> dense id.
// The probe then aggregates into a G x nacc array that stays in L2.
__global__ void k_dim_claim(const __grid_constant__ GroupSpec S, const __grid_constant__ DimCols D, long long n,
                            uint32_t* dslot, int* err) {
    for (long long d = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; d < n;
         d += static_cast<long long>(gridDim.x) * blockDim.x)
        dim_claim_row(S, D, d, dslot, err);
}

__global__ void __launch_bounds__(kNumberThreads) k_dense_number(const __grid_constant__ GroupSpec S,
                                                                 uint32_t* slot2dense, unsigned long long* keys_out,
                                                                 unsigned long long* acc_out, long long* d_n,
                                                                 long long per_block) {
    const long long s0 = blockIdx.x * per_block;
    const long long s1 = (s0 + per_block < S.cap + 1) ? s0 + per_block : S.cap + 1;
    dense_number_range(S, slot2dense, keys_out, acc_out, d_n, s0, s1);
}

__global__ void k_ht_direct(JoinHT H, const uint32_t* dgs) {
    for (long long s = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; s <= H.cap;
         s += static_cast<long long>(gridDim.x) * blockDim.x)
        ht_direct_slot(H, dgs, s);
}

__global__ void k_dim_remap(const uint32_t* dslot, const uint32_t* slot2dense, long long n, uint32_t* dgs) {
    for (long long d = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; d < n;
         d += static_cast<long long>(gridDim.x) * blockDim.x)
        dgs[d] = slot2dense[dslot[d]];
}

// Zero the key-first accumulators over a direct-mapped table's key range
// (a hashed table leaves them unused).
__global__ void k_keyfirst_zero(const JoinHT H, unsigned long long* kacc, int nk) {
    long long kmin;
    if (!ht_is_direct(H, &kmin)) return;
    const long long n = (__ldg(&H.meta[1]) - kmin + 1) * nk;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x)
        kacc[i] = 0;
}

__global__ void __launch_bounds__(kFoldThreads) k_keyfirst_fold(const JoinHT H, const unsigned char* dkey, int dkey_type,
                                                                long long nd, const uint32_t* dgs,
                                                                const __grid_constant__ GroupSpec S,
                                                                const unsigned long long* kacc, int nk, int has_sum,
                                                                unsigned long long* acc, int64_t* d_num_joined,
                                                                int64_t* d_sum) {
    keyfirst_fold_block(H, dkey, dkey_type, nd, dgs, S, kacc, nk, has_sum, acc, d_num_joined, d_sum, blockIdx.x,
                        gridDim.x);
}

__global__ void __launch_bounds__(kEngineThreads, PlanJoinBody::kMinBlocks) k_plan_join(const __grid_constant__ PlanJoinArgs P) {
    extern __shared__ __align__(128) unsigned char smem[];
    const PlanJoinArgs& A = stage_args(P, smem + kHeaderBytes);
    PlanJoinBody body(A, smem + kHeaderBytes + args_bytes<PlanJoinArgs>());
    run_engine(A.G, A.ctl, body, smem, args_bytes<PlanJoinArgs>());
}

void lower_join_fast(PlanJoinArgs* A) {
    A->pjfast = 0;
    if (A->S.minmax) return;  // the closed-form fast paths only add: MIN/MAX take the general one
    A->nsum = A->S.nacc > 0 ? A->S.nacc - 1 : 0;
    const ColRef& fk = A->G.col[A->fk_col];
    if (fk.slot < 0) return;
    A->fk_soff = fk.soff;
    A->fk_type = fk.type;
    if (A->has_sum && !lower_prod(A->sum, A->G, &A->psum)) return;
    if (A->dgs) {
        if (A->nsum > PlanJoinBody::kJoinSums) return;
        for (int a = 0; a < A->nsum; ++a)
            if (!lower_prod(A->S.acc_expr[a], A->G, &A->pacc[a])) return;
    }
    A->pjfast = 1;
}

static bool expr_uses_only(const tqp_expr& e, int lo, int hi) {
    for (int i = 0; i < e.n && i < TQP_MAX_EXPR; ++i)
        if (e.op[i] == TQP_X_COL && (e.v[i] < lo || e.v[i] >= hi)) return false;
    return true;
}

tqp_status dense_groups_launch(tqp_ctx* ctx, const tqp_table* D, const GroupSpec& S, long long maxg,
                               const JoinHT* H, uint32_t* dgs, unsigned long long* dkeys, unsigned long long* dacc,
                               unsigned long long* ndistinct, cudaStream_t stream) {
    const long long cap = group_table_cap(maxg);
    const long long nd_rows = std::max<long long>(1, D->num_rows);
    GroupSpec claim = S;
    claim.cap = cap;
    claim.max_groups = maxg;
    claim.ndistinct = ndistinct;
    claim.keys = static_cast<unsigned long long*>(arena_alloc(ctx, static_cast<size_t>(cap + 1) * 8));
    uint32_t* slot2dense = static_cast<uint32_t*>(arena_alloc(ctx, static_cast<size_t>(cap + 1) * 4));
    uint32_t* dslot = static_cast<uint32_t*>(arena_alloc(ctx, static_cast<size_t>(nd_rows) * 4));
    if (!claim.keys || !slot2dense || !dslot) return arena_oom(ctx, static_cast<size_t>(cap) * 12 + nd_rows * 4);
    long long* d_n = reinterpret_cast<long long*>(ndistinct) + 1;
    TQP_CUDA(cudaMemsetAsync(claim.keys, 0xFF, static_cast<size_t>(cap + 1) * 8, stream));
    TQP_CUDA(cudaMemsetAsync(ndistinct, 0, 16, stream));
    if (D->num_rows == 0) return TQP_OK;
    DimCols DC;
    memset(&DC, 0, sizeof(DC));
    for (int c = 0; c < D->num_cols; ++c) {
        DC.ptr[c] = static_cast<const unsigned char*>(D->cols[c].data);
        DC.type[c] = D->cols[c].type;
    }
    const int threads = 256;
    const int blocks = static_cast<int>(std::min<long long>((D->num_rows + threads - 1) / threads, ctx->num_sms * 16LL));
    k_dim_claim<<<blocks, threads, 0, stream>>>(claim, DC, D->num_rows, dslot, ctx->d_err);
    const long long nb = std::max<long long>(1, std::min<long long>((cap + 1 + 2047) / 2048, ctx->num_sms * 4LL));
    const long long per = (cap + 1 + nb - 1) / nb;
    k_dense_number<<<static_cast<int>(nb), kNumberThreads, 0, stream>>>(claim, slot2dense, dkeys, dacc, d_n, per);
    k_dim_remap<<<blocks, threads, 0, stream>>>(dslot, slot2dense, D->num_rows, dgs);
    if (H) {
        const int hblocks = static_cast<int>(std::min<long long>((H->cap + threads) / threads, ctx->num_sms * 16LL));
        k_ht_direct<<<hblocks, threads, 0, stream>>>(*H, dgs);
    }
    TQP_CUDA(cudaGetLastError());
    return TQP_OK;
}

tqp_status check_prepared(const tqp_ctx* ctx, const tqp_plan* p) {
    const tqp_dim* pd = p->prepared;
    if (pd->ctx->device != ctx->device) return fail(TQP_ERR_INVALID_ARG, "plan.prepared lives on another device");
    if (!p->dim || p->dim->num_rows != pd->nrows || p->dim_key != pd->key_col ||
        p->dim->cols[p->dim_key].data != pd->key_data)
        return fail(TQP_ERR_INVALID_ARG, "plan.prepared was prepared for another dimension table or key");
    if (p->ngc > 0 || p->naggs > 0) {
        if (p->ngc != pd->ngc) return fail(TQP_ERR_INVALID_ARG, "plan.prepared has other group columns");
        for (int i = 0; i < p->ngc; ++i)
            if (p->group_cols[i] - p->fact->num_cols != pd->group_cols[i])
                return fail(TQP_ERR_INVALID_ARG, "plan.prepared has other group columns");
    }
    return TQP_OK;
}

// ---- left semi / anti plans ---------------------------------------------------
// Each passing fact row counts once if it has an equal dim key (semi) / has
// none (anti), and the rest of the plan reads fact columns only (paper
// Section 5's left-semi and left-anti joins).  So the join reduces to one
// more predicate: k_semi_member writes a uint8 membership column (1 = the row
// passes the plan's predicates and is kept), and the plan runs as a scan plan
// over the fact columns plus that column, with the single predicate
// member == 1.

struct SemiArgs {
    long long n;
    int32_t ncond;
    int32_t anti;
    PjCond cond[TQP_MAX_PREDS];
    PjCol fk;
    JoinHT H{};
    uint8_t* member;
    unsigned long long* acc;  // [0] passing fact rows, [1] finished blocks (zeroed)
    int64_t* d_num_rows;      // nullable
};

__global__ void __launch_bounds__(256) k_semi_member(const __grid_constant__ SemiArgs A) {
    __shared__ unsigned long long part[256 / kWarp];
    long long kmin = 0;
    const bool direct = ht_is_direct(A.H, &kmin);
    unsigned long long passed = 0;
    for (long long r = blockIdx.x * 256LL + threadIdx.x; r < A.n; r += static_cast<long long>(gridDim.x) * 256) {
        bool ok = true;
        for (int q = 0; q < A.ncond; ++q) {
            const PjCond& cd = A.cond[q];
            const uint64_t x = static_cast<uint64_t>(ldg_typed(cd.p, cd.type, r));
            ok = ok && (((x - static_cast<uint64_t>(cd.lo)) <= cd.span) != (cd.negate != 0));
        }
        uint8_t m = 0;
        if (ok) {
            ++passed;
            const bool found = ht_match(A.H, direct, kmin, static_cast<uint64_t>(ldg_typed(A.fk.p, A.fk.type, r))).w != 0;
            m = found != (A.anti != 0) ? 1 : 0;
        }
        A.member[r] = m;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) passed += __shfl_xor_sync(0xffffffffu, passed, o);
    if (threadIdx.x % kWarp == 0) part[threadIdx.x / kWarp] = passed;
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int w = 1; w < 256 / kWarp; ++w) passed += part[w];
    if (passed) atomicAdd(&A.acc[0], passed);
    __threadfence();
    if (atomicAdd(&A.acc[1], 1ULL) != static_cast<unsigned long long>(gridDim.x) - 1ULL) return;
    __threadfence();
    if (A.d_num_rows) *A.d_num_rows = static_cast<int64_t>(atomicAdd(&A.acc[0], 0ULL));
}

static tqp_status run_scan_plan(tqp_ctx* ctx, const tqp_plan* p, const tqp_result* r, cudaStream_t stream);

static tqp_status run_semi_anti_plan(tqp_ctx* ctx, const tqp_plan* p, const tqp_result* r, cudaStream_t stream) {
    const tqp_table* F = p->fact;
    const tqp_table* D = p->dim;
    const int nf = F->num_cols;
    for (int i = 0; i < p->ngc; ++i)
        if (p->group_cols[i] < 0 || p->group_cols[i] >= nf)
            return fail(TQP_ERR_INVALID_ARG, "a semi / anti join plan groups by fact columns only");
    for (int a = 0; a < p->naggs; ++a)
        if (p->aggs[a].fn != TQP_COUNT && !expr_uses_only(p->aggs[a].expr, 0, nf))
            return fail(TQP_ERR_INVALID_ARG, "a semi / anti join plan aggregates fact columns only");
    if (p->has_sum && !expr_uses_only(p->sum_expr, 0, nf))
        return fail(TQP_ERR_INVALID_ARG, "a semi / anti join plan sums fact columns only");
    if (nf + 1 > TQP_MAX_COLS) return fail(TQP_ERR_UNSUPPORTED, "a semi / anti join plan takes at most %d fact columns",
                                           TQP_MAX_COLS - 1);
    const tqp_dim* pd = p->prepared;
    if (pd) TQP_TRY(check_prepared(ctx, p));
    TQP_TRY(check_device_cols(D, std::vector<int>{p->dim_key}, "tqp_run_plan(dim)"));
    Cond cond[TQP_MAX_PREDS];
    int ncond = 0;
    TQP_TRY(lower_preds(F, p->preds, p->npreds, cond, &ncond));
    std::vector<int> fcols{p->fact_fk};
    for (int q = 0; q < ncond; ++q) fcols.push_back(cond[q].col);
    TQP_TRY(check_device_cols(F, fcols, "tqp_run_plan(fact)"));

    // passing fact row ids (before the join) come from the filter kernel
    const bool ids = p->emit_row_ids && r->d_row_ids;
    if (ids) {
        if (!r->d_num_rows) return fail(TQP_ERR_INVALID_ARG, "emit_row_ids needs d_num_rows");
        TQP_TRY(launch_filter(ctx, F, p->preds, p->npreds, nullptr, nullptr, r->d_row_ids, r->capacity_rows,
                              r->d_num_rows, stream, nullptr));
    }
    JoinHT H{};
    if (pd) {
        H = pd->H;
    } else {
        uint32_t* next = nullptr;
        TQP_TRY(ht_build_chain(ctx, D, p->dim_key, &H, &next, stream));
    }
    const long long n = F->num_rows;
    uint8_t* member = static_cast<uint8_t*>(arena_alloc(ctx, static_cast<size_t>(std::max<long long>(n, 16))));
    unsigned long long* acc = static_cast<unsigned long long*>(arena_alloc(ctx, 64));
    if (!member || !acc) return arena_oom(ctx, static_cast<size_t>(n) + 64);
    TQP_CUDA(cudaMemsetAsync(acc, 0, 64, stream));
    SemiArgs A;
    memset(&A, 0, sizeof(A));
    A.n = n;
    A.ncond = ncond;
    A.anti = p->join_kind == TQP_JOIN_LEFT_ANTI;
    for (int q = 0; q < ncond; ++q)
        A.cond[q] = PjCond{static_cast<const unsigned char*>(F->cols[cond[q].col].data), F->cols[cond[q].col].type,
                           cond[q].negate, cond[q].lo, cond[q].span};
    A.fk = PjCol{static_cast<const unsigned char*>(F->cols[p->fact_fk].data), F->cols[p->fact_fk].type, 0};
    A.H = H;
    A.member = member;
    A.acc = acc;
    A.d_num_rows = ids ? nullptr : r->d_num_rows;
    if (n > 0) {
        const int blocks = static_cast<int>(std::min<long long>((n + 255) / 256, 8LL * ctx->num_sms));
        k_semi_member<<<blocks, 256, 0, stream>>>(A);
        TQP_CUDA(cudaGetLastError());
    } else if (A.d_num_rows) {
        TQP_CUDA(cudaMemsetAsync(A.d_num_rows, 0, 8, stream));
    }
    // the scan plan over the fact columns and the membership column
    tqp_column cols[TQP_MAX_COLS];
    for (int c = 0; c < nf; ++c) cols[c] = F->cols[c];
    cols[nf] = tqp_column{member, TQP_U8, 0};
    const tqp_table FM{n, nf + 1, 0, cols};
    tqp_plan q = *p;
    q.fact = &FM;
    q.dim = nullptr;
    q.prepared = nullptr;
    q.join_kind = TQP_JOIN_INNER;
    q.emit_row_ids = 0;
    q.npreds = 1;
    q.preds[0] = tqp_pred{nf, TQP_EQ, 1, 0};
    tqp_result rs = *r;
    rs.d_row_ids = nullptr;
    rs.capacity_rows = 0;
    rs.d_num_rows = r->d_num_joined;  // the scan's passing rows are the kept fact rows
    rs.d_num_joined = nullptr;
    return run_scan_plan(ctx, &q, &rs, stream);
}

static tqp_status run_join_plan(tqp_ctx* ctx, const tqp_plan* p, const tqp_result* r, cudaStream_t stream) {
    const tqp_table* F = p->fact;
    const tqp_table* D = p->dim;
    TQP_TRY(check_table(D, "plan.dim"));
    if (p->join_kind == TQP_JOIN_LEFT_SEMI || p->join_kind == TQP_JOIN_LEFT_ANTI) {
        if (p->fact_fk < 0 || p->fact_fk >= F->num_cols) return fail(TQP_ERR_INVALID_ARG, "fact_fk out of range");
        if (p->dim_key < 0 || p->dim_key >= D->num_cols) return fail(TQP_ERR_INVALID_ARG, "dim_key out of range");
        return run_semi_anti_plan(ctx, p, r, stream);
    }
    if (p->join_kind == TQP_JOIN_LEFT_OUTER)
        return fail(TQP_ERR_UNSUPPORTED, "left outer joins are for tqp_hash_join_kind; plans take inner, semi, anti");
    if (p->join_kind != TQP_JOIN_INNER) return fail(TQP_ERR_INVALID_ARG, "join_kind %d is not a tqp_join_kind",
                                                    p->join_kind);
    const int nf = F->num_cols, nd = D->num_cols;
    if (p->fact_fk < 0 || p->fact_fk >= nf) return fail(TQP_ERR_INVALID_ARG, "fact_fk out of range");
    if (p->dim_key < 0 || p->dim_key >= nd) return fail(TQP_ERR_INVALID_ARG, "dim_key out of range");
    if (nf + nd > 2 * TQP_MAX_COLS) return fail(TQP_ERR_INVALID_ARG, "too many columns");
    for (int i = 0; i < p->ngc; ++i)
        if (p->group_cols[i] < nf || p->group_cols[i] >= nf + nd)
            return fail(TQP_ERR_UNSUPPORTED, "with a join, group columns must be dimension columns");
    for (int a = 0; a < p->naggs; ++a) {
        if (p->aggs[a].fn != TQP_COUNT && !expr_uses_only(p->aggs[a].expr, 0, nf))
            return fail(TQP_ERR_UNSUPPORTED, "with a join, aggregate expressions must use fact columns only");
    }
    if (p->has_sum && !expr_uses_only(p->sum_expr, 0, nf))
        return fail(TQP_ERR_UNSUPPORTED, "with a join, the sum expression must use fact columns only");
    const tqp_dim* pd = p->prepared;
    if (pd) TQP_TRY(check_prepared(ctx, p));
    {
        std::vector<int> dcols{p->dim_key};
        for (int i = 0; i < p->ngc; ++i) dcols.push_back(p->group_cols[i] - nf);
        TQP_TRY(check_device_cols(D, dcols, "tqp_run_plan(dim)"));
    }

    // passing fact row ids (before the join) come from the filter kernel
    if (p->emit_row_ids && r->d_row_ids) {
        if (!r->d_num_rows) return fail(TQP_ERR_INVALID_ARG, "emit_row_ids needs d_num_rows");
        TQP_TRY(launch_filter(ctx, F, p->preds, p->npreds, nullptr, nullptr, r->d_row_ids, r->capacity_rows,
                              r->d_num_rows, stream, nullptr));
    }

    JoinHT H{};
    uint32_t* next = nullptr;
    if (pd) {
        H = pd->H;
        next = pd->next;
    } else {
        TQP_TRY(ht_build_chain(ctx, D, p->dim_key, &H, &next, stream));
    }

    PlanJoinArgs A;
    memset(&A, 0, sizeof(A));
    int ncond = 0;
    TQP_TRY(lower_preds(F, p->preds, p->npreds, A.cond, &ncond));
    A.ncond = ncond;
    A.fk_col = p->fact_fk;
    A.H = H;
    A.next = next;
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
        if (pd) {
            // resident dense ids and keys; this plan's accumulators only
            const size_t acc_bytes = static_cast<size_t>(pd->groups + 1) * A.S.nacc * 8;
            unsigned long long* dacc = static_cast<unsigned long long*>(arena_alloc(ctx, acc_bytes));
            if (!dacc) return arena_oom(ctx, acc_bytes);
            TQP_CUDA(cudaMemsetAsync(dacc, 0, acc_bytes, stream));
            A.S.keys = pd->dkeys;
            A.S.acc = dacc;
            A.S.cap = pd->groups;
            A.S.max_groups = pd->groups;
            A.S.ndistinct = reinterpret_cast<unsigned long long*>(pd->d_groups);
            A.S.d_dense_n = pd->d_groups;
            A.dgs = pd->dgs;
        } else {
            const long long maxg =
                p->max_groups > 0 ? p->max_groups : (p->ngc == 0 ? 1 : std::max<long long>(1, D->num_rows));
            const long long cap = group_table_cap(maxg);
            const long long nd_rows = std::max<long long>(1, D->num_rows);
            // dense accumulators: one entry per distinct dim group (<= maxg, and <= cap + 1 claimed slots)
            const long long dmax = std::min<long long>(maxg, cap + 1);
            unsigned long long* nds = static_cast<unsigned long long*>(arena_alloc(ctx, 256));
            uint32_t* dgs = static_cast<uint32_t*>(arena_alloc(ctx, static_cast<size_t>(nd_rows) * 4));
            unsigned long long* dkeys =
                static_cast<unsigned long long*>(arena_alloc(ctx, static_cast<size_t>(dmax + 1) * 8));
            unsigned long long* dacc =
                static_cast<unsigned long long*>(arena_alloc(ctx, static_cast<size_t>(dmax + 1) * A.S.nacc * 8));
            if (!nds || !dgs || !dkeys || !dacc)
                return arena_oom(ctx, static_cast<size_t>(dmax) * (8 + 8 * A.S.nacc) + nd_rows * 4);
            TQP_TRY(dense_groups_launch(ctx, D, A.S, maxg, &H, dgs, dkeys, dacc, nds, stream));
            long long* d_n = reinterpret_cast<long long*>(nds) + 1;
            // the aggregation state in dense form: entries [0, *d_n)
            A.S.keys = dkeys;
            A.S.acc = dacc;
            A.S.cap = dmax;
            A.S.max_groups = maxg;
            A.S.ndistinct = reinterpret_cast<unsigned long long*>(d_n);
            A.S.d_dense_n = d_n;
            A.dgs = dgs;
        }
    }

    // stage the conditions, the foreign key and every aggregated fact column
    std::vector<int> staged;
    for (int i = 0; i < ncond; ++i) staged.push_back(A.cond[i].col);
    staged.push_back(p->fact_fk);
    if (A.has_sum) expr_cols(A.sum, staged);
    for (int a = 1; a < A.S.nacc; ++a) expr_cols(A.S.acc_expr[a - 1], staged);
    std::sort(staged.begin(), staged.end());
    staged.erase(std::unique(staged.begin(), staged.end()), staged.end());
    TQP_TRY(check_device_cols(F, staged, "tqp_run_plan(fact)"));
    if (static_cast<int>(staged.size()) > kMaxStaged) staged.resize(kMaxStaged);
    int bpr = 0;
    for (int c : staged) bpr += F->cols[c].type == TQP_I64 ? 8 : (F->cols[c].type == TQP_I32 ? 4 : 1);
    const tqp_tuning tu = default_tuning(ctx, bpr, PlanJoinBody::kSmemBytes + args_bytes<PlanJoinArgs>());
    size_t smem = 0;
    TQP_TRY(make_geom(ctx, F, staged, tu, PlanJoinBody::kSmemBytes + args_bytes<PlanJoinArgs>(), &A.G, &smem));
    lower_fast(A.cond, A.ncond, A.G, A.cf, &A.fast);
    lower_join_fast(&A);

    unsigned long long* sc = static_cast<unsigned long long*>(arena_alloc(ctx, 8 * 8));
    if (!sc) return arena_oom(ctx, 64);
    TQP_CUDA(cudaMemsetAsync(sc, 0, 8 * 8, stream));
    A.acc = sc + 1;
    A.d_num_joined = r->d_num_joined;
    A.d_sum = p->has_sum ? r->d_sum : nullptr;
    A.d_num_rows = (p->emit_row_ids && r->d_row_ids) ? nullptr : r->d_num_rows;
    // Radix-partitioned aggregation (partjoin.cuh): the joined rows' group
    // updates land in shared memory instead of L2 reductions.  It declines
    // (nothing launched) for plans outside its shapes or short of scratch,
    // and the fused probe below runs instead.
    bool parted = false;
    if (grouped && F->num_rows >= kPartJoinMinRows && tuned_variant(ctx) == 0) {
        const tqp_status ps = launch_part_join(ctx, A, F, A.S.max_groups, A.acc, stream);
        if (ps == TQP_OK) parted = true;
        else if (ps != TQP_ERR_UNSUPPORTED) return ps;
    }
    // Aggregate by join key first when the fact rows outnumber the build rows:
    // a probe row then costs its key entry's atomics only (no slot load), and
    // one pass over the build rows moves the per-key totals to the groups.
    // Used only if the table turns out direct-mapped; off when scratch is short.
    if (!parted && grouped && A.pjfast && A.fast && H.meta && F->num_rows >= 2 * std::max<long long>(1, D->num_rows)) {
        A.nk = A.S.nacc + (A.has_sum ? 1 : 0);
        const size_t used = ctx->used;
        A.kacc = static_cast<unsigned long long*>(arena_alloc(ctx, static_cast<size_t>(H.cap) * A.nk * 8));
        if (!A.kacc) ctx->used = used;
    }
    if (A.kacc) {
        const long long n = H.cap * A.nk;
        const int blocks = static_cast<int>(std::min<long long>((n + 1023) / 1024, 8LL * ctx->num_sms));
        k_keyfirst_zero<<<std::max(blocks, 1), 256, 0, stream>>>(A.H, A.kacc, A.nk);
        TQP_CUDA(cudaGetLastError());
    }
    if (parted) {
        // launched: counts, sums and group accumulators come from the partitioned kernels
    } else if (F->num_rows > 0) {
        static SmemFlags attr_done;
        TQP_TRY(allow_smem(ctx, reinterpret_cast<const void*>(k_plan_join), attr_done));
        const int g = engine_grid(ctx, reinterpret_cast<const void*>(k_plan_join), smem, A.G.ntiles, tu.ctas_per_sm);
        A.ctl.chunk_tiles = (A.G.ntiles + g - 1) / g;
        A.ctl.nchunks = (A.G.ntiles + A.ctl.chunk_tiles - 1) / A.ctl.chunk_tiles;
        A.ctl.ticket = sc;
        A.ctl.err = ctx->d_err;
        A.ctl.wait_cap = ctx->wait_cap;
        k_plan_join<<<static_cast<int>(A.ctl.nchunks), kEngineThreads, smem, stream>>>(A);
        TQP_CUDA(cudaGetLastError());
        if (A.kacc) {
            const long long nd = D->num_rows;
            const int blocks =
                static_cast<int>(std::min<long long>((nd + kFoldThreads - 1) / kFoldThreads, 4LL * ctx->num_sms));
            k_keyfirst_fold<<<std::max(blocks, 1), kFoldThreads, 0, stream>>>(
                A.H, static_cast<const unsigned char*>(D->cols[p->dim_key].data), D->cols[p->dim_key].type, nd, A.dgs,
                A.S, A.kacc, A.nk, A.has_sum, A.acc, A.d_num_joined, A.d_sum);
            TQP_CUDA(cudaGetLastError());
        }
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

// String columns feed IN / LIKE predicates only: no group key, expression or
// join key may read one (fact columns first, then dimension columns).
static tqp_status check_plan_numeric(const tqp_plan* p) {
    const int F = p->fact->num_cols;
    std::vector<int> fc, dc;
    auto add = [&](int c) {
        if (c < F) fc.push_back(c);
        else dc.push_back(c - F);
    };
    for (int i = 0; i < p->ngc && i < TQP_MAX_GROUP_COLS; ++i) add(p->group_cols[i]);
    auto add_expr = [&](const tqp_expr& e) {
        for (int i = 0; i < e.n && i < TQP_MAX_EXPR; ++i)
            if (e.op[i] == TQP_X_COL) add(static_cast<int>(e.v[i]));
    };
    for (int a = 0; a < p->naggs && a < TQP_MAX_AGGS; ++a)
        if (p->aggs[a].fn != TQP_COUNT) add_expr(p->aggs[a].expr);
    if (p->has_sum) add_expr(p->sum_expr);
    if (p->dim) {
        fc.push_back(p->fact_fk);
        dc.push_back(p->dim_key);
        TQP_TRY(check_table(p->dim, "plan.dim"));
        TQP_TRY(check_numeric_cols(p->dim, dc, "plan (dimension)"));
    }
    return check_numeric_cols(p->fact, fc, "plan");
}

tqp_status run_plan_one(tqp_ctx* ctx, const tqp_plan* p, const tqp_result* r, cudaStream_t stream) {
    if (!p || !r) return fail(TQP_ERR_INVALID_ARG, "plan or result is NULL");
    TQP_TRY(check_table(p->fact, "plan.fact"));
    if (p->ngc < 0 || p->ngc > TQP_MAX_GROUP_COLS) return fail(TQP_ERR_INVALID_ARG, "ngc out of range");
    if (p->naggs < 0 || p->naggs > TQP_MAX_AGGS) return fail(TQP_ERR_INVALID_ARG, "naggs out of range");
    if (p->topk < 0) return fail(TQP_ERR_INVALID_ARG, "topk < 0");
    if (p->ngc + p->naggs > 0 && r->capacity_groups < 1) return fail(TQP_ERR_INVALID_ARG, "capacity_groups < 1");
    TQP_TRY(check_plan_numeric(p));
    arena_reset(ctx);
    // IN / LIKE / NOT LIKE on fact columns: one pre-pass appends a pass column to the fact table
    // (column F); dimension columns, addressed from F on, move up by one
    StrLowered SL;
    TQP_TRY(str_prepass(ctx, p->fact, p->preds, p->npreds, stream, &SL));
    if (SL.active) {
        tqp_plan q = *p;
        const int F = p->fact->num_cols;
        q.fact = &SL.t;
        q.npreds = SL.npreds;
        for (int i = 0; i < SL.npreds; ++i) q.preds[i] = SL.preds[i];
        auto shift = [F](tqp_expr& e) {
            for (int i = 0; i < e.n && i < TQP_MAX_EXPR; ++i)
                if (e.op[i] == TQP_X_COL && e.v[i] >= F) ++e.v[i];
        };
        for (int i = 0; i < q.ngc; ++i)
            if (q.group_cols[i] >= F) ++q.group_cols[i];
        for (int a2 = 0; a2 < q.naggs; ++a2) shift(q.aggs[a2].expr);
        shift(q.sum_expr);
        if (q.dim) return run_join_plan(ctx, &q, r, stream);
        return run_scan_plan(ctx, &q, r, stream);
    }
    if (p->dim) return run_join_plan(ctx, p, r, stream);
    return run_scan_plan(ctx, p, r, stream);
}

static void* top_bytes(tqp_ctx* ctx, size_t bytes) { return arena_alloc_top(ctx, (bytes + 15) / 16 * 16); }

static tqp_status dim_prepare(tqp_ctx* ctx, const tqp_table* D, int32_t key_col, const int32_t* group_cols,
                              int32_t ngc, int64_t max_groups, tqp_dim* d, cudaStream_t st) {
    {
        std::vector<int> cols{key_col};
        for (int i = 0; i < ngc; ++i) cols.push_back(group_cols[i]);
        TQP_TRY(check_device_cols(D, cols, "tqp_dim_prepare"));
    }
    const long long n = D->num_rows;
    d->nrows = n;
    d->key_col = key_col;
    d->ngc = ngc;
    for (int i = 0; i < ngc; ++i) d->group_cols[i] = group_cols[i];
    d->key_data = D->cols[key_col].data;
    // key range first: dense keys get a direct-mapped table sized to their range
    long long* meta = static_cast<long long*>(top_bytes(ctx, 64));
    if (!meta) return arena_oom(ctx, 64);
    TQP_TRY(ht_key_range_launch(ctx, D, key_col, meta, st));
    long long mm[2] = {0, -1};
    TQP_CUDA(cudaMemcpyAsync(mm, meta, sizeof(mm), cudaMemcpyDeviceToHost, st));
    TQP_CUDA(cudaStreamSynchronize(st));
    const bool dense = n > 0 && mm[1] >= mm[0] &&
                       static_cast<unsigned long long>(mm[1]) - static_cast<unsigned long long>(mm[0]) <
                           2ull * static_cast<unsigned long long>(n) + 64;
    d->H.cap = dense ? mm[1] - mm[0] + 1 : ht_cap_dense(n);
    d->H.meta = meta;
    d->H.bidx = nullptr;
    d->H.slots = static_cast<uint4*>(top_bytes(ctx, static_cast<size_t>(d->H.cap + 1) * 16));
    d->next = static_cast<uint32_t*>(top_bytes(ctx, static_cast<size_t>(std::max<long long>(1, n)) * 4));
    d->dgs = static_cast<uint32_t*>(top_bytes(ctx, static_cast<size_t>(std::max<long long>(1, n)) * 4));
    d->d_groups = static_cast<long long*>(top_bytes(ctx, 16));
    if (!d->H.slots || !d->next || !d->dgs || !d->d_groups)
        return arena_oom(ctx, static_cast<size_t>(d->H.cap) * 16 + static_cast<size_t>(n) * 8);
    TQP_TRY(ht_chain_insert_launch(ctx, D, key_col, d->H, d->next, st));
    // dense group ids of the rows (per-call scratch holds the claim table)
    int32_t kt[TQP_MAX_GROUP_COLS] = {0, 0, 0, 0};
    for (int i = 0; i < ngc; ++i) kt[i] = D->cols[group_cols[i]].type;
    GroupSpec S;
    TQP_TRY(lower_group(group_cols, kt, ngc, nullptr, 0, D->num_cols, &S));
    const long long maxg = max_groups > 0 ? max_groups : (ngc == 0 ? 1 : std::max<long long>(1, n));
    const long long dmax = std::min<long long>(maxg, group_table_cap(maxg) + 1);
    unsigned long long* nds = static_cast<unsigned long long*>(arena_alloc(ctx, 256));
    unsigned long long* dkeys = static_cast<unsigned long long*>(arena_alloc(ctx, static_cast<size_t>(dmax + 1) * 8));
    unsigned long long* dacc =
        static_cast<unsigned long long*>(arena_alloc(ctx, static_cast<size_t>(dmax + 1) * S.nacc * 8));
    if (!nds || !dkeys || !dacc) return arena_oom(ctx, static_cast<size_t>(dmax) * 16);
    TQP_TRY(dense_groups_launch(ctx, D, S, maxg, &d->H, d->dgs, dkeys, dacc, nds, st));
    TQP_TRY(take_device_error(ctx, st));
    long long G = 0;
    TQP_CUDA(cudaMemcpy(&G, reinterpret_cast<long long*>(nds) + 1, sizeof(G), cudaMemcpyDeviceToHost));
    if (G > maxg) return fail(TQP_ERR_CAPACITY, "dimension has more than max_groups = %lld groups", (long long)maxg);
    d->groups = G;
    d->dkeys = static_cast<unsigned long long*>(top_bytes(ctx, static_cast<size_t>(G + 1) * 8));
    if (!d->dkeys) return arena_oom(ctx, static_cast<size_t>(G + 1) * 8);
    TQP_CUDA(cudaMemcpy(d->dkeys, dkeys, static_cast<size_t>(G + 1) * 8, cudaMemcpyDeviceToDevice));
    TQP_CUDA(cudaMemcpy(d->d_groups, &G, sizeof(G), cudaMemcpyHostToDevice));
    TQP_CUDA(cudaDeviceSynchronize());
    return TQP_OK;
}

}  // namespace tqp

using namespace tqp;

extern "C" tqp_status tqp_dim_prepare(tqp_ctx* ctx, const tqp_table* dim, int32_t key_col, const int32_t* group_cols,
                                      int32_t ngc, int64_t max_groups, void* stream, tqp_dim** out) {
    clear_error();
    TQP_TRY(check_ctx(ctx));
    if (!out) return fail(TQP_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    TQP_TRY(check_table(dim, "dim"));
    if (key_col < 0 || key_col >= dim->num_cols) return fail(TQP_ERR_INVALID_ARG, "key_col out of range");
    {
        std::vector<int> kc{key_col};
        for (int i = 0; i < ngc && group_cols && i < TQP_MAX_GROUP_COLS; ++i) kc.push_back(group_cols[i]);
        TQP_TRY(check_numeric_cols(dim, kc, "tqp_dim_prepare"));
    }
    if (ngc < 0 || ngc > TQP_MAX_GROUP_COLS || (ngc > 0 && !group_cols))
        return fail(TQP_ERR_INVALID_ARG, "bad group columns");
    for (int i = 0; i < ngc; ++i)
        if (group_cols[i] < 0 || group_cols[i] >= dim->num_cols)
            return fail(TQP_ERR_INVALID_ARG, "group column %d out of range", group_cols[i]);
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(TQP_ERR_CUDA, "cannot select device %d", ctx->device);
    arena_reset(ctx);
    tqp_dim* d = new (std::nothrow) tqp_dim();
    if (!d) return fail(TQP_ERR_OUT_OF_MEMORY, "host allocation failed");
    d->ctx = ctx;
    top_open(ctx);
    d->top_before = ctx->top;
    const tqp_status s = dim_prepare(ctx, dim, key_col, group_cols, ngc, max_groups, d, static_cast<cudaStream_t>(stream));
    d->top_after = ctx->top;
    if (s != TQP_OK) {
        top_close(ctx, d->top_before, d->top_after);
        delete d;
        return s;
    }
    *out = d;
    return TQP_OK;
}

extern "C" int64_t tqp_dim_groups(const tqp_dim* d) { return d ? d->groups : -1; }

extern "C" tqp_status tqp_dim_destroy(tqp_dim* d) {
    clear_error();
    if (!d) return TQP_OK;
    {
        DeviceGuard g(d->ctx->device);
        cudaDeviceSynchronize();  // no plan in flight may still read the prepared tables
        top_close(d->ctx, d->top_before, d->top_after);
    }
    delete d;
    return TQP_OK;
}

extern "C" tqp_status tqp_run_plan(tqp_ctx* ctx, const tqp_plan* plan, const tqp_result* res, void* stream) {
    clear_error();
    TQP_TRY(check_ctx(ctx));
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(TQP_ERR_CUDA, "cannot select device %d", ctx->device);
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!plan || !res || !plan->fact) return run_plan_one(ctx, plan, res, st);  // reports the error
    std::vector<int> cols;
    for (int i = 0; i < plan->npreds && i < TQP_MAX_PREDS; ++i) cols.push_back(plan->preds[i].col);
    if (plan->dim) cols.push_back(plan->fact_fk);
    for (int i = 0; i < plan->ngc && i < TQP_MAX_GROUP_COLS && !plan->dim; ++i) cols.push_back(plan->group_cols[i]);
    for (int a = 0; a < plan->naggs && a < TQP_MAX_AGGS; ++a)
        if (plan->aggs[a].fn != TQP_COUNT) expr_col_ids(&plan->aggs[a].expr, cols);
    if (plan->has_sum) expr_col_ids(&plan->sum_expr, cols);
    char key[96];
    snprintf(key, sizeof(key), "plan r%d b%d j%d p%d g%d k%d", rows_class(plan->fact->num_rows),
             row_bytes(plan->fact, cols), plan->dim ? rows_class(plan->dim->num_rows) + 1 : 0,
             plan->prepared ? 1 : 0, plan->ngc + plan->naggs > 0 ? 1 : 0, plan->topk > 0 ? 1 : 0);
    auto run = [&]() { return run_plan_one(ctx, plan, res, st); };
    int opts = 0;
    if (plan->dim && !plan->prepared) opts |= kTuneHt;
    if (plan->dim && (plan->ngc > 0 || plan->naggs > 0) && plan->fact->num_rows >= kPartJoinMinRows)
        opts |= kTuneVariant | kTuneV0Shapeless;
    return tuned(ctx, key, st, opts, run);
}
