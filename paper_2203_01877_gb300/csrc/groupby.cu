// tqp_groupby_agg: hash group-by aggregation with exact int64 sums.
//
// Semantics of paper Section 5.4 (Algorithm 3: one output row per distinct
// key tuple, keys ascending, aggregates evaluated per group), computed
// without sorting the input:
//   * group keys are packed into one order-preserving uint64 (uint8 -> 8 bits,
//     int32 -> 32 bits with the sign bit flipped, int64 -> 64 bits flipped;
//     first key column most significant), so unsigned order of packed keys is
//     the lexicographic order of the int64-widened tuples;
//   * each persistent CTA pre-aggregates into a shared-memory open-addressing
//     table (bounded probing; rows that do not fit go straight to the global
//     table), and flushes it once into a global open-addressing table with
//     64-bit atomics -- few global atomics when groups are few (the Q1 shape);
//   * finalize collects the occupied slots, orders them by packed key (one
//     CTA bitonic sort for small tables, the radix sort otherwise), unpacks
//     the keys and computes AVG as one IEEE division of the exact sum by the
//     count.
// int64 addition is associative and commutative, so the sums do not depend on
// the order atomics land in.
#include <cstdio>

#include "host.h"
#include "group.cuh"
#include "bodies.cuh"
#include "finalize.cuh"
#include "groupdirect.cuh"

namespace tqp {

tqp_status radix_sort_pairs(uint64_t* k0, uint32_t* v0, uint64_t* k1, uint32_t* v1, const long long* d_n,
                            long long n_max, int begin_bit, int end_bit, void* scratch, cudaStream_t stream,
                            bool* result_in_1);
size_t radix_sort_scratch(long long n_max);



__global__ void __launch_bounds__(kEngineThreads, GroupBody::kMinBlocks) k_groupby(const __grid_constant__ GroupArgs P) {
    extern __shared__ __align__(128) unsigned char smem[];
    const GroupArgs& A = stage_args(P, smem + kHeaderBytes);
    GroupBody body(A, smem + kHeaderBytes + args_bytes<GroupArgs>());
    run_engine(A.G, A.ctl, body, smem, args_bytes<GroupArgs>());
}

__global__ void __launch_bounds__(kDirThreads, kDirMinBlocks) k_groupby_direct(const __grid_constant__ GroupDirectArgs A) {
    extern __shared__ __align__(16) unsigned char dsm[];
    group_direct_block<false>(A, dsm, blockIdx.x, gridDim.x);
}

// The same for tables with MIN/MAX accumulators (a separate kernel keeps the
// sums-only one's register allocation).
__global__ void __launch_bounds__(kDirThreads, kDirMinBlocks) k_groupby_direct_mm(const __grid_constant__ GroupDirectArgs A) {
    extern __shared__ __align__(16) unsigned char dsm[];
    group_direct_block<true>(A, dsm, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(kDirThreads) k_groupby_dprep(const __grid_constant__ GroupDirectArgs A,
                                                               unsigned long long* kpart) {
    group_direct_prep_block(A, kpart, blockIdx.x, gridDim.x);
}

// ---- finalize ----------------------------------------------------------------

__global__ void __launch_bounds__(kFinThreads) k_groupby_finalize_small(const __grid_constant__ GroupSpec S,
                                                                        const __grid_constant__ GroupOut O) {
    extern __shared__ __align__(16) unsigned char fsm[];
    finalize_small_block(S, O, fsm);
}

// Large tables: collect (key, slot) pairs, radix sort, emit.
__global__ void k_groupby_collect(const __grid_constant__ GroupSpec S, uint64_t* pk, uint32_t* ps,
                                  long long* n_out) {
    // warp-uniform trip count: blockDim is a multiple of 32
    for (long long base = blockIdx.x * static_cast<long long>(blockDim.x); base <= S.cap;
         base += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long i = base + threadIdx.x;
        const bool used = i <= S.cap && slot_used(S, i);
        const long long p = warp_claim(reinterpret_cast<unsigned long long*>(n_out), used);
        if (used) {
            pk[p] = slot_key(S, i);
            ps[p] = static_cast<uint32_t>(i);
        }
    }
}

__global__ void k_groupby_emit(const __grid_constant__ GroupSpec S, const __grid_constant__ GroupOut O,
                               const uint64_t* pk, const uint32_t* ps, const long long* n_in) {
    const long long G = *n_in;
    const bool overflow = static_cast<long long>(*S.ndistinct) > S.max_groups || G > O.capacity;
    if (overflow) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            *O.num_groups = -1;
            latch_error(O.err, TQP_ERR_CAPACITY);
        }
        return;
    }
    for (long long g = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; g < G;
         g += static_cast<long long>(gridDim.x) * blockDim.x)
        emit_group(S, O, g, pk[g], ps[g]);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (S.ngc == 0 && G == 0) {
            emit_group(S, O, 0, 0, -1);
            if (O.fvals)
                for (int j = 0; j < S.naggs; ++j)
                    if (S.agg_fn[j] == TQP_AVG) O.fvals[j] = __longlong_as_double(0x7ff8000000000000LL);
            *O.num_groups = 1;
        } else {
            *O.num_groups = G;
        }
    }
}

// ---- host ------------------------------------------------------------------------

static bool same_expr(const DExpr& a, const DExpr& b) {
    if (a.n != b.n) return false;
    for (int i = 0; i < a.n; ++i)
        if (a.op[i] != b.op[i] || a.v[i] != b.v[i]) return false;
    return true;
}

// Fill the key/aggregate part of a GroupSpec (table pointers are set later).
// key_types[i] is the dtype of key column i; exprs address `ncols` columns.
tqp_status lower_group(const int32_t* key_cols, const int32_t* key_types, int32_t ngc, const tqp_agg* aggs,
                       int32_t naggs, int ncols, GroupSpec* S) {
    memset(S, 0, sizeof(*S));
    if (ngc < 0 || ngc > TQP_MAX_GROUP_COLS)
        return fail(TQP_ERR_INVALID_ARG, "ngc %d outside [0, %d]", ngc, TQP_MAX_GROUP_COLS);
    if (naggs < 0 || naggs > TQP_MAX_AGGS)
        return fail(TQP_ERR_INVALID_ARG, "naggs %d outside [0, %d]", naggs, TQP_MAX_AGGS);
    if (naggs > 0 && !aggs) return fail(TQP_ERR_INVALID_ARG, "aggs is NULL");
    S->ngc = ngc;
    int width = 0;
    for (int i = 0; i < ngc; ++i) {
        if (key_cols[i] < 0 || key_cols[i] >= ncols)
            return fail(TQP_ERR_INVALID_ARG, "group column %d out of range", key_cols[i]);
        S->key_col[i] = key_cols[i];
        S->key_bits[i] = key_types[i] == TQP_U8 ? 8 : (key_types[i] == TQP_I32 ? 32 : 64);
        width += S->key_bits[i];
    }
    if (width > 64) return fail(TQP_ERR_UNSUPPORTED, "group key tuple is %d bits wide (at most 64 supported)", width);
    S->width = width;
    S->nacc = 1;
    S->naggs = naggs;
    for (int j = 0; j < naggs; ++j) {
        const int fn = aggs[j].fn;
        if (fn != TQP_SUM && fn != TQP_COUNT && fn != TQP_AVG && fn != TQP_MIN && fn != TQP_MAX)
            return fail(TQP_ERR_INVALID_ARG, "aggregate %d: unknown function %d", j, fn);
        S->agg_fn[j] = fn;
        if (fn == TQP_COUNT) {
            S->agg_acc[j] = 0;
            continue;
        }
        const int kind = fn == TQP_MAX ? kAccMax : (fn == TQP_MIN ? kAccMin : kAccSum);
        DExpr e;
        TQP_TRY(lower_expr(&aggs[j].expr, ncols, &e));
        int found = -1;
        for (int a = 1; a < S->nacc; ++a)
            if (same_expr(S->acc_expr[a - 1], e) && S->acc_kind[a - 1] == kind) found = a;
        if (found < 0) {
            found = S->nacc++;
            S->acc_expr[found - 1] = e;
            S->acc_kind[found - 1] = kind;
            if (kind != kAccSum) S->minmax = 1;
        }
        S->agg_acc[j] = found;
    }
    return TQP_OK;
}

long long group_table_cap(long long capacity_groups) {
    long long cap = 64;
    while (cap < 2 * capacity_groups) cap <<= 1;
    return cap;
}

size_t group_table_bytes(long long cap, int nacc) {
    return (static_cast<size_t>(cap + 1) * 8 + 255) / 256 * 256 + static_cast<size_t>(cap + 1) * nacc * 8 + 256;
}

// Carve the table out of `mem` and clear it on `stream`.
tqp_status group_table_init(GroupSpec* S, void* mem, long long cap, long long max_groups, cudaStream_t stream,
                            bool clear) {
    unsigned char* p = static_cast<unsigned char*>(mem);
    S->cap = cap;
    S->max_groups = max_groups;
    S->keys = reinterpret_cast<unsigned long long*>(p);
    p += (static_cast<size_t>(cap + 1) * 8 + 255) / 256 * 256;
    S->acc = reinterpret_cast<unsigned long long*>(p);
    S->ndistinct = S->acc + (cap + 1) * S->nacc;
    if (!clear) return TQP_OK;  // the caller's first kernel clears it
    TQP_CUDA(cudaMemsetAsync(S->keys, 0xFF, static_cast<size_t>(cap + 1) * 8, stream));
    TQP_CUDA(cudaMemsetAsync(S->acc, 0, static_cast<size_t>(cap + 1) * S->nacc * 8 + 8, stream));
    return TQP_OK;
}

// Finalize a filled table into the caller's output arrays.
tqp_status group_finalize(tqp_ctx* ctx, const GroupSpec& S, const GroupOut& O, cudaStream_t stream) {
    if (S.cap <= kSmallCap) {
        const size_t smem = static_cast<size_t>(2 * kSmallCap) * (8 + 4);
        static SmemFlags attr_done;
        TQP_TRY(allow_smem(ctx, reinterpret_cast<const void*>(k_groupby_finalize_small), attr_done));
        k_groupby_finalize_small<<<1, kFinThreads, smem, stream>>>(S, O);
        TQP_CUDA(cudaGetLastError());
        return TQP_OK;
    }
    const long long nmax = S.cap + 1;
    const size_t pair_bytes = static_cast<size_t>(nmax) * 12 + 512;
    unsigned char* buf = static_cast<unsigned char*>(arena_alloc(ctx, 2 * pair_bytes + 256));
    void* rs = arena_alloc(ctx, radix_sort_scratch(nmax));
    if (!buf || !rs) return arena_oom(ctx, 2 * pair_bytes + radix_sort_scratch(nmax));
    long long* d_n = reinterpret_cast<long long*>(buf);
    uint64_t* k0 = reinterpret_cast<uint64_t*>(buf + 256);
    uint64_t* k1 = k0 + nmax;
    uint32_t* v0 = reinterpret_cast<uint32_t*>(k1 + nmax);
    uint32_t* v1 = v0 + nmax;
    TQP_CUDA(cudaMemsetAsync(d_n, 0, sizeof(long long), stream));
    const int threads = 256;
    const int blocks = static_cast<int>(std::min<long long>((nmax + threads - 1) / threads, ctx->num_sms * 8LL));
    k_groupby_collect<<<blocks, threads, 0, stream>>>(S, k0, v0, d_n);
    bool in1 = false;
    const int end_bit = (S.width + 7) / 8 * 8;
    TQP_TRY(radix_sort_pairs(k0, v0, k1, v1, d_n, nmax, 0, end_bit, rs, stream, &in1));
    const int eblocks = static_cast<int>(
        std::max<long long>(1, std::min<long long>((std::min(nmax, O.capacity) + threads - 1) / threads,
                                                   ctx->num_sms * 8LL)));
    k_groupby_emit<<<eblocks, threads, 0, stream>>>(S, O, in1 ? k1 : k0, in1 ? v1 : v0, d_n);
    TQP_CUDA(cudaGetLastError());
    return TQP_OK;
}

__global__ void __launch_bounds__(kTopThreads) k_topk_level0(const __grid_constant__ GroupSpec S, int rank_acc, int k,
                                                             TopBuf out, unsigned long long* total,
                                                             const unsigned int* run) {
    topk_level0_block(S, rank_acc, k, out, total, blockIdx.x, run);
}

__global__ void __launch_bounds__(kTopThreads) k_topk_reduce(const __grid_constant__ GroupSpec S, TopBuf in,
                                                             long long n_in, int k, TopBuf out, int emit,
                                                             const __grid_constant__ GroupOut O,
                                                             const unsigned long long* total, int64_t* total_out,
                                                             const unsigned int* run) {
    topk_reduce_block(S, in, n_in, k, out, emit, O, total, total_out, blockIdx.x, run);
}

__global__ void __launch_bounds__(kSelThreads) k_topsel_pass(const __grid_constant__ GroupSpec S, int rank_acc, int k,
                                                             TopSel* sel, int pass, long long nblocks) {
    topsel_pass_block(S, rank_acc, k, sel, pass, blockIdx.x, nblocks);
}

__global__ void __launch_bounds__(kSelThreads) k_topsel_collect(const __grid_constant__ GroupSpec S, int rank_acc,
                                                                TopSel* sel, TopBuf cand) {
    topsel_collect_block(S, rank_acc, sel, cand, blockIdx.x);
}

__global__ void __launch_bounds__(kTopThreads) k_topsel_emit(const __grid_constant__ GroupSpec S, int k, const TopSel* sel,
                                                             TopBuf cand, const __grid_constant__ GroupOut O,
                                                             int64_t* total_out) {
    topsel_emit_block(S, k, sel, cand, O, total_out);
}

tqp_status group_topk(tqp_ctx* ctx, const GroupSpec& S, const GroupOut& O, int k, int agg, int64_t* total_groups,
                      cudaStream_t stream) {
    if (k < 1 || k > kTopBlock / 2) return fail(TQP_ERR_UNSUPPORTED, "top-k needs 1 <= k <= %d", kTopBlock / 2);
    if (agg < 0 || agg >= S.naggs) return fail(TQP_ERR_INVALID_ARG, "topk_agg %d out of range", agg);
    const int rank_acc = S.agg_acc[agg];
    const long long nb0 = (S.cap + 1 + kTopBlock - 1) / kTopBlock;
    const long long ncand = nb0 * k;
    auto alloc_buf = [&](TopBuf* b) -> bool {
        b->rank = static_cast<long long*>(arena_alloc(ctx, ncand * 8));
        b->key = static_cast<uint64_t*>(arena_alloc(ctx, ncand * 8));
        b->slot = static_cast<uint32_t*>(arena_alloc(ctx, ncand * 4));
        return b->rank && b->key && b->slot;
    };
    TopBuf a, b, cand;
    unsigned long long* total = static_cast<unsigned long long*>(arena_alloc(ctx, 256));
    TopSel* sel = static_cast<TopSel*>(arena_alloc(ctx, sizeof(TopSel)));
    cand.rank = static_cast<long long*>(arena_alloc(ctx, kSelCand * 8));
    cand.key = static_cast<uint64_t*>(arena_alloc(ctx, kSelCand * 8));
    cand.slot = static_cast<uint32_t*>(arena_alloc(ctx, kSelCand * 4));
    if (!alloc_buf(&a) || !alloc_buf(&b) || !total || !sel || !cand.rank || !cand.key || !cand.slot)
        return arena_oom(ctx, ncand * 40 + sizeof(TopSel) + kSelCand * 20);
    TQP_CUDA(cudaMemsetAsync(total, 0, 8, stream));
    TQP_CUDA(cudaMemsetAsync(sel, 0, sizeof(TopSel), stream));
    // radix select of the k-th largest, then one sort of the candidates
    const long long nbs = (S.cap + 1 + kSelSlots - 1) / kSelSlots;
    for (int pass = 0; pass < kSelPasses; ++pass)
        k_topsel_pass<<<static_cast<unsigned>(nbs), kSelThreads, 0, stream>>>(S, rank_acc, k, sel, pass, nbs);
    k_topsel_collect<<<static_cast<unsigned>(nbs), kSelThreads, 0, stream>>>(S, rank_acc, sel, cand);
    k_topsel_emit<<<1, kTopThreads, 0, stream>>>(S, k, sel, cand, O, total_groups);
    // the tournament, only when the select ended with too many ties (its blocks return early otherwise)
    const unsigned int* run = &sel->fallback;
    k_topk_level0<<<static_cast<unsigned>(nb0), kTopThreads, 0, stream>>>(S, rank_acc, k, a, total, run);
    long long n = ncand;
    while (n > kTopBlock) {
        const long long blocks = (n + kTopBlock - 1) / kTopBlock;
        k_topk_reduce<<<static_cast<unsigned>(blocks), kTopThreads, 0, stream>>>(S, a, n, k, b, 0, O, total, nullptr,
                                                                              run);
        std::swap(a, b);
        n = blocks * k;
    }
    k_topk_reduce<<<1, kTopThreads, 0, stream>>>(S, a, n, k, b, 1, O, total, total_groups, run);
    TQP_CUDA(cudaGetLastError());
    return TQP_OK;
}

void lower_group_fast(GroupArgs* A) {
    A->kfast = 0;
    const GroupSpec& S = A->S;
    if (S.nacc - 1 > kFastSums) return;
    for (int i = 0; i < S.ngc; ++i) {
        const int c = S.key_col[i];
        if (c < 0 || c >= A->G.ncols || A->G.col[c].slot < 0) return;
        const int t = A->G.col[c].type;
        if (S.key_bits[i] != (t == TQP_U8 ? 8 : (t == TQP_I32 ? 32 : 64))) return;
        A->key_soff[i] = A->G.col[c].soff;
        A->key_type[i] = t;
    }
    for (int a = 0; a + 1 < S.nacc; ++a)
        if (!lower_prod(S.acc_expr[a], A->G, &A->pf[a])) return;
    A->kfast = 1;
}

// The direct (unstaged) kernel applies when groups are few (max_groups <=
// kDirMaxGroups), the accumulators are the count and at most three
// closed-form sums, and conditions are at most kDirConds.  Columns are
// 16-byte aligned, as every table requires, so its vector loads are too.
// Lowered through a geometry whose stage offset of every column is its
// column number, so that the lowered forms name columns.
constexpr long long kDirMaxGroups = 64;

bool lower_group_direct(const tqp_table* t, const GroupArgs& A, long long max_groups, GroupDirectArgs* D) {
    if (max_groups > kDirMaxGroups || A.ncond > kDirConds || A.S.nacc > kDirAcc || t->num_rows <= 0) return false;
    ScanGeom G;
    memset(&G, 0, sizeof(G));
    G.n = t->num_rows;
    G.ncols = t->num_cols;
    for (int c = 0; c < t->num_cols; ++c) {
        G.col[c].ptr = static_cast<const unsigned char*>(t->cols[c].data);
        G.col[c].type = t->cols[c].type;
        G.col[c].slot = 0;
        G.col[c].soff = c;
    }
    memset(D, 0, sizeof(*D));
    D->n = t->num_rows;
    // the distinct columns a step reads, each with its block in a warp slot
    int lane_bytes = 0;
    // (returns the column's block offset in a warp slot, -1 when the slot is full)
    auto pref = [&](int c) -> int {
        for (int i = 0; i < D->npref; ++i)
            if (D->pref[i].p == G.col[c].ptr && D->pref[i].type == G.col[c].type) return D->pref[i].off;
        if (D->npref == kDirPrefCols) return -1;
        const int es = t->cols[c].type == TQP_I64 ? 8 : (t->cols[c].type == TQP_I32 ? 4 : 1);
        D->pref[D->npref] = DirPref{G.col[c].ptr, t->cols[c].type, 32 * lane_bytes};
        lane_bytes += 4 * es;
        return D->pref[D->npref++].off;
    };
    CondFast cf[TQP_MAX_PREDS];
    int32_t fast = 0;
    lower_fast(A.cond, A.ncond, G, cf, &fast);
    if (!fast) return false;
    D->ncond = A.ncond;
    for (int q = 0; q < A.ncond; ++q) {
        const int c = cf[q].soff;
        D->cond[q] = DirCond{G.col[c].ptr, cf[q].type, cf[q].negate, cf[q].lo, cf[q].span, pref(c), 0};
        if (D->cond[q].soff < 0) return false;
    }
    D->ngc = A.S.ngc;
    for (int i = 0; i < A.S.ngc; ++i) {
        const int c = A.S.key_col[i];
        D->key[i] = DirCol{G.col[c].ptr, t->cols[c].type, pref(c)};
        if (D->key[i].soff < 0) return false;
    }
    D->nsum = A.S.nacc - 1;
    for (int a = 0; a < D->nsum; ++a) {
        ProdForm pf;
        if (!lower_prod(A.S.acc_expr[a], G, &pf)) return false;
        for (int k = 0; k < 2; ++k) {
            const bool col = pf.kind[k] != kFacConst;
            const int so = col ? pref(pf.soff[k]) : 0;
            if (so < 0) return false;
            D->f[a][k] = DirFactor{col ? G.col[pf.soff[k]].ptr : nullptr, col ? pf.type[k] : 0, pf.kind[k], pf.a[k],
                                   pf.b[k], so, 0};
        }
    }
    D->kw32 = A.S.width <= 32;
    return lane_bytes <= kDirLaneBytes;
}

tqp_status launch_sort_agg(tqp_ctx* ctx, const tqp_table* t, const Cond* cond, int ncond, GroupSpec* S,
                           long long cap_groups, cudaStream_t stream);

tqp_status launch_groupby(tqp_ctx* ctx, const tqp_table* t, const tqp_pred* preds, int32_t npreds,
                          const int32_t* group_cols, int32_t ngc, const tqp_agg* aggs, int32_t naggs,
                          int64_t* d_keys, int64_t* d_ivals, double* d_fvals, int64_t capacity_groups,
                          int64_t* d_num_groups, cudaStream_t stream, long long max_groups, int topk, int topk_agg,
                          int64_t* d_total_groups) {
    // the top-k arguments first: a call rejected for them launches nothing
    if (topk > 0 && topk > kTopBlock / 2)
        return fail(TQP_ERR_UNSUPPORTED, "top-k needs 1 <= k <= %d", kTopBlock / 2);
    if (topk > 0 && (topk_agg < 0 || topk_agg >= naggs))
        return fail(TQP_ERR_INVALID_ARG, "topk_agg %d out of range", topk_agg);
    // IN / LIKE / NOT LIKE: one pre-pass writes a pass column that the scan then filters on
    StrLowered SL;
    TQP_TRY(str_prepass(ctx, t, preds, npreds, stream, &SL));
    if (SL.active) {
        t = &SL.t;
        preds = SL.preds;
        npreds = SL.npreds;
    }
    GroupArgs A;
    memset(&A, 0, sizeof(A));
    int ncond = 0;
    TQP_TRY(lower_preds(t, preds, npreds, A.cond, &ncond));
    A.ncond = ncond;
    if (ngc > 0 && !group_cols) return fail(TQP_ERR_INVALID_ARG, "group_cols is NULL");
    int32_t types[TQP_MAX_GROUP_COLS] = {0, 0, 0, 0};
    for (int i = 0; i < ngc && i < TQP_MAX_GROUP_COLS; ++i) {
        if (group_cols[i] < 0 || group_cols[i] >= t->num_cols)
            return fail(TQP_ERR_INVALID_ARG, "group column %d out of range", group_cols[i]);
        types[i] = t->cols[group_cols[i]].type;
    }
    TQP_TRY(check_numeric_cols(t, std::vector<int>(group_cols, group_cols + std::max(0, ngc)), "tqp_groupby_agg"));
    TQP_TRY(lower_group(group_cols, types, ngc, aggs, naggs, t->num_cols, &A.S));
    bool need_f = false;
    for (int j = 0; j < naggs; ++j) need_f |= aggs[j].fn == TQP_AVG;
    if (need_f && !d_fvals) return fail(TQP_ERR_INVALID_ARG, "d_fvals is NULL but an AVG is requested");

    // stage every referenced column: group-by inputs are usually mostly passing rows
    std::vector<int> staged;
    for (int i = 0; i < ncond; ++i) staged.push_back(A.cond[i].col);
    for (int i = 0; i < ngc; ++i) staged.push_back(group_cols[i]);
    for (int a = 1; a < A.S.nacc; ++a) expr_cols(A.S.acc_expr[a - 1], staged);
    TQP_TRY(check_numeric_cols(t, staged, "tqp_groupby_agg"));
    TQP_TRY(check_device_cols(t, staged, "tqp_groupby_agg"));
    std::vector<int> u = staged;
    std::sort(u.begin(), u.end());
    u.erase(std::unique(u.begin(), u.end()), u.end());
    if (static_cast<int>(u.size()) > kMaxStaged) u.resize(kMaxStaged);
    int bpr = 0;
    for (int c : u) bpr += t->cols[c].type == TQP_I64 ? 8 : (t->cols[c].type == TQP_I32 ? 4 : 1);
    const tqp_tuning tu = default_tuning(ctx, bpr, GroupBody::kSmemBytes + args_bytes<GroupArgs>());
    size_t smem = 0;
    TQP_TRY(make_geom(ctx, t, u, tu, GroupBody::kSmemBytes + args_bytes<GroupArgs>(), &A.G, &smem));
    lower_fast(A.cond, A.ncond, A.G, A.cf, &A.fast);
    lower_group_fast(&A);

    // variant 1: the sort-based aggregation (Algorithm 3), timed against this path by the autotuner
    // (and MIN/MAX beyond the direct kernel's shapes: the hash engine body only adds)
    GroupDirectArgs D;
    const bool direct = lower_group_direct(t, A, max_groups, &D);
    if ((ngc > 0 && tuned_variant(ctx) == 1) || (A.S.minmax && !direct)) {
        GroupOut O{d_keys, d_ivals, d_fvals, capacity_groups, d_num_groups, ctx->d_err};
        TQP_TRY(launch_sort_agg(ctx, t, A.cond, A.ncond, &A.S, std::max<long long>(max_groups, 1), stream));
        if (topk > 0) return group_topk(ctx, A.S, O, topk, topk_agg, d_total_groups, stream);
        return group_finalize(ctx, A.S, O, stream);
    }
    const long long cap = group_table_cap(max_groups);
    void* tab = arena_alloc(ctx, group_table_bytes(cap, A.S.nacc));
    unsigned long long* ticket = static_cast<unsigned long long*>(arena_alloc(ctx, 256));
    if (!tab || !ticket) return arena_oom(ctx, group_table_bytes(cap, A.S.nacc));
    GroupOut O{d_keys, d_ivals, d_fvals, capacity_groups, d_num_groups, ctx->d_err};
    TQP_TRY(group_table_init(&A.S, tab, cap, max_groups, stream, !direct));
    if (direct) {
        // two launches: the range pass (which also clears the table), then the
        // aggregation, whose last CTA finalizes the table unless top-k follows
        D.S = A.S;
        D.err = ctx->d_err;
        D.O = O;
        D.fin = topk > 0 ? 0 : 1;
        static SmemFlags attr_done, attr_mm;
        const void* kern = A.S.minmax ? reinterpret_cast<const void*>(k_groupby_direct_mm)
                                      : reinterpret_cast<const void*>(k_groupby_direct);
        TQP_TRY(allow_smem(ctx, kern, A.S.minmax ? attr_mm : attr_done));
        // large inputs: the kernel compiled for this query's shape (same arguments and results)
        const void* jk = A.S.minmax ? nullptr : jit_group_direct(ctx, D, t->num_rows);
        if (jk) kern = jk;
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kDirThreads, kDirSmemBytes) != cudaSuccess ||
            occ < 1)
            occ = 1;
        const long long nq = (t->num_rows + 3) / 4;
        const long long blocks = std::min<long long>((nq + kDirThreads - 1) / kDirThreads,
                                                     static_cast<long long>(occ) * ctx->num_sms);
        // key ranges first (few distinct values get dense slot ids): one
        // record per range block, reduced by every CTA of the aggregation
        const int nparts = static_cast<int>(
            std::max<long long>(1, std::min<long long>((t->num_rows + 8191) / 8192, ctx->num_sms)));
        unsigned long long* kpart =
            static_cast<unsigned long long*>(arena_alloc(ctx, static_cast<size_t>(nparts) * 2 * kDirKeys * 8));
        unsigned int* done = static_cast<unsigned int*>(arena_alloc(ctx, 16));
        if (!kpart || !done) return arena_oom(ctx, static_cast<size_t>(nparts) * 2 * kDirKeys * 8 + 16);
        D.done = done;
        if (D.ngc > 0) {
            D.kpart = kpart;
            D.nparts = nparts;
        }
        k_groupby_dprep<<<D.ngc > 0 ? nparts : 1, kDirThreads, 0, stream>>>(D, kpart);
        TQP_CUDA(cudaGetLastError());
        const unsigned grid = static_cast<unsigned>(std::max<long long>(blocks, 1));
        if (jk) {
            void* args[] = {&D};
            TQP_CUDA(cudaLaunchKernel(jk, dim3(grid), dim3(kDirThreads), args, kDirSmemBytes, stream));
            jit_count_launch();
        } else if (A.S.minmax) {
            k_groupby_direct_mm<<<grid, kDirThreads, kDirSmemBytes, stream>>>(D);
        } else {
            k_groupby_direct<<<grid, kDirThreads, kDirSmemBytes, stream>>>(D);
        }
        TQP_CUDA(cudaGetLastError());
        if (topk > 0) return group_topk(ctx, A.S, O, topk, topk_agg, d_total_groups, stream);
        return TQP_OK;
    } else if (t->num_rows > 0) {
        static SmemFlags attr_done;
        TQP_TRY(allow_smem(ctx, reinterpret_cast<const void*>(k_groupby), attr_done));
        const int g = engine_grid(ctx, reinterpret_cast<const void*>(k_groupby), smem, A.G.ntiles, tu.ctas_per_sm);
        A.ctl.chunk_tiles = (A.G.ntiles + g - 1) / g;
        A.ctl.nchunks = (A.G.ntiles + A.ctl.chunk_tiles - 1) / A.ctl.chunk_tiles;
        A.ctl.ticket = ticket;
        A.ctl.err = ctx->d_err;
        A.ctl.wait_cap = ctx->wait_cap;
        TQP_CUDA(cudaMemsetAsync(ticket, 0, 8, stream));
        k_groupby<<<static_cast<int>(A.ctl.nchunks), kEngineThreads, smem, stream>>>(A);
        TQP_CUDA(cudaGetLastError());
    }
    if (topk > 0) return group_topk(ctx, A.S, O, topk, topk_agg, d_total_groups, stream);
    return group_finalize(ctx, A.S, O, stream);
}

}  // namespace tqp

using namespace tqp;

extern "C" tqp_status tqp_groupby_agg(tqp_ctx* ctx, const tqp_table* t, const tqp_pred* preds, int32_t npreds,
                                      const int32_t* group_cols, int32_t ngc, const tqp_agg* aggs, int32_t naggs,
                                      int64_t* d_keys, int64_t* d_ivals, double* d_fvals, int64_t capacity_groups,
                                      int64_t* d_num_groups, void* stream) {
    clear_error();
    TQP_TRY(check_ctx(ctx));
    TQP_TRY(check_table(t, "tqp_groupby_agg"));
    if (!d_num_groups) return fail(TQP_ERR_INVALID_ARG, "d_num_groups is NULL");
    if (capacity_groups < 1 || capacity_groups > (1LL << 30))
        return fail(TQP_ERR_INVALID_ARG, "capacity_groups %lld outside [1, 2^30]", (long long)capacity_groups);
    if (ngc > 0 && !d_keys) return fail(TQP_ERR_INVALID_ARG, "d_keys is NULL");
    if (naggs > 0 && !d_ivals) return fail(TQP_ERR_INVALID_ARG, "d_ivals is NULL");
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(TQP_ERR_CUDA, "cannot select device %d", ctx->device);
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::vector<int> cols;
    for (int i = 0; i < npreds && i < TQP_MAX_PREDS && preds; ++i) cols.push_back(preds[i].col);
    for (int i = 0; i < ngc && i < TQP_MAX_GROUP_COLS && group_cols; ++i) cols.push_back(group_cols[i]);
    for (int a = 0; a < naggs && a < TQP_MAX_AGGS && aggs; ++a)
        if (aggs[a].fn != TQP_COUNT) expr_col_ids(&aggs[a].expr, cols);
    char key[96];
    snprintf(key, sizeof(key), "groupby r%d b%d g%d a%d", rows_class(t->num_rows), row_bytes(t, cols), ngc, naggs);
    auto run = [&]() {
        arena_reset(ctx);
        return launch_groupby(ctx, t, preds, npreds, group_cols, ngc, aggs, naggs, d_keys, d_ivals, d_fvals,
                              capacity_groups, d_num_groups, st, capacity_groups, 0, 0, nullptr);
    };
    return tuned(ctx, key, st, ngc > 0 ? (kTuneVariant | kTuneV1Shapeless) : 0, run);
}
