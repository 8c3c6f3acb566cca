// tqp_filter_shared: shared scans of many filter queries (see multi.cuh for
// the kernel).  This file holds the host side: lowering each query, packing
// queries into launches (at most 32 queries, 8 staged columns, 2 distinct sum
// expressions and the shared-memory table budget per launch), tabulating the
// interval masks of every condition column, and the launches themselves.
// The batched executor (batch.cu) packs the filter-only plans of a batch with
// the same functions.
#include <algorithm>
#include <climits>
#include <cstdio>
#include <vector>

#include "host.h"
#include "multi.cuh"

namespace tqp {

static void type_range(int type, int64_t* tmin, int64_t* tmax) {
    if (type == TQP_I32) {
        *tmin = INT32_MIN;
        *tmax = INT32_MAX;
    } else if (type == TQP_U8) {
        *tmin = 0;
        *tmax = 255;
    } else {
        *tmin = INT64_MIN;
        *tmax = INT64_MAX;
    }
}

// The range test of a lowered condition (the engine's Cond semantics).
static bool cond_pass(const Cond& c, int64_t x) {
    const bool in = static_cast<uint64_t>(x) - static_cast<uint64_t>(c.lo) <= c.span;
    return in != (c.negate != 0);
}

static bool same_expr(const DExpr& a, const DExpr& b) {
    if (a.n != b.n) return false;
    for (int i = 0; i < a.n; ++i)
        if (a.op[i] != b.op[i] || a.v[i] != b.v[i]) return false;
    return true;
}

// Whether a query can share a scan: numeric columns only, and no LIKE.
static bool mq_shareable(const tqp_table* t, const tqp_pred* preds, int32_t npreds) {
    for (int i = 0; i < npreds && i < TQP_MAX_PREDS && preds; ++i) {
        if (preds[i].op == TQP_LIKE || preds[i].op == TQP_NOT_LIKE) return false;
        if (preds[i].col >= 0 && preds[i].col < t->num_cols && t->cols[preds[i].col].type == TQP_CHAR) return false;
    }
    return true;
}

tqp_status mq_lower_query(const tqp_table* t, const tqp_pred* preds, int32_t npreds, const tqp_expr* sum_expr,
                          MqQuery* q) {
    *q = MqQuery();
    // IN lists on numeric columns become membership tests of the column tables; the rest are ranges
    if (npreds < 0 || npreds > TQP_MAX_PREDS)
        return fail(TQP_ERR_INVALID_ARG, "npreds %d outside [0, %d]", npreds, TQP_MAX_PREDS);
    if (npreds > 0 && !preds) return fail(TQP_ERR_INVALID_ARG, "preds is NULL");
    tqp_pred ranges[TQP_MAX_PREDS];
    int nr = 0;
    size_t used = 0;  // the value bytes the single-query pre-pass would hold (same budget)
    for (int i = 0; i < npreds; ++i) {
        const tqp_pred& p = preds[i];
        if (p.op != TQP_IN) {
            ranges[nr++] = p;
            continue;
        }
        if (p.col < 0 || p.col >= t->num_cols)
            return fail(TQP_ERR_INVALID_ARG, "predicate %d: column %d out of range", i, p.col);
        if (p.hi < 0 || (p.hi > 0 && p.lo == 0))
            return fail(TQP_ERR_INVALID_ARG, "predicate %d: bad value list", i);
        const int64_t* v = reinterpret_cast<const int64_t*>(static_cast<uintptr_t>(p.lo));
        std::vector<int64_t> vals(v, v + p.hi);
        std::sort(vals.begin(), vals.end());
        vals.erase(std::unique(vals.begin(), vals.end()), vals.end());
        if (used + vals.size() * 8 > static_cast<size_t>(TQP_MAX_SET_BYTES))
            return fail(TQP_ERR_UNSUPPORTED, "IN / LIKE values take more than %d bytes", TQP_MAX_SET_BYTES);
        used = (used + vals.size() * 8 + 15) / 16 * 16;
        q->ins.push_back({p.col, vals});
    }
    TQP_TRY(lower_preds(t, ranges, nr, q->cond, &q->ncond));
    std::vector<int> cols;
    for (int i = 0; i < q->ncond; ++i) cols.push_back(q->cond[i].col);
    for (const auto& in : q->ins) cols.push_back(in.first);
    if (sum_expr) {
        TQP_TRY(lower_expr(sum_expr, t->num_cols, &q->sum));
        q->has_sum = true;
        expr_cols(q->sum, cols);
        TQP_TRY(check_numeric_cols(t, cols, "tqp_filter_shared sum_expr"));
        // the closed product form is required: try it with every column staged
        ScanGeom G;
        memset(&G, 0, sizeof(G));
        G.ncols = t->num_cols;
        for (int c = 0; c < t->num_cols; ++c) {
            G.col[c].slot = c;
            G.col[c].type = t->cols[c].type;
        }
        ProdForm pf;
        q->closed = lower_prod(q->sum, G, &pf);
    }
    std::sort(cols.begin(), cols.end());
    cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
    q->cols = cols;
    if (q->has_sum) expr_cols(q->sum, q->ecols);
    for (int i = 0; i < q->ncond; ++i) {
        const Cond& cd = q->cond[i];
        int64_t tmin, tmax;
        type_range(t->cols[cd.col].type, &tmin, &tmax);
        const uint64_t ends[2] = {static_cast<uint64_t>(cd.lo), static_cast<uint64_t>(cd.lo) + cd.span + 1u};
        for (uint64_t e : ends) {
            const int64_t b = static_cast<int64_t>(e);
            if (b > tmin && b <= tmax) q->bps.push_back({cd.col, b});
        }
    }
    for (const auto& in : q->ins) {  // each value v is the interval [v, v + 1)
        int64_t tmin, tmax;
        type_range(t->cols[in.first].type, &tmin, &tmax);
        for (int64_t v : in.second)
            for (uint64_t e : {static_cast<uint64_t>(v), static_cast<uint64_t>(v) + 1u}) {
                const int64_t b = static_cast<int64_t>(e);
                if (b > tmin && b <= tmax) q->bps.push_back({in.first, b});
            }
    }
    std::sort(q->bps.begin(), q->bps.end());
    q->bps.erase(std::unique(q->bps.begin(), q->bps.end()), q->bps.end());
    return TQP_OK;
}

// Interval masks of every condition column of the queries `members` (in that
// lane order).  Fills A->nq, A->all, A->ncols and A->c[] (all but the stage
// offsets); false when the tables exceed the shared-memory budget.
static bool mq_tables(const tqp_table* t, const std::vector<MqQuery>& qs, const std::vector<int>& members,
                      MultiArgs* A, std::vector<uint32_t>* words, std::vector<int64_t>* breaks,
                      bool want_masks = true) {
    const int nq = static_cast<int>(members.size());
    A->nq = nq;
    A->all = nq >= 32 ? 0xffffffffu : ((1u << nq) - 1u);
    A->ncols = 0;
    words->clear();
    breaks->clear();
    std::vector<int> ccols;
    for (int m : members) {
        for (int i = 0; i < qs[m].ncond; ++i) ccols.push_back(qs[m].cond[i].col);
        for (const auto& in : qs[m].ins) ccols.push_back(in.first);
    }
    std::sort(ccols.begin(), ccols.end());
    ccols.erase(std::unique(ccols.begin(), ccols.end()), ccols.end());

    struct ColTab {
        int col, type;
        std::vector<int64_t> B;   // breakpoints inside the type's range, ascending
        std::vector<uint32_t> M;  // B.size() + 1 interval masks
    };
    std::vector<ColTab> tabs;
    for (int c : ccols) {
        ColTab ct;
        ct.col = c;
        ct.type = t->cols[c].type;
        int64_t tmin, tmax;
        type_range(ct.type, &tmin, &tmax);
        for (int m : members)
            for (const auto& b : qs[m].bps)
                // (only breakpoints inside the column's range: one at or below the
                // smallest value, or above the largest, separates no two values)
                if (b.first == c) ct.B.push_back(b.second);
        std::sort(ct.B.begin(), ct.B.end());
        ct.B.erase(std::unique(ct.B.begin(), ct.B.end()), ct.B.end());
        auto mask_at = [&](int64_t x) {
            uint32_t mk = 0;
            for (int l = 0; l < nq; ++l) {
                const MqQuery& q = qs[members[l]];
                bool ok = true;
                for (int i = 0; i < q.ncond; ++i)
                    if (q.cond[i].col == c && !cond_pass(q.cond[i], x)) ok = false;
                for (const auto& in : q.ins)
                    if (in.first == c && !std::binary_search(in.second.begin(), in.second.end(), x)) ok = false;
                if (ok) mk |= 1u << l;
            }
            return mk;
        };
        // every breakpoint is > tmin, so B[0] - 1 is a value of the column
        // (sizes only: masks of zero, the packing decisions do not need them)
        ct.M.push_back(want_masks ? mask_at(ct.B.empty() ? tmin : ct.B[0] - 1) : 0u);
        for (int64_t b : ct.B) ct.M.push_back(want_masks ? mask_at(b) : 0u);
        if (ct.B.empty()) {
            A->all &= ct.M[0];  // the same outcome for every value: no lookup needed
            continue;
        }
        tabs.push_back(ct);
    }
    if (static_cast<int>(tabs.size()) > kMaxStaged) return false;
    // direct tables where they fit beside the searched form of the later columns
    std::vector<size_t> searched_words(tabs.size() + 1, 0);
    for (size_t i = tabs.size(); i-- > 0;) searched_words[i] = searched_words[i + 1] + tabs[i].B.size() + 1;
    for (size_t i = 0; i < tabs.size(); ++i) {
        const ColTab& ct = tabs[i];
        MqCol& mc = A->c[A->ncols++];
        memset(&mc, 0, sizeof(mc));
        mc.col = ct.col;
        mc.type = ct.type;
        const uint64_t span = static_cast<uint64_t>(ct.B.back()) - static_cast<uint64_t>(ct.B.front());
        const size_t len = span <= static_cast<uint64_t>(kMqDirectMax - 2) ? static_cast<size_t>(span) + 2 : 0;
        mc.off = static_cast<int32_t>(words->size());
        if (len && words->size() + len + searched_words[i + 1] <= static_cast<size_t>(kMqWords)) {
            mc.direct = 1;
            mc.base = ct.B.front();
            mc.len = static_cast<int32_t>(len);
            words->push_back(ct.M[0]);
            if (!want_masks) {
                words->resize(words->size() + len - 1);
                continue;
            }
            size_t j = 0;  // breakpoints <= the entry's value
            for (size_t d = 0; d + 1 < len; ++d) {
                const int64_t x = static_cast<int64_t>(static_cast<uint64_t>(ct.B.front()) + d);
                while (j < ct.B.size() && ct.B[j] <= x) ++j;
                words->push_back(ct.M[j]);
            }
        } else {
            mc.direct = 0;
            mc.len = static_cast<int32_t>(ct.B.size());
            mc.boff = static_cast<int32_t>(breaks->size());
            int s = 1;
            while (s * 2 <= mc.len) s *= 2;
            mc.steps = s;
            for (int64_t b : ct.B) breaks->push_back(b);
            for (uint32_t mk : ct.M) words->push_back(mk);
        }
    }
    return words->size() <= static_cast<size_t>(kMqWords) && breaks->size() <= static_cast<size_t>(kMqBreaks);
}

// Columns a launch stages: the condition columns that need a lookup and every
// column of the sum expressions.
static std::vector<int> mq_staged(const std::vector<MqQuery>& qs, const std::vector<int>& members,
                                  const MultiArgs& A) {
    std::vector<int> staged;
    for (int k = 0; k < A.ncols; ++k) staged.push_back(A.c[k].col);
    for (int m : members)
        if (qs[m].has_sum) expr_cols(qs[m].sum, staged);
    std::sort(staged.begin(), staged.end());
    staged.erase(std::unique(staged.begin(), staged.end()), staged.end());
    return staged;
}

// Distinct sum expressions of `members`, in first-use order.
static std::vector<DExpr> mq_exprs(const std::vector<MqQuery>& qs, const std::vector<int>& members) {
    std::vector<DExpr> ex;
    for (int m : members) {
        if (!qs[m].has_sum) continue;
        bool seen = false;
        for (const DExpr& e : ex) seen = seen || same_expr(e, qs[m].sum);
        if (!seen) ex.push_back(qs[m].sum);
    }
    return ex;
}

// One pack under construction: its members, expressions, and per condition
// column the sorted breakpoints (the sizes of its lookup tables follow from
// them exactly as mq_tables lays them out).
struct PackState {
    std::vector<int> members;
    std::vector<DExpr> exprs;
    std::vector<int> ecols;                        // expression columns
    std::vector<std::pair<int, std::vector<int64_t>>> B;  // ascending column order

    std::vector<int64_t>* col_bps(int c) {
        for (auto& e : B)
            if (e.first == c) return &e.second;
        return nullptr;
    }
};

// Would `q` fit `g` (members, expressions, staged columns, table budget)?
static bool pack_try(const PackState& g, const MqQuery& q) {
    if (g.members.size() + 1 > static_cast<size_t>(kMqMax)) return false;
    size_t nex = g.exprs.size();
    if (q.has_sum) {
        bool seen = false;
        for (const DExpr& e : g.exprs) seen = seen || same_expr(e, q.sum);
        if (!seen) ++nex;
    }
    if (nex > static_cast<size_t>(kMqExprs)) return false;
    // per condition column: breakpoint count and span after adding q's
    struct Sz {
        int col;
        size_t k;
        int64_t lo, hi;
    };
    std::vector<Sz> sz;
    for (const auto& e : g.B) sz.push_back({e.first, e.second.size(), e.second.front(), e.second.back()});
    for (const auto& b : q.bps) {
        Sz* z = nullptr;
        for (auto& x : sz)
            if (x.col == b.first) z = &x;
        const std::vector<int64_t>* old = nullptr;
        for (const auto& e : g.B)
            if (e.first == b.first) old = &e.second;
        if (!z) {
            sz.push_back({b.first, 0, b.second, b.second});
            z = &sz.back();
        }
        // (q's own breakpoints are distinct: sorted and deduplicated when lowered)
        if (!(old && std::binary_search(old->begin(), old->end(), b.second))) ++z->k;
        z->lo = std::min(z->lo, b.second);
        z->hi = std::max(z->hi, b.second);
    }
    std::sort(sz.begin(), sz.end(), [](const Sz& a, const Sz& b) { return a.col < b.col; });
    if (sz.size() > static_cast<size_t>(kMaxStaged)) return false;
    // staged columns: the lookup columns and every expression column
    std::vector<int> staged = g.ecols;
    staged.insert(staged.end(), q.ecols.begin(), q.ecols.end());
    for (const auto& z : sz) staged.push_back(z.col);
    std::sort(staged.begin(), staged.end());
    staged.erase(std::unique(staged.begin(), staged.end()), staged.end());
    if (staged.size() > static_cast<size_t>(kMaxStaged)) return false;
    // the table budget, decided as mq_tables decides it
    std::vector<size_t> searched(sz.size() + 1, 0);
    for (size_t i = sz.size(); i-- > 0;) searched[i] = searched[i + 1] + sz[i].k + 1;
    size_t words = 0, breaks = 0;
    for (size_t i = 0; i < sz.size(); ++i) {
        const uint64_t span = static_cast<uint64_t>(sz[i].hi) - static_cast<uint64_t>(sz[i].lo);
        const size_t len = span <= static_cast<uint64_t>(kMqDirectMax - 2) ? static_cast<size_t>(span) + 2 : 0;
        if (len && words + len + searched[i + 1] <= static_cast<size_t>(kMqWords)) {
            words += len;
        } else {
            words += sz[i].k + 1;
            breaks += sz[i].k;
        }
    }
    return words <= static_cast<size_t>(kMqWords) && breaks <= static_cast<size_t>(kMqBreaks);
}

static void pack_add(PackState* g, const MqQuery& q, int idx) {
    g->members.push_back(idx);
    if (q.has_sum) {
        bool seen = false;
        for (const DExpr& e : g->exprs) seen = seen || same_expr(e, q.sum);
        if (!seen) g->exprs.push_back(q.sum);
    }
    g->ecols.insert(g->ecols.end(), q.ecols.begin(), q.ecols.end());
    for (const auto& b : q.bps) {
        std::vector<int64_t>* v = g->col_bps(b.first);
        if (!v) {
            g->B.push_back({b.first, {}});
            std::sort(g->B.begin(), g->B.end(),
                      [](const std::pair<int, std::vector<int64_t>>& x, const std::pair<int, std::vector<int64_t>>& y) {
                          return x.first < y.first;
                      });
            v = g->col_bps(b.first);
        }
        auto it = std::lower_bound(v->begin(), v->end(), b.second);
        if (it == v->end() || *it != b.second) v->insert(it, b.second);
    }
}

void mq_pack(const tqp_table* t, const std::vector<MqQuery>& qs, std::vector<std::vector<int>>* groups,
             std::vector<int>* singles) {
    (void)t;
    groups->clear();
    singles->clear();
    std::vector<PackState> packs;
    for (int i = 0; i < static_cast<int>(qs.size()); ++i) {
        const MqQuery& q = qs[i];
        if (q.alone || (q.has_sum && !q.closed) || q.cols.size() > static_cast<size_t>(kMaxStaged)) {
            singles->push_back(i);
            continue;
        }
        bool placed = false;
        for (auto& g : packs)  // first fit
            if (pack_try(g, q)) {
                pack_add(&g, q, i);
                placed = true;
                break;
            }
        if (placed) continue;
        PackState g;
        if (pack_try(g, q)) {
            pack_add(&g, q, i);
            packs.push_back(std::move(g));
        } else {
            singles->push_back(i);
        }
    }
    for (auto& g : packs) {
        if (g.members.size() >= static_cast<size_t>(kMqMinPack)) groups->push_back(g.members);
        else singles->insert(singles->end(), g.members.begin(), g.members.end());
    }
    std::sort(singles->begin(), singles->end());
}

tqp_status mq_lower_group(const tqp_ctx* ctx, const tqp_table* t, const std::vector<MqQuery>& qs,
                          const std::vector<int>& members, const tqp_tuning* tu_in, int extra_smem, bool fixed_body,
                          MultiArgs* A, std::vector<unsigned char>* blob, size_t* smem, int* ctas_per_sm) {
    memset(A, 0, sizeof(*A));
    std::vector<uint32_t> words;
    std::vector<int64_t> breaks;
    if (!mq_tables(t, qs, members, A, &words, &breaks))
        return fail(TQP_ERR_UNSUPPORTED, "shared scan: lookup tables exceed the shared-memory budget");
    A->body_bytes = fixed_body ? MultiBody::kSmemBytes
                               : mq_body_bytes(static_cast<int>(words.size()), static_cast<int>(breaks.size()));
    const int body_smem = extra_smem + A->body_bytes;
    const std::vector<int> staged = mq_staged(qs, members, *A);
    if (staged.size() > static_cast<size_t>(kMaxStaged))
        return fail(TQP_ERR_UNSUPPORTED, "shared scan: more than %d columns", kMaxStaged);
    TQP_TRY(check_device_cols(t, staged, "tqp_filter_shared"));
    int bpr = 0;
    for (int c : staged) bpr += t->cols[c].type == TQP_I64 ? 8 : (t->cols[c].type == TQP_I32 ? 4 : 1);
    const tqp_tuning tu = tu_in ? *tu_in : default_tuning(ctx, bpr, body_smem);
    TQP_TRY(make_geom(ctx, t, staged, tu, body_smem, &A->G, smem));
    *ctas_per_sm = tu.ctas_per_sm;
    for (int k = 0; k < A->ncols; ++k) A->c[k].soff = A->G.col[A->c[k].col].soff;
    const std::vector<DExpr> ex = mq_exprs(qs, members);
    A->nexpr = static_cast<int32_t>(ex.size());
    for (size_t e = 0; e < ex.size(); ++e) {
        if (!lower_prod(ex[e], A->G, &A->e[e]))
            return fail(TQP_ERR_UNSUPPORTED, "shared scan: sum expression is not a product of affine factors");
        // the table column of each factor (ragged tiles read the columns directly)
        for (int i = 0; i < 2; ++i) {
            A->ecol[e][i] = -1;
            if (A->e[e].kind[i] == kFacConst) continue;
            for (int c = 0; c < A->G.ncols; ++c)
                if (A->G.col[c].slot >= 0 && A->G.col[c].soff == A->e[e].soff[i]) A->ecol[e][i] = c;
        }
    }
    A->esel = 0;
    std::vector<MqOut> outs;
    for (size_t l = 0; l < members.size(); ++l) {
        const MqQuery& q = qs[members[l]];
        if (q.has_sum && ex.size() > 1 && same_expr(q.sum, ex[1])) A->esel |= 1u << l;
        outs.push_back(q.out);
    }
    A->nwords = static_cast<int32_t>(words.size());
    A->nbreaks = static_cast<int32_t>(breaks.size());
    // blob: words | breakpoints (8-aligned) | outputs (8-aligned)
    const size_t wbytes = (words.size() * 4 + 15) / 16 * 16;
    const size_t bbytes = (breaks.size() * 8 + 15) / 16 * 16;
    blob->assign(wbytes + bbytes + outs.size() * sizeof(MqOut), 0);
    if (!words.empty()) memcpy(blob->data(), words.data(), words.size() * 4);
    if (!breaks.empty()) memcpy(blob->data() + wbytes, breaks.data(), breaks.size() * 8);
    memcpy(blob->data() + wbytes + bbytes, outs.data(), outs.size() * sizeof(MqOut));
    // device offsets (set to real pointers by mq_bind)
    A->words = reinterpret_cast<const uint32_t*>(static_cast<uintptr_t>(0));
    A->breaks = reinterpret_cast<const int64_t*>(static_cast<uintptr_t>(wbytes));
    A->out = reinterpret_cast<const MqOut*>(static_cast<uintptr_t>(wbytes + bbytes));
    return TQP_OK;
}

void mq_bind(MultiArgs* A, const unsigned char* d_blob) {
    A->words = reinterpret_cast<const uint32_t*>(d_blob + reinterpret_cast<uintptr_t>(A->words));
    A->breaks = reinterpret_cast<const int64_t*>(d_blob + reinterpret_cast<uintptr_t>(A->breaks));
    A->out = reinterpret_cast<const MqOut*>(d_blob + reinterpret_cast<uintptr_t>(A->out));
}

__global__ void __launch_bounds__(kEngineThreads, MultiBody::kMinBlocks)
    k_filter_multi(const __grid_constant__ MultiLaunch P) {
    extern __shared__ __align__(128) unsigned char smem[];
    const MultiArgs& A = stage_args(P.A, smem + kHeaderBytes);
    MultiBody body(A, smem + kHeaderBytes + args_bytes<MultiArgs>(), P.words, P.breaks, P.out);
    run_engine(A.G, A.ctl, body, smem, args_bytes<MultiArgs>(), A.body_bytes);
}

// Zero outputs of queries over an empty table.
static tqp_status mq_zero(const MqOut& o, cudaStream_t st) {
    if (o.count) TQP_CUDA(cudaMemsetAsync(o.count, 0, sizeof(int64_t), st));
    if (o.count2) TQP_CUDA(cudaMemsetAsync(o.count2, 0, sizeof(int64_t), st));
    if (o.sum) TQP_CUDA(cudaMemsetAsync(o.sum, 0, sizeof(int64_t), st));
    return TQP_OK;
}

// The host checks of the single-query scan (its pre-pass, predicates and sum),
// so that a bad query stops the call before anything is launched.
static tqp_status check_alone(tqp_ctx* ctx, const tqp_table* t, const tqp_scan_query& q) {
    StrLowered SL;
    TQP_TRY(str_prepass(ctx, t, q.preds, q.npreds, nullptr, &SL, true));
    Cond cond[TQP_MAX_PREDS];
    int ncond = 0;
    TQP_TRY(lower_preds(t, SL.preds, SL.npreds, cond, &ncond));
    if (q.has_sum) {
        DExpr e;
        TQP_TRY(lower_expr(&q.sum_expr, t->num_cols, &e));
        std::vector<int> c;
        expr_cols(e, c);
        TQP_TRY(check_numeric_cols(t, c, "tqp_filter_shared sum_expr"));
    }
    return TQP_OK;
}

static tqp_status shared_run(tqp_ctx* ctx, const tqp_table* t, const tqp_scan_query* q, int32_t nq,
                             int32_t* launch_of, cudaStream_t st) {
    std::vector<MqQuery> qs(nq);
    for (int i = 0; i < nq; ++i) {
        if (!mq_shareable(t, q[i].preds, q[i].npreds)) {
            TQP_TRY(check_alone(ctx, t, q[i]));
            qs[i].alone = true;
            continue;
        }
        TQP_TRY(mq_lower_query(t, q[i].preds, q[i].npreds, q[i].has_sum ? &q[i].sum_expr : nullptr, &qs[i]));
        qs[i].out.count = q[i].d_count;
        qs[i].out.sum = q[i].has_sum ? q[i].d_sum : nullptr;
        qs[i].out.rlo = 0;
        qs[i].out.rhi = t->num_rows;
    }
    std::vector<std::vector<int>> groups;
    std::vector<int> singles;
    mq_pack(t, qs, &groups, &singles);
    if (launch_of) {
        for (int i = 0; i < nq; ++i) launch_of[i] = -1;
        for (size_t g = 0; g < groups.size(); ++g)
            for (int m : groups[g]) launch_of[m] = static_cast<int32_t>(g);
    }
    static SmemFlags attr;
    TQP_TRY(allow_smem(ctx, reinterpret_cast<const void*>(k_filter_multi), attr));
    for (const auto& g : groups) {
        MultiArgs A;
        std::vector<unsigned char> blob;
        size_t smem = 0;
        int per_sm = 0;
        TQP_TRY(mq_lower_group(ctx, t, qs, g, nullptr, args_bytes<MultiArgs>(), false, &A, &blob, &smem, &per_sm));
        if (A.G.ntiles == 0) {
            for (int m : g) TQP_TRY(mq_zero(qs[m].out, st));
            continue;
        }
        const size_t acc_bytes = (2 * kMqMax + 2) * sizeof(unsigned long long);
        unsigned char* d = static_cast<unsigned char*>(arena_alloc(ctx, acc_bytes));
        if (!d) return arena_oom(ctx, acc_bytes);
        TQP_CUDA(cudaMemsetAsync(d, 0, acc_bytes, st));
        // the tables and outputs go in the kernel parameters (offsets as recorded by mq_lower_group)
        std::vector<MultiLaunch> L(1);
        memcpy(L[0].words, blob.data(), static_cast<size_t>(A.nwords) * 4);
        memcpy(L[0].breaks, blob.data() + reinterpret_cast<uintptr_t>(A.breaks), static_cast<size_t>(A.nbreaks) * 8);
        memcpy(L[0].out, blob.data() + reinterpret_cast<uintptr_t>(A.out), static_cast<size_t>(A.nq) * sizeof(MqOut));
        A.words = nullptr;
        A.breaks = nullptr;
        A.out = nullptr;
        A.ctl.ticket = reinterpret_cast<unsigned long long*>(d);
        A.acc = reinterpret_cast<unsigned long long*>(d) + 1;
        A.ctl.err = ctx->d_err;
        A.ctl.wait_cap = ctx->wait_cap;
        const int grid = engine_grid(ctx, reinterpret_cast<const void*>(k_filter_multi), smem, A.G.ntiles, per_sm);
        A.ctl.chunk_tiles = (A.G.ntiles + grid - 1) / grid;
        A.ctl.nchunks = (A.G.ntiles + A.ctl.chunk_tiles - 1) / A.ctl.chunk_tiles;
        L[0].A = A;
        k_filter_multi<<<static_cast<unsigned>(A.ctl.nchunks), kEngineThreads, smem, st>>>(L[0]);
        TQP_CUDA(cudaGetLastError());
    }
    for (int i : singles)
        TQP_TRY(launch_filter(ctx, t, q[i].preds, q[i].npreds, q[i].has_sum ? &q[i].sum_expr : nullptr,
                              q[i].has_sum ? q[i].d_sum : nullptr, nullptr, 0, q[i].d_count, st, nullptr));
    return TQP_OK;
}

}  // namespace tqp

using namespace tqp;

extern "C" tqp_status tqp_filter_shared(tqp_ctx* ctx, const tqp_table* t, const tqp_scan_query* queries, int32_t nq,
                                        int32_t* launch_of, void* stream) {
    clear_error();
    TQP_TRY(check_ctx(ctx));
    TQP_TRY(check_table(t, "tqp_filter_shared"));
    if (nq < 0) return fail(TQP_ERR_INVALID_ARG, "nq < 0");
    if (nq > 0 && !queries) return fail(TQP_ERR_INVALID_ARG, "queries is NULL");
    for (int i = 0; i < nq; ++i) {
        if (!queries[i].d_count) return fail(TQP_ERR_INVALID_ARG, "query %d: d_count is NULL", i);
        if ((queries[i].has_sum != 0) != (queries[i].d_sum != nullptr))
            return fail(TQP_ERR_INVALID_ARG, "query %d: has_sum and d_sum must both be set or both be unset", i);
    }
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(TQP_ERR_CUDA, "cannot select device %d", ctx->device);
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    // shape class: rows, bytes per row of every column the queries read, query count
    std::vector<int> cols;
    for (int i = 0; i < nq; ++i) {
        for (int k = 0; k < queries[i].npreds && k < TQP_MAX_PREDS; ++k) cols.push_back(queries[i].preds[k].col);
        if (queries[i].has_sum) expr_col_ids(&queries[i].sum_expr, cols);
    }
    for (int& c : cols) c = c < 0 || c >= t->num_cols ? 0 : c;
    char key[96];
    snprintf(key, sizeof(key), "shared r%d b%d q%d", rows_class(t->num_rows), row_bytes(t, cols),
             nq <= 2 ? nq : (nq <= 8 ? 8 : (nq <= 16 ? 16 : 32)));
    auto run = [&]() {
        arena_reset(ctx);
        return shared_run(ctx, t, queries, nq, launch_of, st);
    };
    return tuned(ctx, key, st, 0, run);
}
