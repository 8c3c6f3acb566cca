// Batched execution of many independent plans: tqp_batch_create / _run /
// _destroy and tqp_run_plans.
//
// The paper runs one query at a time with intra-operator parallelism only
// (Section 4.3).  Here every plan of a batch is lowered into jobs once, and
// each phase of all jobs runs as ONE kernel over a flattened block space
// (a host-built map gives every block its job), so the number of launches
// does not grow with the number of plans:
//   fill      clear every job's scratch (tables, counters)
//   range     build-key [min, max] of every join (direct-mapped tables)
//   build     chained hash tables + dimension group claims of all joins
//   number    dense group ids (claim-table ranges)
//   remap     dimension row -> dense group id
//   direct    dense ids into the slots of unique build keys
//   few-group group-bys (at most 64 groups, closed-form sums): the key-range
//             pass, then the direct kernel (vector reads one warp step ahead,
//             lane-private tables), each job a contiguous range of blocks
//   scan      one persistent launch of the staged scan engine per body kind
//             (filter, shared filter, group-by, joined aggregation): CTAs draw chunk
//             tickets across the tables of every job of that kind (uneven
//             sizes balance themselves); each kind gets its own shared-memory
//             layout and occupancy.  Filter-only work (counts and sums
//             without row ids) of several plans over the same table is packed
//             into shared scans: one pass evaluates up to 32 of them
//             (multi.cuh), so a batch of such queries reads the table once
//             per pack instead of once per plan
//   fold      joins that aggregated by join key: key totals -> groups
//   compact   selection masks -> row ids
//   finalize  one CTA per small group table (keys ascending)
//   top-k     radix select of the k-th largest (histogram passes, a collect
//             and one sort per plan); the bitonic tournament, one
//             launch per level, only for plans whose select ends in ties
// A tqp_batch is lowered and captured into a CUDA graph once; each run is
// one graph launch.  Plans outside these shapes (large group tables without
// top-k) run through the single-plan path after the batch's kernels, inside
// the same graph, with scratch of their own.
#include <algorithm>
#include <new>
#include <vector>

#include "host.h"
#include "bodies.cuh"
#include "dimgroups.cuh"
#include "dim.cuh"
#include "finalize.cuh"
#include "groupdirect.cuh"
#include "multi.cuh"

namespace tqp {

tqp_status run_plan_one(tqp_ctx* ctx, const tqp_plan* p, const tqp_result* r, cudaStream_t stream);
bool lower_group_direct(const tqp_table* t, const GroupArgs& A, long long max_groups, GroupDirectArgs* D);

constexpr int kBatchTile = 1024;
constexpr int kBatchStages = 3;
constexpr int kJobFilter = 1, kJobGroup = 2, kJobJoin = 3, kJobMulti = 4;
constexpr int kKinds = 4;  // scan bodies: filter, group-by, joined aggregation, shared filter
constexpr int kFlatThreads = 256;
constexpr int kFillPer = 4096;  // 16-byte units per fill block
constexpr int kRowsPer = 2048;  // elements per block of the element-wise phases
constexpr int kFinSmemBytes = 2 * kSmallCap * (8 + 4);
constexpr int kCounterBytes = 64;

struct FillRange {
    uint4* ptr;
    long long n16;  // 16-byte units
    uint4 pattern;
    long long first_block;
};

struct BuildJob {
    JoinHT H{};
    uint32_t* next;
    const unsigned char* key_col;
    int32_t key_type;
    int32_t grouped;
    long long nrows;
    GroupSpec claim;
    DimCols D;
    uint32_t* dslot;
    uint32_t* slot2dense;
    uint32_t* dgs;
    unsigned long long* dkeys;
    unsigned long long* dacc;
    long long* d_n;
    long long row_block, num_block, slot_block;  // first block of this job in each phase
};

struct alignas(16) ScanJob {
    int32_t kind;
    int32_t pad;
    long long chunk_base;
    union U {
        FilterArgs f;
        GroupArgs g;
        PlanJoinArgs j;
        MultiArgs m;
    } u;
};
static_assert(sizeof(ScanJob) % 16 == 0, "ScanJob is copied in 16-byte units");

struct CompactJob {
    const uint32_t* mask;
    const uint32_t* block_tot;
    long long n;
    int32_t* row_ids;
    long long capacity;
    long long first_block;
};

struct FinJob {
    GroupSpec S;
    GroupOut O;
    int64_t* total_out;
};

struct TopJob {
    GroupSpec S;
    GroupOut O;
    int32_t k;
    int32_t rank_acc;
    TopBuf buf[2];
    TopBuf cand;
    TopSel* sel;
    unsigned long long* total;
    int64_t* total_out;
    long long first_block;  // level 0 of the tournament
    long long sel_block;    // first block in the radix-select passes
    long long sel_nblocks;
};

// The fold of a join that aggregated by join key first (blocks
// [first_block, first_block + nblocks) of its launch).
struct FoldJob {
    JoinHT H{};
    const unsigned char* dkey;
    int32_t dkey_type;
    int32_t nk;
    long long nd;
    const uint32_t* dgs;
    GroupSpec S;
    const unsigned long long* kacc;
    unsigned long long* acc;
    int64_t* d_num_joined;
    int64_t* d_sum;
    int32_t has_sum;
    int32_t pad;
    long long first_block, nblocks;
};
constexpr long long kFoldRowsPerBlock = 8 * kFoldThreads;

// A few-groups group-by run by the direct kernel: blocks [first_block,
// first_block + nblocks) of its launch, and of the key-range pass.
struct DirJob {
    GroupDirectArgs A;
    unsigned long long* kmeta;  // = A.kmeta (zeroed by the fill), written by the range pass
    long long first_block, nblocks;
    long long range_first, range_nblocks;
};
constexpr int kDirArgsBytes = (static_cast<int>(sizeof(GroupDirectArgs)) + 127) / 128 * 128;
constexpr long long kDirRowsPerBlock = 32768;    // direct kernel: 32 128-row steps per warp
constexpr long long kDirRangeRowsPerBlock = 65536;

struct TopItem {
    int32_t job;
    int32_t emit;
    int32_t in_buf;
    int32_t pad;
    long long n_in;
    long long first_block;
};

__global__ void __launch_bounds__(kFlatThreads) k_b_fill(const FillRange* R, const int32_t* bjob, int64_t* const* zero,
                                                         int nzero) {
    const FillRange& r = R[bjob[blockIdx.x]];
    const long long u0 = (static_cast<long long>(blockIdx.x) - r.first_block) * kFillPer;
    const long long u1 = (u0 + kFillPer < r.n16) ? u0 + kFillPer : r.n16;
    for (long long u = u0 + threadIdx.x; u < u1; u += kFlatThreads) r.ptr[u] = r.pattern;
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i < nzero; i += kFlatThreads) *zero[i] = 0;
}

__global__ void __launch_bounds__(kFlatThreads) k_b_range(const BuildJob* B, const int32_t* bjob) {
    const BuildJob& b = B[bjob[blockIdx.x]];
    const long long i0 = (static_cast<long long>(blockIdx.x) - b.row_block) * kRowsPer;
    const long long i1 = (i0 + kRowsPer < b.nrows) ? i0 + kRowsPer : b.nrows;
    ht_key_range(b.H, b.key_col, b.key_type, i0 + threadIdx.x, i1, kFlatThreads);
}

__global__ void __launch_bounds__(kFlatThreads) k_b_build(const BuildJob* B, const int32_t* bjob, int* err) {
    const BuildJob& b = B[bjob[blockIdx.x]];
    const long long i0 = (static_cast<long long>(blockIdx.x) - b.row_block) * kRowsPer;
    const long long i1 = (i0 + kRowsPer < b.nrows) ? i0 + kRowsPer : b.nrows;
    for (long long i = i0 + threadIdx.x; i < i1; i += kFlatThreads) {
        ht_chain_insert_row(b.H, b.key_col, b.key_type, i, b.next, err);
        if (b.grouped) dim_claim_row(b.claim, b.D, i, b.dslot, err);
    }
}

__global__ void __launch_bounds__(kNumberThreads) k_b_number(const BuildJob* B, const int32_t* bjob) {
    const BuildJob& b = B[bjob[blockIdx.x]];
    const long long s0 = (static_cast<long long>(blockIdx.x) - b.num_block) * kRowsPer;
    const long long s1 = (s0 + kRowsPer < b.claim.cap + 1) ? s0 + kRowsPer : b.claim.cap + 1;
    dense_number_range(b.claim, b.slot2dense, b.dkeys, b.dacc, b.d_n, s0, s1);
}

__global__ void __launch_bounds__(kFlatThreads) k_b_remap(const BuildJob* B, const int32_t* bjob) {
    const BuildJob& b = B[bjob[blockIdx.x]];
    if (!b.grouped) return;
    const long long i0 = (static_cast<long long>(blockIdx.x) - b.row_block) * kRowsPer;
    const long long i1 = (i0 + kRowsPer < b.nrows) ? i0 + kRowsPer : b.nrows;
    for (long long i = i0 + threadIdx.x; i < i1; i += kFlatThreads) b.dgs[i] = b.slot2dense[b.dslot[i]];
}

__global__ void __launch_bounds__(kFlatThreads) k_b_direct(const BuildJob* B, const int32_t* bjob) {
    const BuildJob& b = B[bjob[blockIdx.x]];
    const long long s0 = (static_cast<long long>(blockIdx.x) - b.slot_block) * kRowsPer;
    const long long s1 = (s0 + kRowsPer < b.H.cap + 1) ? s0 + kRowsPer : b.H.cap + 1;
    for (long long s = s0 + threadIdx.x; s < s1; s += kFlatThreads) ht_direct_slot(b.H, b.dgs, s);
}

template <class Body, class Args>
__device__ __forceinline__ void scan_chunk(const Args& a, unsigned char* body_smem, long long local, EngineHeader* h,
                                           unsigned char* stages, long long& it, bool& aborted, uint64_t policy,
                                           int warp, int lane) {
    Body body(a, body_smem);
    __syncthreads();
    const long long t0 = local * a.ctl.chunk_tiles;
    const long long t1 = (t0 + a.ctl.chunk_tiles < a.G.ntiles) ? t0 + a.ctl.chunk_tiles : a.G.ntiles;
    run_chunk(a.G, a.ctl, body, local, t0, t1, h, stages, it, aborted, policy, warp, lane);
}

template <class Body> struct BodyArgs;
template <> struct BodyArgs<FilterBody> {
    static __device__ __forceinline__ const FilterArgs& of(const ScanJob& j) { return j.u.f; }
};
template <> struct BodyArgs<GroupBody> {
    static __device__ __forceinline__ const GroupArgs& of(const ScanJob& j) { return j.u.g; }
};
template <> struct BodyArgs<PlanJoinBody> {
    static __device__ __forceinline__ const PlanJoinArgs& of(const ScanJob& j) { return j.u.j; }
};
template <> struct BodyArgs<MultiBody> {
    static __device__ __forceinline__ const MultiArgs& of(const ScanJob& j) { return j.u.m; }
};

constexpr int kJobBytes = (sizeof(ScanJob) + 127) / 128 * 128;
template <class Body>
constexpr int body_bytes() { return (Body::kSmemBytes + 127) / 128 * 128; }

// The persistent multi-plan scan of one body kind: chunk tickets span the
// tables of every job of that kind.
template <class Body>
__global__ void __launch_bounds__(kEngineThreads, Body::kMinBlocks) k_b_scan(const ScanJob* J, const int32_t* cjob,
                                                              unsigned long long* ticket, long long total_chunks) {
    extern __shared__ __align__(128) unsigned char smem[];
    EngineHeader* h = reinterpret_cast<EngineHeader*>(smem);
    ScanJob* sj = reinterpret_cast<ScanJob*>(smem + kHeaderBytes);
    unsigned char* body_smem = smem + kHeaderBytes + kJobBytes;
    unsigned char* stages = body_smem + body_bytes<Body>();
    __shared__ int job_sm;
    const int warp = threadIdx.x / kWarp;
    const int lane = threadIdx.x % kWarp;
    init_stage_ring(h, kBatchStages);
    __syncthreads();
    long long it = 0;
    bool aborted = false;
    const uint64_t policy = l2_evict_first_policy();
    while (true) {
        if (threadIdx.x == 0) {
            const long long c = static_cast<long long>(atomicAdd(ticket, 1ULL));
            h->chunk = c;
            job_sm = c < total_chunks ? cjob[c] : -1;
        }
        __syncthreads();
        const long long chunk = h->chunk;
        if (chunk >= total_chunks) break;
        {
            const uint4* src = reinterpret_cast<const uint4*>(&J[job_sm]);
            uint4* dst = reinterpret_cast<uint4*>(sj);
            for (int i = threadIdx.x; i < static_cast<int>(sizeof(ScanJob) / 16); i += kEngineThreads) dst[i] = src[i];
        }
        __syncthreads();
        const long long local = chunk - sj->chunk_base;
        scan_chunk<Body>(BodyArgs<Body>::of(*sj), body_smem, local, h, stages, it, aborted, policy, warp, lane);
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kCompactThreads) k_b_compact(const CompactJob* C, const int32_t* bjob) {
    const CompactJob& c = C[bjob[blockIdx.x]];
    compact_block(c.mask, c.block_tot, c.n, c.row_ids, c.capacity, static_cast<long long>(blockIdx.x) - c.first_block);
}

__global__ void __launch_bounds__(kFoldThreads) k_b_fold(const FoldJob* J, const int32_t* bjob) {
    const FoldJob& f = J[bjob[blockIdx.x]];
    keyfirst_fold_block(f.H, f.dkey, f.dkey_type, f.nd, f.dgs, f.S, f.kacc, f.nk, f.has_sum, f.acc, f.d_num_joined,
                        f.d_sum, static_cast<long long>(blockIdx.x) - f.first_block, f.nblocks);
}

__global__ void __launch_bounds__(kDirThreads) k_b_grange(const DirJob* J, const int32_t* bjob) {
    const DirJob& j = J[bjob[blockIdx.x]];
    group_direct_range_block(j.A, j.kmeta, nullptr, static_cast<long long>(blockIdx.x) - j.range_first,
                             j.range_nblocks);
}

// The job's arguments are copied into shared memory after the kernel's own
// layout, so the hot loop reads them with shared-memory loads.
__global__ void __launch_bounds__(kDirThreads, kDirMinBlocks) k_b_gdirect(const DirJob* J, const int32_t* bjob) {
    extern __shared__ __align__(16) unsigned char dsm[];
    const DirJob& j = J[bjob[blockIdx.x]];
    const GroupDirectArgs& A = stage_args(j.A, dsm + kDirSmemBytes);
    group_direct_block<false>(A, dsm, static_cast<long long>(blockIdx.x) - j.first_block, j.nblocks);
}

__global__ void __launch_bounds__(kFinThreads) k_b_finalize(const FinJob* F) {
    extern __shared__ __align__(16) unsigned char fsm[];
    const FinJob& f = F[blockIdx.x];
    finalize_small_block(f.S, f.O, fsm);
    __syncthreads();
    if (threadIdx.x == 0 && f.total_out) *f.total_out = *f.O.num_groups;
}

__global__ void __launch_bounds__(kTopThreads) k_b_topk0(const TopJob* T, const int32_t* bjob) {
    const TopJob& t = T[bjob[blockIdx.x]];
    topk_level0_block(t.S, t.rank_acc, t.k, t.buf[0], t.total, static_cast<long long>(blockIdx.x) - t.first_block,
                      &t.sel->fallback);
}

__global__ void __launch_bounds__(kTopThreads) k_b_topk(const TopJob* T, const TopItem* items, const int32_t* bjob) {
    const TopItem& it = items[bjob[blockIdx.x]];
    const TopJob& t = T[it.job];
    topk_reduce_block(t.S, t.buf[it.in_buf], it.n_in, t.k, t.buf[1 - it.in_buf], it.emit, t.O, t.total, t.total_out,
                      static_cast<long long>(blockIdx.x) - it.first_block, &t.sel->fallback);
}

__global__ void __launch_bounds__(kSelThreads) k_b_sel(const TopJob* T, const int32_t* bjob, int pass) {
    const TopJob& t = T[bjob[blockIdx.x]];
    topsel_pass_block(t.S, t.rank_acc, t.k, t.sel, pass, static_cast<long long>(blockIdx.x) - t.sel_block,
                      t.sel_nblocks);
}

__global__ void __launch_bounds__(kSelThreads) k_b_selcollect(const TopJob* T, const int32_t* bjob) {
    const TopJob& t = T[bjob[blockIdx.x]];
    topsel_collect_block(t.S, t.rank_acc, t.sel, t.cand, static_cast<long long>(blockIdx.x) - t.sel_block);
}

__global__ void __launch_bounds__(kTopThreads) k_b_selemit(const TopJob* T) {
    const TopJob& t = T[blockIdx.x];
    topsel_emit_block(t.S, t.k, t.sel, t.cand, t.O, t.total_out);
}

}  // namespace tqp

using namespace tqp;

struct tqp_batch {
    tqp_ctx* ctx = nullptr;
    bool persistent = false;  // scratch from the arena's long-lived top region
    int tile = tqp::kBatchTile;  // rows per tile of the scans (clamped per job to what fits)
    size_t top_before = 0;
    size_t top_after = 0;
    // lowered jobs
    std::vector<FillRange> fill;
    std::vector<int64_t*> zero;
    std::vector<BuildJob> build;
    std::vector<ScanJob> scan[kKinds];
    std::vector<CompactJob> compact;
    std::vector<FinJob> fin;
    std::vector<TopJob> top;
    std::vector<DirJob> gdir;
    std::vector<FoldJob> fold;
    std::vector<std::vector<TopItem>> levels;
    // block -> job maps, concatenated
    std::vector<int32_t> maps;
    long long fill_blocks = 0, row_blocks = 0, num_blocks = 0, slot_blocks = 0, compact_blocks = 0, top0_blocks = 0,
              sel_blocks = 0, grange_blocks = 0, gdirect_blocks = 0, fold_blocks = 0;
    long long scan_chunks[kKinds] = {0, 0, 0, 0};
    // lookup tables and outputs of the shared scans (one blob; per job its offset)
    std::vector<unsigned char> mblob;
    std::vector<size_t> mblob_off;
    unsigned char* d_mblob = nullptr;
    std::vector<long long> level_blocks;
    size_t off_fill = 0, off_row = 0, off_num = 0, off_slot = 0, off_compact = 0, off_top0 = 0, off_sel = 0,
           off_grange = 0, off_gdirect = 0, off_fold = 0;
    size_t off_scan[kKinds] = {0, 0, 0, 0};
    std::vector<size_t> off_level;
    // small zeroed counters share one slab (one fill range)
    unsigned char* slab = nullptr;
    size_t slab_bytes = 0, slab_used = 0;
    // device copies
    FillRange* d_fill = nullptr;
    int64_t** d_zero = nullptr;
    BuildJob* d_build = nullptr;
    ScanJob* d_scan[kKinds] = {nullptr, nullptr, nullptr, nullptr};
    CompactJob* d_compact = nullptr;
    FinJob* d_fin = nullptr;
    TopJob* d_top = nullptr;
    DirJob* d_gdir = nullptr;
    FoldJob* d_fold = nullptr;
    std::vector<TopItem*> d_levels;
    int32_t* d_maps = nullptr;
    unsigned long long* d_ticket[kKinds] = {nullptr, nullptr, nullptr, nullptr};
    size_t scan_smem[kKinds] = {0, 0, 0, 0};
    int scan_grid[kKinds] = {0, 0, 0, 0};
    // plans run through the single-plan path, and their scratch
    std::vector<tqp_plan> fb_plans;
    std::vector<tqp_result> fb_res;
    unsigned char* fb_arena = nullptr;
    size_t fb_bytes = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace tqp {

static void* balloc(tqp_batch* b, size_t bytes) {
    bytes = (bytes + 15) / 16 * 16;
    return b->persistent ? arena_alloc_top(b->ctx, bytes) : arena_alloc(b->ctx, bytes);
}

static void add_fill(tqp_batch* b, void* ptr, size_t bytes, uint4 pattern) {
    FillRange r;
    r.ptr = static_cast<uint4*>(ptr);
    r.n16 = static_cast<long long>((bytes + 15) / 16);
    r.pattern = pattern;
    r.first_block = 0;
    if (r.n16 > 0) b->fill.push_back(r);
}

static const uint4 kZero16 = {0u, 0u, 0u, 0u};
static const uint4 kOnes16 = {~0u, ~0u, ~0u, ~0u};

// A zeroed 64-byte counter block from the slab (sized for every job's needs).
static unsigned long long* counter(tqp_batch* b) {
    unsigned long long* p = reinterpret_cast<unsigned long long*>(b->slab + b->slab_used);
    b->slab_used += kCounterBytes;
    return p;
}

// Staged geometry of one scan in the batch: the batch's tile size (3 stages),
// halved until the stages fit beside the body of the job's kind.
static tqp_status batch_geom(const tqp_batch* b, const tqp_table* t, std::vector<int> staged, int body_bytes,
                             ScanGeom* G) {
    std::sort(staged.begin(), staged.end());
    staged.erase(std::unique(staged.begin(), staged.end()), staged.end());
    if (static_cast<int>(staged.size()) > kMaxStaged) staged.resize(kMaxStaged);
    int stage_row = 0;
    for (int c : staged) stage_row += t->cols[c].type == TQP_I64 ? 8 : (t->cols[c].type == TQP_I32 ? 4 : 1);
    const long long room = static_cast<long long>(b->ctx->smem_optin) - 1024 - kHeaderBytes - kJobBytes - body_bytes;
    int T = b->tile;
    while (T > kBatchTile && static_cast<long long>(kBatchStages) * (static_cast<long long>(T) * stage_row +
                                                                     128LL * kMaxStaged) > room)
        T /= 2;
    const tqp_tuning tu{T, kBatchStages, 2, 1};
    size_t smem = 0;
    return make_geom(b->ctx, t, staged, tu, 0, G, &smem);
}

static tqp_status add_filter_job(tqp_batch* b, const tqp_plan* p, const tqp_result* r, bool ids, bool with_sum,
                                 int64_t* d_count, int64_t* d_count2) {
    tqp_ctx* ctx = b->ctx;
    ScanJob J;
    memset(&J, 0, sizeof(J));
    J.kind = kJobFilter;
    FilterArgs& A = J.u.f;
    int ncond = 0;
    TQP_TRY(lower_preds(p->fact, p->preds, p->npreds, A.cond, &ncond));
    A.ncond = ncond;
    std::vector<int> staged;
    for (int i = 0; i < ncond; ++i) staged.push_back(A.cond[i].col);
    if (with_sum) {
        TQP_TRY(lower_expr(&p->sum_expr, p->fact->num_cols, &A.sum));
        A.has_sum = 1;
        if (ncond == 0) expr_cols(A.sum, staged);
    }
    TQP_TRY(batch_geom(b, p->fact, staged, body_bytes<FilterBody>(), &A.G));
    lower_fast(A.cond, A.ncond, A.G, A.cf, &A.fast);
    A.acc = counter(b);
    A.d_count = d_count;
    A.d_count2 = d_count2;
    A.d_sum = with_sum ? r->d_sum : nullptr;
    if (ids) {
        const long long nblocks = (A.G.n + kCompactRows - 1) / kCompactRows;
        const size_t tot_bytes = static_cast<size_t>(nblocks) * 4 + 16;
        const size_t mask_bytes = static_cast<size_t>(A.G.ntiles) * (A.G.T / kWarp) * 4;
        A.block_tot = static_cast<uint32_t*>(balloc(b, tot_bytes));
        A.mask = static_cast<uint32_t*>(balloc(b, mask_bytes + 16));
        if (!A.block_tot || !A.mask) return arena_oom(ctx, tot_bytes + mask_bytes);
        add_fill(b, A.block_tot, tot_bytes, kZero16);
        A.capacity = r->capacity_rows;
        if (nblocks > 0) {
            CompactJob C{A.mask, A.block_tot, A.G.n, r->d_row_ids, r->capacity_rows, b->compact_blocks};
            b->compact_blocks += nblocks;
            b->compact.push_back(C);
        }
    }
    A.ctl.err = ctx->d_err;
    A.ctl.wait_cap = ctx->wait_cap;
    if (A.G.ntiles == 0) {  // nothing is scanned: the results of an empty table
        b->zero.push_back(d_count);
        if (d_count2) b->zero.push_back(d_count2);
        if (A.d_sum) b->zero.push_back(A.d_sum);
        return TQP_OK;
    }
    b->scan[kJobFilter - 1].push_back(J);
    return TQP_OK;
}

static tqp_status add_top_job(tqp_batch* b, const GroupSpec& S, const GroupOut& O, const tqp_plan* p,
                              const tqp_result* r) {
    TopJob T;
    memset(&T, 0, sizeof(T));
    T.S = S;
    T.O = O;
    T.k = p->topk;
    T.rank_acc = S.agg_acc[p->topk_agg];
    const long long nb0 = (S.cap + 1 + kTopBlock - 1) / kTopBlock;
    for (int q = 0; q < 2; ++q) {
        const size_t n = static_cast<size_t>(nb0) * T.k;
        T.buf[q].rank = static_cast<long long*>(balloc(b, n * 8));
        T.buf[q].key = static_cast<uint64_t*>(balloc(b, n * 8));
        T.buf[q].slot = static_cast<uint32_t*>(balloc(b, n * 4));
        if (!T.buf[q].rank || !T.buf[q].key || !T.buf[q].slot) return arena_oom(b->ctx, n * 20);
    }
    T.cand.rank = static_cast<long long*>(balloc(b, kSelCand * 8));
    T.cand.key = static_cast<uint64_t*>(balloc(b, kSelCand * 8));
    T.cand.slot = static_cast<uint32_t*>(balloc(b, kSelCand * 4));
    T.sel = static_cast<TopSel*>(balloc(b, sizeof(TopSel)));
    if (!T.cand.rank || !T.cand.key || !T.cand.slot || !T.sel) return arena_oom(b->ctx, sizeof(TopSel) + kSelCand * 20);
    add_fill(b, T.sel, sizeof(TopSel), kZero16);
    T.total = counter(b);
    T.total_out = r->d_total_groups;
    T.first_block = b->top0_blocks;
    b->top0_blocks += nb0;
    T.sel_nblocks = (S.cap + 1 + kSelSlots - 1) / kSelSlots;
    T.sel_block = b->sel_blocks;
    b->sel_blocks += T.sel_nblocks;
    b->top.push_back(T);
    return TQP_OK;
}

static tqp_status add_group_job(tqp_batch* b, const tqp_plan* p, const tqp_result* r) {
    tqp_ctx* ctx = b->ctx;
    const tqp_table* t = p->fact;
    ScanJob J;
    memset(&J, 0, sizeof(J));
    J.kind = kJobGroup;
    GroupArgs& A = J.u.g;
    int ncond = 0;
    TQP_TRY(lower_preds(t, p->preds, p->npreds, A.cond, &ncond));
    A.ncond = ncond;
    int32_t types[TQP_MAX_GROUP_COLS] = {0, 0, 0, 0};
    for (int i = 0; i < p->ngc; ++i) types[i] = t->cols[p->group_cols[i]].type;
    TQP_TRY(lower_group(p->group_cols, types, p->ngc, p->aggs, p->naggs, t->num_cols, &A.S));
    std::vector<int> staged;
    for (int i = 0; i < ncond; ++i) staged.push_back(A.cond[i].col);
    for (int i = 0; i < p->ngc; ++i) staged.push_back(p->group_cols[i]);
    for (int a = 1; a < A.S.nacc; ++a) expr_cols(A.S.acc_expr[a - 1], staged);
    TQP_TRY(batch_geom(b, t, staged, body_bytes<GroupBody>(), &A.G));
    lower_fast(A.cond, A.ncond, A.G, A.cf, &A.fast);
    lower_group_fast(&A);
    const long long maxg = p->max_groups > 0 ? p->max_groups : std::max<long long>(1, r->capacity_groups);
    const long long cap = group_table_cap(maxg);
    A.S.cap = cap;
    A.S.max_groups = maxg;
    const size_t key_bytes = static_cast<size_t>(cap + 1) * 8;
    const size_t acc_bytes = static_cast<size_t>(cap + 1) * A.S.nacc * 8;
    A.S.keys = static_cast<unsigned long long*>(balloc(b, key_bytes));
    A.S.acc = static_cast<unsigned long long*>(balloc(b, acc_bytes));
    A.S.ndistinct = counter(b);
    if (!A.S.keys || !A.S.acc) return arena_oom(ctx, key_bytes + acc_bytes);
    add_fill(b, A.S.keys, key_bytes, kOnes16);
    add_fill(b, A.S.acc, acc_bytes, kZero16);
    A.ctl.err = ctx->d_err;
    A.ctl.wait_cap = ctx->wait_cap;
    const GroupOut O{r->d_keys, r->d_ivals, r->d_fvals, r->capacity_groups, r->d_num_groups, ctx->d_err};
    if (p->topk > 0) {
        TQP_TRY(add_top_job(b, A.S, O, p, r));
    } else {
        FinJob F;
        memset(&F, 0, sizeof(F));
        F.S = A.S;
        F.O = O;
        F.total_out = r->d_total_groups;
        b->fin.push_back(F);
    }
    DirJob D;
    memset(&D, 0, sizeof(D));
    if (lower_group_direct(t, A, maxg, &D.A)) {
        D.A.S = A.S;
        D.A.err = ctx->d_err;
        if (D.A.ngc > 0) {
            D.kmeta = counter(b);
            D.A.kmeta = D.kmeta;
            D.range_first = b->grange_blocks;
            D.range_nblocks = (t->num_rows + kDirRangeRowsPerBlock - 1) / kDirRangeRowsPerBlock;
            b->grange_blocks += D.range_nblocks;
        }
        D.first_block = b->gdirect_blocks;
        D.nblocks = (t->num_rows + kDirRowsPerBlock - 1) / kDirRowsPerBlock;
        b->gdirect_blocks += D.nblocks;
        b->gdir.push_back(D);
        return TQP_OK;
    }
    if (A.G.ntiles > 0) b->scan[kJobGroup - 1].push_back(J);
    return TQP_OK;
}

static tqp_status add_join_job(tqp_batch* b, const tqp_plan* p, const tqp_result* r) {
    tqp_ctx* ctx = b->ctx;
    const tqp_table* F = p->fact;
    const tqp_table* D = p->dim;
    const tqp_dim* pd = p->prepared;
    const int nf = F->num_cols, nd = D->num_cols;
    const long long ndr = D->num_rows;
    const size_t nd_rows = static_cast<size_t>(std::max<long long>(1, ndr));
    // build side: the chained table, and the dimension rows' dense group ids
    // (a prepared dimension has both resident)
    BuildJob B;
    memset(&B, 0, sizeof(B));
    if (pd) {
        B.H = pd->H;
        B.next = pd->next;
    } else {
        B.H.cap = ht_cap_dense(ndr);
        B.H.slots = static_cast<uint4*>(balloc(b, static_cast<size_t>(B.H.cap + 1) * 16));
        B.next = static_cast<uint32_t*>(balloc(b, nd_rows * 4));
        if (!B.H.slots || !B.next) return arena_oom(ctx, static_cast<size_t>(B.H.cap + 1) * 16 + nd_rows * 4);
        add_fill(b, B.H.slots, static_cast<size_t>(B.H.cap + 1) * 16, uint4{~0u, ~0u, kNoRow, 0u});
        long long* meta = static_cast<long long*>(balloc(b, 16));
        if (!meta) return arena_oom(ctx, 16);
        add_fill(b, meta, 16, uint4{~0u, 0x7FFFFFFFu, 0u, 0x80000000u});  // min = INT64_MAX, max = INT64_MIN
        B.H.meta = meta;
        B.key_col = static_cast<const unsigned char*>(D->cols[p->dim_key].data);
        B.key_type = D->cols[p->dim_key].type;
        B.nrows = ndr;
        for (int c = 0; c < nd; ++c) {
            B.D.ptr[c] = static_cast<const unsigned char*>(D->cols[c].data);
            B.D.type[c] = D->cols[c].type;
        }
    }
    // probe side: filter + probe + aggregate, one fused scan body
    ScanJob J;
    memset(&J, 0, sizeof(J));
    J.kind = kJobJoin;
    PlanJoinArgs& A = J.u.j;
    int ncond = 0;
    TQP_TRY(lower_preds(F, p->preds, p->npreds, A.cond, &ncond));
    A.ncond = ncond;
    A.fk_col = p->fact_fk;
    A.H = B.H;
    A.next = B.next;
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
        if (pd) {
            const size_t acc_bytes = static_cast<size_t>(pd->groups + 1) * A.S.nacc * 8;
            unsigned long long* dacc = static_cast<unsigned long long*>(balloc(b, acc_bytes));
            if (!dacc) return arena_oom(ctx, acc_bytes);
            add_fill(b, dacc, acc_bytes, kZero16);
            A.S.keys = pd->dkeys;
            A.S.acc = dacc;
            A.S.cap = pd->groups;
            A.S.max_groups = pd->groups;
            A.S.ndistinct = reinterpret_cast<unsigned long long*>(pd->d_groups);
            A.S.d_dense_n = pd->d_groups;
            A.dgs = pd->dgs;
        } else {
            const long long maxg =
                p->max_groups > 0 ? p->max_groups : (p->ngc == 0 ? 1 : std::max<long long>(1, ndr));
            const long long cap = group_table_cap(maxg);
            const long long dmax = std::min<long long>(maxg, cap + 1);
            B.grouped = 1;
            B.claim = A.S;
            B.claim.cap = cap;
            B.claim.max_groups = maxg;
            B.claim.keys = static_cast<unsigned long long*>(balloc(b, static_cast<size_t>(cap + 1) * 8));
            B.claim.ndistinct = counter(b);
            B.d_n = reinterpret_cast<long long*>(B.claim.ndistinct) + 1;
            B.slot2dense = static_cast<uint32_t*>(balloc(b, static_cast<size_t>(cap + 1) * 4));
            B.dslot = static_cast<uint32_t*>(balloc(b, nd_rows * 4));
            B.dgs = static_cast<uint32_t*>(balloc(b, nd_rows * 4));
            B.dkeys = static_cast<unsigned long long*>(balloc(b, static_cast<size_t>(dmax + 1) * 8));
            B.dacc = static_cast<unsigned long long*>(balloc(b, static_cast<size_t>(dmax + 1) * A.S.nacc * 8));
            if (!B.claim.keys || !B.slot2dense || !B.dslot || !B.dgs || !B.dkeys || !B.dacc)
                return arena_oom(ctx, static_cast<size_t>(cap) * 12 + static_cast<size_t>(dmax) * (8 + 8 * A.S.nacc));
            add_fill(b, B.claim.keys, static_cast<size_t>(cap + 1) * 8, kOnes16);
            // the aggregation state in dense form: entries [0, *d_n)
            A.S.keys = B.dkeys;
            A.S.acc = B.dacc;
            A.S.cap = dmax;
            A.S.max_groups = maxg;
            A.S.ndistinct = reinterpret_cast<unsigned long long*>(B.d_n);
            A.S.d_dense_n = B.d_n;
            A.dgs = B.dgs;
        }
        const GroupOut O{r->d_keys, r->d_ivals, r->d_fvals, r->capacity_groups, r->d_num_groups, ctx->d_err};
        if (p->topk > 0) {
            TQP_TRY(add_top_job(b, A.S, O, p, r));
        } else {
            FinJob Fj;
            memset(&Fj, 0, sizeof(Fj));
            Fj.S = A.S;
            Fj.O = O;
            Fj.total_out = r->d_total_groups;
            b->fin.push_back(Fj);
        }
    }
    if (!pd) {
        B.row_block = b->row_blocks;
        b->row_blocks += (ndr + kRowsPer - 1) / kRowsPer;
        if (B.grouped) {
            B.num_block = b->num_blocks;
            b->num_blocks += (B.claim.cap + 1 + kRowsPer - 1) / kRowsPer;
            B.slot_block = b->slot_blocks;
            b->slot_blocks += (B.H.cap + 1 + kRowsPer - 1) / kRowsPer;
        }
        b->build.push_back(B);
    }
    std::vector<int> staged;
    for (int i = 0; i < ncond; ++i) staged.push_back(A.cond[i].col);
    staged.push_back(p->fact_fk);
    if (A.has_sum) expr_cols(A.sum, staged);
    for (int a = 1; a < A.S.nacc; ++a) expr_cols(A.S.acc_expr[a - 1], staged);
    TQP_TRY(batch_geom(b, F, staged, body_bytes<PlanJoinBody>(), &A.G));
    lower_fast(A.cond, A.ncond, A.G, A.cf, &A.fast);
    lower_join_fast(&A);
    A.acc = counter(b);
    A.d_num_joined = r->d_num_joined;
    A.d_sum = p->has_sum ? r->d_sum : nullptr;
    A.d_num_rows = (p->emit_row_ids && r->d_row_ids) ? nullptr : r->d_num_rows;
    A.ctl.err = ctx->d_err;
    A.ctl.wait_cap = ctx->wait_cap;
    // aggregation by join key first (used on the device only if the table is
    // direct-mapped), as in the single-plan path
    if (grouped && A.pjfast && A.fast && A.H.meta && A.G.ntiles > 0 && F->num_rows >= 2 * std::max<long long>(1, ndr)) {
        A.nk = A.S.nacc + (A.has_sum ? 1 : 0);
        const size_t kbytes = static_cast<size_t>(A.H.cap) * A.nk * 8;
        A.kacc = static_cast<unsigned long long*>(balloc(b, kbytes));
        if (!A.kacc) return arena_oom(ctx, kbytes);
        add_fill(b, A.kacc, kbytes, kZero16);
        FoldJob Fo;
        memset(&Fo, 0, sizeof(Fo));
        Fo.H = A.H;
        Fo.dkey = static_cast<const unsigned char*>(D->cols[p->dim_key].data);
        Fo.dkey_type = D->cols[p->dim_key].type;
        Fo.nk = A.nk;
        Fo.nd = ndr;
        Fo.dgs = A.dgs;
        Fo.S = A.S;
        Fo.kacc = A.kacc;
        Fo.acc = A.acc;
        Fo.d_num_joined = A.d_num_joined;
        Fo.d_sum = A.d_sum;
        Fo.has_sum = A.has_sum;
        Fo.first_block = b->fold_blocks;
        Fo.nblocks = std::max<long long>(1, (ndr + kFoldRowsPerBlock - 1) / kFoldRowsPerBlock);
        b->fold_blocks += Fo.nblocks;
        b->fold.push_back(Fo);
    }
    if (A.G.ntiles > 0) {
        b->scan[kJobJoin - 1].push_back(J);
    } else {
        if (A.d_num_joined) b->zero.push_back(A.d_num_joined);
        if (A.d_sum) b->zero.push_back(A.d_sum);
        if (A.d_num_rows) b->zero.push_back(A.d_num_rows);
    }
    if (p->emit_row_ids && r->d_row_ids) TQP_TRY(add_filter_job(b, p, r, true, false, r->d_num_rows, nullptr));
    return TQP_OK;
}

static bool expr_in(const tqp_expr& e, int lo, int hi) {
    for (int i = 0; i < e.n && i < TQP_MAX_EXPR; ++i)
        if (e.op[i] == TQP_X_COL && (e.v[i] < lo || e.v[i] >= hi)) return false;
    return true;
}

// Plans the batch lowers itself; the rest (including every malformed plan,
// which then reports its error) take the single-plan path.
// (every column of its tables in device memory: host columns, allowed in one
// place only, go through the single-plan path and its checks)
static bool all_device(const tqp_table* t) {
    std::vector<int> cols;
    for (int c = 0; c < t->num_cols; ++c) cols.push_back(c);
    const bool ok = check_device_cols(t, cols, "batch") == TQP_OK;
    clear_error();
    return ok;
}

static bool has_strings(const tqp_table* t) {
    for (int c = 0; c < t->num_cols && t->cols; ++c)
        if (t->cols[c].type == TQP_CHAR) return true;
    return false;
}

static bool batchable(const tqp_ctx* ctx, const tqp_plan* p, const tqp_result* r) {
    if (!p->fact || p->npreds < 0 || p->npreds > TQP_MAX_PREDS) return false;
    // IN / LIKE and string columns: the single-plan path (its pre-pass)
    if (has_strings(p->fact) || (p->dim && has_strings(p->dim)) || has_set_preds(p->fact, p->preds, p->npreds))
        return false;
    if (p->dim && p->join_kind != TQP_JOIN_INNER) return false;  // semi / anti plans: the single-plan path
    if (p->ngc < 0 || p->ngc > TQP_MAX_GROUP_COLS || p->naggs < 0 || p->naggs > TQP_MAX_AGGS) return false;
    if (p->topk < 0 || p->topk > kTopBlock / 2) return false;
    const bool grouped = p->ngc > 0 || p->naggs > 0;
    if (grouped && (!r->d_num_groups || r->capacity_groups < 1)) return false;
    if (grouped && p->topk > 0 && (p->topk_agg < 0 || p->topk_agg >= p->naggs)) return false;
    const int nf = p->fact->num_cols;
    for (int a = 0; a < p->naggs; ++a) {
        if (p->aggs[a].fn == TQP_AVG && !r->d_fvals) return false;
        if (p->aggs[a].fn == TQP_MIN || p->aggs[a].fn == TQP_MAX) return false;  // the single-plan path has them
    }
    if (p->emit_row_ids && r->d_row_ids && !r->d_num_rows) return false;
    if (!p->dim) {
        for (int i = 0; i < p->ngc; ++i)
            if (p->group_cols[i] < 0 || p->group_cols[i] >= nf) return false;
        if (!grouped || p->topk > 0) return true;
        const long long maxg = p->max_groups > 0 ? p->max_groups : std::max<long long>(1, r->capacity_groups);
        return group_table_cap(maxg) <= kSmallCap;
    }
    const int nd = p->dim->num_cols;
    if (p->fact_fk < 0 || p->fact_fk >= nf || p->dim_key < 0 || p->dim_key >= nd) return false;
    for (int i = 0; i < p->ngc; ++i)
        if (p->group_cols[i] < nf || p->group_cols[i] >= nf + nd) return false;
    for (int a = 0; a < p->naggs; ++a)
        if (p->aggs[a].fn != TQP_COUNT && !expr_in(p->aggs[a].expr, 0, nf)) return false;
    if (p->has_sum && !expr_in(p->sum_expr, 0, nf)) return false;
    if (p->prepared) {
        if (check_prepared(ctx, p) != TQP_OK) return false;  // the single-plan path reports it
        return !(grouped && p->topk == 0 && p->prepared->groups > kSmallCap);
    }
    if (grouped && p->topk == 0) {
        const long long ndr = p->dim->num_rows;
        const long long maxg = p->max_groups > 0 ? p->max_groups : (p->ngc == 0 ? 1 : std::max<long long>(1, ndr));
        if (std::min<long long>(maxg, group_table_cap(maxg) + 1) > kSmallCap) return false;
    }
    return true;
}

// Filter-only work of one plan (counts and sum, no row ids): a candidate for a
// shared scan.
struct SharedCand {
    const tqp_plan* p;
    const tqp_result* r;
    bool sum;
    int64_t* cnt;
    int64_t* cnt2;
};

static bool same_table(const tqp_table* a, const tqp_table* b) {
    if (a == b) return true;
    if (a->num_rows != b->num_rows || a->num_cols != b->num_cols) return false;
    for (int c = 0; c < a->num_cols; ++c)
        if (a->cols[c].data != b->cols[c].data || a->cols[c].type != b->cols[c].type) return false;
    return true;
}

// One shared scan of `members` (indices into qs) over table t.
static tqp_status add_multi_job(tqp_batch* b, const tqp_table* t, const std::vector<MqQuery>& qs,
                                const std::vector<int>& members) {
    tqp_ctx* ctx = b->ctx;
    // the batch's tile size, halved until the stages fit beside the tables
    std::vector<int> cols;
    for (int m : members) cols.insert(cols.end(), qs[m].cols.begin(), qs[m].cols.end());
    std::sort(cols.begin(), cols.end());
    cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
    int stage_row = 0;
    for (int c : cols) stage_row += t->cols[c].type == TQP_I64 ? 8 : (t->cols[c].type == TQP_I32 ? 4 : 1);
    const long long room =
        static_cast<long long>(ctx->smem_optin) - 1024 - kHeaderBytes - kJobBytes - body_bytes<MultiBody>();
    int T = b->tile;
    while (T > kBatchTile &&
           static_cast<long long>(kBatchStages) * (static_cast<long long>(T) * stage_row + 128LL * kMaxStaged) > room)
        T /= 2;
    const tqp_tuning tu{T, kBatchStages, 2, 1};
    ScanJob J;
    memset(&J, 0, sizeof(J));
    J.kind = kJobMulti;
    MultiArgs& A = J.u.m;
    std::vector<unsigned char> blob;
    size_t smem = 0;
    int per_sm = 0;
    TQP_TRY(mq_lower_group(ctx, t, qs, members, &tu, kJobBytes, true, &A, &blob, &smem, &per_sm));
    if (A.G.ntiles == 0) {  // an empty table: every output is zero
        for (int m : members) {
            const MqOut& o = qs[m].out;
            for (int64_t* z : {o.count, o.count2, o.sum})
                if (z) b->zero.push_back(z);
        }
        return TQP_OK;
    }
    const size_t acc_bytes = (2 * kMqMax + 2) * sizeof(unsigned long long);
    A.acc = static_cast<unsigned long long*>(balloc(b, acc_bytes));
    if (!A.acc) return arena_oom(ctx, acc_bytes);
    add_fill(b, A.acc, acc_bytes, kZero16);
    A.ctl.err = ctx->d_err;
    A.ctl.wait_cap = ctx->wait_cap;
    const size_t off = (b->mblob.size() + 15) / 16 * 16;
    b->mblob.resize(off + blob.size());
    memcpy(b->mblob.data() + off, blob.data(), blob.size());
    b->mblob_off.push_back(off);
    b->scan[kJobMulti - 1].push_back(J);
    return TQP_OK;
}

// Pack the filter-only work of plans over the same table into shared scans;
// a plan alone on its table, or one that fits no pack, keeps its own filter
// scan.
static tqp_status add_shared_jobs(tqp_batch* b, const std::vector<SharedCand>& cands) {
    std::vector<bool> done(cands.size(), false);
    for (size_t i = 0; i < cands.size(); ++i) {
        if (done[i]) continue;
        std::vector<size_t> same;
        for (size_t j = i; j < cands.size(); ++j)
            if (!done[j] && same_table(cands[i].p->fact, cands[j].p->fact)) {
                same.push_back(j);
                done[j] = true;
            }
        auto single = [&](size_t k) {
            const SharedCand& c = cands[k];
            return add_filter_job(b, c.p, c.r, false, c.sum, c.cnt, c.cnt2);
        };
        if (same.size() == 1) {
            TQP_TRY(single(same[0]));
            continue;
        }
        const tqp_table* t = cands[i].p->fact;
        std::vector<MqQuery> qs(same.size());
        for (size_t k = 0; k < same.size(); ++k) {
            const SharedCand& c = cands[same[k]];
            TQP_TRY(mq_lower_query(t, c.p->preds, c.p->npreds, c.sum ? &c.p->sum_expr : nullptr, &qs[k]));
            qs[k].out.count = c.cnt;
            qs[k].out.count2 = c.cnt2;
            qs[k].out.sum = c.sum ? c.r->d_sum : nullptr;
            qs[k].out.rlo = 0;
            qs[k].out.rhi = t->num_rows;
        }
        std::vector<std::vector<int>> groups;
        std::vector<int> singles;
        mq_pack(t, qs, &groups, &singles);
        for (int k : singles) TQP_TRY(single(same[k]));
        for (const auto& g : groups) {
            if (g.size() == 1) TQP_TRY(single(same[g[0]]));
            else TQP_TRY(add_multi_job(b, t, qs, g));
        }
    }
    return TQP_OK;
}

static tqp_status lower_batch(tqp_batch* b, const tqp_plan* plans, const tqp_result* res, int32_t n) {
    // per plan at most 6 counters (group table, key ranges, top-k, filter, a
    // count, spare) and the tickets
    b->slab_bytes = static_cast<size_t>(kCounterBytes) * (6 * static_cast<size_t>(n) + kKinds + 1);
    b->slab = static_cast<unsigned char*>(balloc(b, b->slab_bytes));
    if (!b->slab) return arena_oom(b->ctx, b->slab_bytes);
    add_fill(b, b->slab, b->slab_bytes, kZero16);
    for (int k = 0; k < kKinds; ++k) b->d_ticket[k] = counter(b);
    std::vector<SharedCand> shared;
    for (int32_t i = 0; i < n; ++i) {
        const tqp_plan* p = &plans[i];
        const tqp_result* r = &res[i];
        if (!batchable(b->ctx, p, r) || check_table(p->fact, "plan.fact") != TQP_OK ||
            (p->dim && check_table(p->dim, "plan.dim") != TQP_OK) || !all_device(p->fact) ||
            (p->dim && !all_device(p->dim))) {
            clear_error();
            b->fb_plans.push_back(*p);
            b->fb_res.push_back(*r);
            continue;
        }
        if (p->dim) {
            TQP_TRY(add_join_job(b, p, r));
            continue;
        }
        const bool grouped = p->ngc > 0 || p->naggs > 0;
        const bool ids = p->emit_row_ids && r->d_row_ids;
        const bool sum = p->has_sum && r->d_sum;
        int64_t* cnt = r->d_num_rows ? r->d_num_rows : r->d_num_joined;
        int64_t* cnt2 = r->d_num_rows ? r->d_num_joined : nullptr;
        if (grouped) TQP_TRY(add_group_job(b, p, r));
        if (ids || sum || cnt) {
            if (!cnt) cnt = reinterpret_cast<int64_t*>(counter(b));
            if (ids) TQP_TRY(add_filter_job(b, p, r, ids, sum, cnt, cnt2));
            else shared.push_back(SharedCand{p, r, sum, cnt, cnt2});
        }
    }
    return add_shared_jobs(b, shared);
}

static const ScanGeom& job_geom(const ScanJob& j) {
    return j.kind == kJobFilter ? j.u.f.G : j.kind == kJobGroup ? j.u.g.G : j.kind == kJobJoin ? j.u.j.G : j.u.m.G;
}
static long long job_tiles(const ScanJob& j) { return job_geom(j).ntiles; }
static EngineCtl& job_ctl(ScanJob& j) {
    return j.kind == kJobFilter ? j.u.f.ctl : j.kind == kJobGroup ? j.u.g.ctl : j.kind == kJobJoin ? j.u.j.ctl : j.u.m.ctl;
}
static int job_stage_bytes(const ScanJob& j) { return job_geom(j).stage_bytes; }

// Chunks of equal size across the jobs of one kind (a job's last chunk may be
// short): about four per persistent CTA, so that the uneven tails of the
// largest tables still balance while each chunk amortises its pipeline fill.
static void assign_chunks(tqp_batch* b, int k) {
    long long tiles = 0;
    for (auto& j : b->scan[k]) tiles += job_tiles(j);
    const long long target = std::max<long long>(1, static_cast<long long>(b->scan_grid[k]) * 4);
    const long long ct = std::max<long long>(8, (tiles + target - 1) / target);
    long long base = 0;
    for (auto& j : b->scan[k]) {
        EngineCtl& ctl = job_ctl(j);
        ctl.chunk_tiles = ct;
        ctl.nchunks = (job_tiles(j) + ct - 1) / ct;
        ctl.ticket = nullptr;
        j.chunk_base = base;
        base += ctl.nchunks;
    }
    b->scan_chunks[k] = base;
}

// Top-k reduction levels: each level cuts every unfinished job's candidates
// by kTopBlock / k; a job whose candidates fit one block emits in that level.
static void plan_top_levels(tqp_batch* b) {
    const size_t nt = b->top.size();
    std::vector<long long> n(nt);
    std::vector<int> buf(nt, 0);
    std::vector<bool> done(nt, false);
    for (size_t j = 0; j < nt; ++j) {
        const long long nb0 = (j + 1 < nt ? b->top[j + 1].first_block : b->top0_blocks) - b->top[j].first_block;
        n[j] = nb0 * b->top[j].k;
    }
    while (true) {
        std::vector<TopItem> items;
        long long blocks = 0;
        for (size_t j = 0; j < nt; ++j) {
            if (done[j]) continue;
            TopItem it;
            memset(&it, 0, sizeof(it));
            it.job = static_cast<int32_t>(j);
            it.in_buf = buf[j];
            it.n_in = n[j];
            it.first_block = blocks;
            if (n[j] <= kTopBlock) {
                it.emit = 1;
                blocks += 1;
                done[j] = true;
            } else {
                const long long nb = (n[j] + kTopBlock - 1) / kTopBlock;
                blocks += nb;
                n[j] = nb * b->top[j].k;
                buf[j] ^= 1;
            }
            items.push_back(it);
        }
        if (items.empty()) break;
        b->levels.push_back(items);
        b->level_blocks.push_back(blocks);
    }
}

// Block -> job maps of every flattened phase, in one array.
static void build_maps(tqp_batch* b) {
    auto& M = b->maps;
    auto push = [&M](size_t j, long long nblocks) {
        for (long long k = 0; k < nblocks; ++k) M.push_back(static_cast<int32_t>(j));
    };
    b->off_fill = M.size();
    for (size_t r = 0; r < b->fill.size(); ++r) {
        b->fill[r].first_block = static_cast<long long>(M.size() - b->off_fill);
        push(r, (b->fill[r].n16 + kFillPer - 1) / kFillPer);
    }
    b->fill_blocks = static_cast<long long>(M.size() - b->off_fill);
    b->off_row = M.size();
    for (size_t j = 0; j < b->build.size(); ++j) push(j, (b->build[j].nrows + kRowsPer - 1) / kRowsPer);
    b->off_num = M.size();
    for (size_t j = 0; j < b->build.size(); ++j)
        if (b->build[j].grouped) push(j, (b->build[j].claim.cap + 1 + kRowsPer - 1) / kRowsPer);
    b->off_slot = M.size();
    for (size_t j = 0; j < b->build.size(); ++j)
        if (b->build[j].grouped) push(j, (b->build[j].H.cap + 1 + kRowsPer - 1) / kRowsPer);
    for (int k = 0; k < kKinds; ++k) {
        b->off_scan[k] = M.size();
        for (size_t j = 0; j < b->scan[k].size(); ++j) push(j, job_ctl(b->scan[k][j]).nchunks);
    }
    b->off_grange = M.size();
    for (size_t j = 0; j < b->gdir.size(); ++j) push(j, b->gdir[j].range_nblocks);
    b->off_gdirect = M.size();
    for (size_t j = 0; j < b->gdir.size(); ++j) push(j, b->gdir[j].nblocks);
    b->off_fold = M.size();
    for (size_t j = 0; j < b->fold.size(); ++j) push(j, b->fold[j].nblocks);
    b->off_compact = M.size();
    for (size_t j = 0; j < b->compact.size(); ++j) push(j, (b->compact[j].n + kCompactRows - 1) / kCompactRows);
    b->off_sel = M.size();
    for (size_t j = 0; j < b->top.size(); ++j) push(j, b->top[j].sel_nblocks);
    b->off_top0 = M.size();
    for (size_t j = 0; j < b->top.size(); ++j)
        push(j, (j + 1 < b->top.size() ? b->top[j + 1].first_block : b->top0_blocks) - b->top[j].first_block);
    for (size_t L = 0; L < b->levels.size(); ++L) {
        b->off_level.push_back(M.size());
        const auto& items = b->levels[L];
        for (size_t i = 0; i < items.size(); ++i)
            push(i, items[i].emit ? 1 : (items[i].n_in + kTopBlock - 1) / kTopBlock);
    }
}

// Descriptor upload: synchronous for a long-lived batch (before any run),
// stream-ordered for a one-shot batch (earlier work on the stream may still
// read the per-call scratch).
template <class T>
static tqp_status upload(tqp_batch* b, const std::vector<T>& v, T** out, cudaStream_t st) {
    *out = nullptr;
    if (v.empty()) return TQP_OK;
    *out = static_cast<T*>(balloc(b, v.size() * sizeof(T)));
    if (!*out) return arena_oom(b->ctx, v.size() * sizeof(T));
    if (b->persistent) TQP_CUDA(cudaMemcpy(*out, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    else TQP_CUDA(cudaMemcpyAsync(*out, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
    return TQP_OK;
}

// The single-plan path for the plans the batch does not lower, with scratch
// [base, base + bytes) of their own (they run one after another and share it).
static tqp_status run_fallbacks(tqp_batch* b, cudaStream_t st, unsigned char* base, size_t bytes, size_t* need) {
    tqp_ctx sub = *b->ctx;
    sub.arena = base;
    sub.arena_bytes = bytes;
    sub.used = kPersistentBytes;
    sub.top = bytes;
    for (size_t i = 0; i < b->fb_plans.size(); ++i) {
        const tqp_status s = run_plan_one(&sub, &b->fb_plans[i], &b->fb_res[i], st);
        if (need) *need = std::max(*need, sub.used);
        if (s != TQP_OK) return s;
    }
    return TQP_OK;
}

static tqp_status batch_launch(tqp_batch* b, cudaStream_t st) {
    tqp_ctx* ctx = b->ctx;
    const int32_t* M = b->d_maps;
    if (b->fill_blocks)
        k_b_fill<<<static_cast<unsigned>(b->fill_blocks), kFlatThreads, 0, st>>>(b->d_fill, M + b->off_fill, b->d_zero,
                                                                                 static_cast<int>(b->zero.size()));
    if (b->row_blocks)
        k_b_range<<<static_cast<unsigned>(b->row_blocks), kFlatThreads, 0, st>>>(b->d_build, M + b->off_row);
    if (b->row_blocks)
        k_b_build<<<static_cast<unsigned>(b->row_blocks), kFlatThreads, 0, st>>>(b->d_build, M + b->off_row, ctx->d_err);
    if (b->num_blocks) {
        k_b_number<<<static_cast<unsigned>(b->num_blocks), kNumberThreads, 0, st>>>(b->d_build, M + b->off_num);
        if (b->row_blocks)
            k_b_remap<<<static_cast<unsigned>(b->row_blocks), kFlatThreads, 0, st>>>(b->d_build, M + b->off_row);
        if (b->slot_blocks)
            k_b_direct<<<static_cast<unsigned>(b->slot_blocks), kFlatThreads, 0, st>>>(b->d_build, M + b->off_slot);
    }
    if (b->grange_blocks)
        k_b_grange<<<static_cast<unsigned>(b->grange_blocks), kDirThreads, 0, st>>>(b->d_gdir, M + b->off_grange);
    if (b->gdirect_blocks)
        k_b_gdirect<<<static_cast<unsigned>(b->gdirect_blocks), kDirThreads, kDirSmemBytes + kDirArgsBytes, st>>>(
            b->d_gdir, M + b->off_gdirect);
    if (b->scan_chunks[0])
        k_b_scan<FilterBody><<<b->scan_grid[0], kEngineThreads, b->scan_smem[0], st>>>(
            b->d_scan[0], M + b->off_scan[0], b->d_ticket[0], b->scan_chunks[0]);
    if (b->scan_chunks[1])
        k_b_scan<GroupBody><<<b->scan_grid[1], kEngineThreads, b->scan_smem[1], st>>>(
            b->d_scan[1], M + b->off_scan[1], b->d_ticket[1], b->scan_chunks[1]);
    if (b->scan_chunks[2])
        k_b_scan<PlanJoinBody><<<b->scan_grid[2], kEngineThreads, b->scan_smem[2], st>>>(
            b->d_scan[2], M + b->off_scan[2], b->d_ticket[2], b->scan_chunks[2]);
    if (b->scan_chunks[3])
        k_b_scan<MultiBody><<<b->scan_grid[3], kEngineThreads, b->scan_smem[3], st>>>(
            b->d_scan[3], M + b->off_scan[3], b->d_ticket[3], b->scan_chunks[3]);
    if (b->fold_blocks)
        k_b_fold<<<static_cast<unsigned>(b->fold_blocks), kFoldThreads, 0, st>>>(b->d_fold, M + b->off_fold);
    if (b->compact_blocks)
        k_b_compact<<<static_cast<unsigned>(b->compact_blocks), kCompactThreads, 0, st>>>(b->d_compact,
                                                                                           M + b->off_compact);
    if (!b->fin.empty())
        k_b_finalize<<<static_cast<unsigned>(b->fin.size()), kFinThreads, kFinSmemBytes, st>>>(b->d_fin);
    if (b->sel_blocks) {
        for (int pass = 0; pass < kSelPasses; ++pass)
            k_b_sel<<<static_cast<unsigned>(b->sel_blocks), kSelThreads, 0, st>>>(b->d_top, M + b->off_sel, pass);
        k_b_selcollect<<<static_cast<unsigned>(b->sel_blocks), kSelThreads, 0, st>>>(b->d_top, M + b->off_sel);
        k_b_selemit<<<static_cast<unsigned>(b->top.size()), kTopThreads, 0, st>>>(b->d_top);
    }
    if (b->top0_blocks) {
        k_b_topk0<<<static_cast<unsigned>(b->top0_blocks), kTopThreads, 0, st>>>(b->d_top, M + b->off_top0);
        for (size_t L = 0; L < b->levels.size(); ++L)
            k_b_topk<<<static_cast<unsigned>(b->level_blocks[L]), kTopThreads, 0, st>>>(b->d_top, b->d_levels[L],
                                                                                       M + b->off_level[L]);
    }
    TQP_CUDA(cudaGetLastError());
    return TQP_OK;
}

// Lower, lay out and upload every batched job (no launch).
// Launch shape of the scan of one body kind: the largest stage of its jobs.
template <class Body>
static tqp_status scan_shape(tqp_batch* b, int k) {
    static SmemFlags attr;
    tqp_ctx* ctx = b->ctx;
    if (b->scan[k].empty()) return TQP_OK;
    TQP_TRY(allow_smem(ctx, reinterpret_cast<const void*>(k_b_scan<Body>), attr));
    int max_stage = 128;
    for (auto& j : b->scan[k]) max_stage = std::max(max_stage, job_stage_bytes(j));
    b->scan_smem[k] = kHeaderBytes + kJobBytes + body_bytes<Body>() + static_cast<size_t>(kBatchStages) * max_stage;
    if (b->scan_smem[k] + 1024 > static_cast<size_t>(ctx->smem_optin))
        return fail(TQP_ERR_UNSUPPORTED, "batched scan needs %zu bytes of shared memory", b->scan_smem[k]);
    int occ = 0;
    TQP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_b_scan<Body>, kEngineThreads, b->scan_smem[k]));
    b->scan_grid[k] = ctx->num_sms * std::max(1, std::min(occ, 2));
    assign_chunks(b, k);
    return TQP_OK;
}

// Lower, lay out and upload every batched job (no launch).
static tqp_status batch_prepare(tqp_ctx* ctx, const tqp_plan* plans, const tqp_result* res, int32_t n, tqp_batch* b,
                                cudaStream_t st) {
    static SmemFlags attr_fin, attr_dir;
    TQP_TRY(allow_smem(ctx, reinterpret_cast<const void*>(k_b_finalize), attr_fin));
    TQP_TRY(allow_smem(ctx, reinterpret_cast<const void*>(k_b_gdirect), attr_dir));
    TQP_TRY(lower_batch(b, plans, res, n));
    TQP_TRY(scan_shape<FilterBody>(b, 0));
    TQP_TRY(scan_shape<GroupBody>(b, 1));
    TQP_TRY(scan_shape<PlanJoinBody>(b, 2));
    TQP_TRY(scan_shape<MultiBody>(b, 3));
    plan_top_levels(b);
    build_maps(b);
    TQP_TRY(upload(b, b->fill, &b->d_fill, st));
    TQP_TRY(upload(b, b->zero, &b->d_zero, st));
    TQP_TRY(upload(b, b->build, &b->d_build, st));
    TQP_TRY(upload(b, b->mblob, &b->d_mblob, st));
    for (size_t i = 0; i < b->scan[kJobMulti - 1].size(); ++i)
        mq_bind(&b->scan[kJobMulti - 1][i].u.m, b->d_mblob + b->mblob_off[i]);
    for (int k = 0; k < kKinds; ++k) TQP_TRY(upload(b, b->scan[k], &b->d_scan[k], st));
    TQP_TRY(upload(b, b->compact, &b->d_compact, st));
    TQP_TRY(upload(b, b->fin, &b->d_fin, st));
    TQP_TRY(upload(b, b->top, &b->d_top, st));
    TQP_TRY(upload(b, b->gdir, &b->d_gdir, st));
    TQP_TRY(upload(b, b->fold, &b->d_fold, st));
    b->d_levels.resize(b->levels.size());
    for (size_t L = 0; L < b->levels.size(); ++L) TQP_TRY(upload(b, b->levels[L], &b->d_levels[L], st));
    TQP_TRY(upload(b, b->maps, &b->d_maps, st));
    return TQP_OK;
}

static tqp_status capture(tqp_batch* b, cudaStream_t cs, bool with_batch, unsigned char* fb_base, size_t fb_bytes,
                          size_t* need, cudaGraph_t* out) {
    *out = nullptr;
    TQP_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    tqp_status s = with_batch ? batch_launch(b, cs) : TQP_OK;
    if (s == TQP_OK) s = run_fallbacks(b, cs, fb_base, fb_bytes, need);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(cs, &g);
    if (s != TQP_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    *out = g;
    return TQP_OK;
}

static tqp_status batch_create(tqp_ctx* ctx, const tqp_plan* plans, const tqp_result* res, int32_t n, tqp_batch* b) {
    b->ctx = ctx;
    b->persistent = true;
    b->top_before = ctx->top;
    TQP_TRY(batch_prepare(ctx, plans, res, n, b, nullptr));
    cudaStream_t cs = nullptr;
    TQP_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    tqp_status s = TQP_OK;
    if (!b->fb_plans.empty()) {
        // size the single-plan path's scratch (a capture that is never run),
        // then give it a long-lived region of its own
        const size_t lo = (ctx->used + 255) / 256 * 256;
        size_t need = 0;
        cudaGraph_t g = nullptr;
        s = lo < ctx->top ? capture(b, cs, false, ctx->arena + lo, ctx->top - lo, &need, &g)
                          : arena_oom(ctx, kPersistentBytes);
        if (g) cudaGraphDestroy(g);
        if (s == TQP_OK) {
            b->fb_bytes = std::max<size_t>(need, kPersistentBytes);
            b->fb_arena = static_cast<unsigned char*>(arena_alloc_top(ctx, b->fb_bytes));
            if (!b->fb_arena) s = arena_oom(ctx, b->fb_bytes);
        }
    }
    if (s == TQP_OK) s = capture(b, cs, true, b->fb_arena, b->fb_bytes, nullptr, &b->graph);
    cudaStreamDestroy(cs);
    TQP_TRY(s);
    TQP_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
    return TQP_OK;
}

tqp_status run_plans_on(tqp_ctx* ctx, const tqp_plan* plans, const tqp_result* res, int32_t n, cudaStream_t st) {
    arena_reset(ctx);
    tqp_batch b;
    b.ctx = ctx;
    b.persistent = false;
    TQP_TRY(batch_prepare(ctx, plans, res, n, &b, st));
    TQP_TRY(batch_launch(&b, st));
    if (b.fb_plans.empty()) return TQP_OK;
    const size_t lo = (ctx->used + 255) / 256 * 256;
    if (lo >= ctx->top) return arena_oom(ctx, lo + kPersistentBytes);
    return run_fallbacks(&b, st, ctx->arena + lo, ctx->top - lo, nullptr);
}

static void release(tqp_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    top_close(b->ctx, b->top_before, b->top_after);
}

// Autotuning of a batch: build it with each candidate tile size, time one
// replay (after a warm-up replay) and keep the fastest.
static tqp_status tune_batch_tile(tqp_ctx* ctx, const tqp_plan* plans, const tqp_result* res, int32_t n, int* tile) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    TQP_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    TQP_CUDA(cudaEventCreate(&ev[0]));
    TQP_CUDA(cudaEventCreate(&ev[1]));
    double best = 1e30;
    for (int T = kBatchTile; T <= 4 * kBatchTile; T *= 2) {
        tqp_batch* c = new (std::nothrow) tqp_batch();
        if (!c) break;
        c->tile = T;
        top_open(ctx);
        tqp_status s = batch_create(ctx, plans, res, n, c);
        c->top_after = ctx->top;
        if (s == TQP_OK) {
            cudaGraphLaunch(c->exec, st);
            cudaEventRecord(ev[0], st);
            cudaGraphLaunch(c->exec, st);
            cudaEventRecord(ev[1], st);
            float ms = 0.f;
            if (cudaEventSynchronize(ev[1]) == cudaSuccess && cudaEventElapsedTime(&ms, ev[0], ev[1]) == cudaSuccess &&
                ms < best) {
                best = ms;
                *tile = T;
            }
        }
        cudaStreamSynchronize(st);
        release(c);
        delete c;
    }
    clear_error();
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    cudaStreamDestroy(st);
    return TQP_OK;
}

}  // namespace tqp

extern "C" {

tqp_status tqp_batch_create(tqp_ctx* ctx, const tqp_plan* plans, const tqp_result* res, int32_t n, tqp_batch** out) {
    clear_error();
    TQP_TRY(check_ctx(ctx));
    if (!out || n < 0 || (n > 0 && (!plans || !res))) return fail(TQP_ERR_INVALID_ARG, "bad batch arguments");
    *out = nullptr;
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(TQP_ERR_CUDA, "cannot select device %d", ctx->device);
    int tile = kBatchTile;
    if (ctx->tuner && ctx->tuner->enabled) TQP_TRY(tune_batch_tile(ctx, plans, res, n, &tile));
    tqp_batch* b = new (std::nothrow) tqp_batch();
    if (!b) return fail(TQP_ERR_OUT_OF_MEMORY, "host allocation failed");
    b->tile = tile;
    top_open(ctx);
    const tqp_status s = batch_create(ctx, plans, res, n, b);
    b->top_after = ctx->top;
    if (s != TQP_OK) {
        release(b);
        delete b;
        return s;
    }
    *out = b;
    return TQP_OK;
}

tqp_status tqp_batch_run(tqp_batch* b, void* stream) {
    clear_error();
    if (!b || !b->exec) return fail(TQP_ERR_INVALID_ARG, "batch is NULL");
    DeviceGuard g(b->ctx->device);
    if (!g.ok) return fail(TQP_ERR_CUDA, "cannot select device %d", b->ctx->device);
    TQP_CUDA(cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream)));
    return TQP_OK;
}

tqp_status tqp_batch_destroy(tqp_batch* b) {
    clear_error();
    if (!b) return TQP_OK;
    {
        DeviceGuard g(b->ctx->device);
        cudaDeviceSynchronize();  // no replay may still read the batch's scratch
        release(b);
    }
    delete b;
    return TQP_OK;
}

tqp_status tqp_run_plans(tqp_ctx* ctx, const tqp_plan* plans, const tqp_result* res, int32_t n, void* stream) {
    clear_error();
    TQP_TRY(check_ctx(ctx));
    if (n < 0 || (n > 0 && (!plans || !res))) return fail(TQP_ERR_INVALID_ARG, "bad plan array");
    if (n == 0) return TQP_OK;
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(TQP_ERR_CUDA, "cannot select device %d", ctx->device);
    return run_plans_on(ctx, plans, res, n, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
