// Radix-partitioned joined aggregation (see partjoin.cuh): kernels and the
// host lowering from the fused probe's arguments.
#include <cstdio>

#include "host.h"
#include "bodies.cuh"
#include "partjoin.cuh"

namespace tqp {

__device__ __forceinline__ int64_t pj_factor(const PjFactor& f, long long r) {
    if (f.kind == kFacConst) return f.b;
    const uint64_t x = static_cast<uint64_t>(ldg_typed(f.p, f.type, r));
    switch (f.kind) {
        case kFacPlain: return static_cast<int64_t>(x);
        case kFacAdd: return static_cast<int64_t>(x + static_cast<uint64_t>(f.b));
        case kFacRsub: return static_cast<int64_t>(static_cast<uint64_t>(f.b) - x);
        default: return static_cast<int64_t>(x * static_cast<uint64_t>(f.a) + static_cast<uint64_t>(f.b));
    }
}

__device__ __forceinline__ int64_t pj_prod(const PjFactor (&f)[2], long long r) {
    const uint64_t a = static_cast<uint64_t>(pj_factor(f[0], r));
    if (f[1].kind == kFacConst && f[1].b == 1) return static_cast<int64_t>(a);
    return static_cast<int64_t>(a * static_cast<uint64_t>(pj_factor(f[1], r)));
}

// A joined row of a key with several build rows: added to each of their groups.
__device__ __forceinline__ void pj_add_chain(const PartJoinArgs& A, const uint4& s, const int64_t (&v)[kPjVals]) {
    const GroupSpec& S = A.S;
    uint32_t d = s.z;
    for (uint32_t k = 0; k < s.w; ++k) {
        unsigned long long* a = S.acc + static_cast<long long>(__ldg(&A.dgs[d])) * S.nacc;
        red_add_u64(&a[0], 1ULL);
#pragma unroll
        for (int i = 0; i < kPjVals; ++i)
            if (i < A.nval) red_add_u64(&a[i + 1], static_cast<unsigned long long>(v[i]));
        if (k + 1 < s.w) d = __ldg(&A.next[d]);
    }
}

__global__ void __launch_bounds__(kPjThreads) k_pj_scatter(const __grid_constant__ PartJoinArgs A) {
    __shared__ uint32_t hist[kPjMaxParts];
    __shared__ uint32_t start[kPjMaxParts + 1];
    __shared__ uint32_t wsum[kPjThreads / kWarp];
    __shared__ uint16_t stg_g[kPjChunk];
    __shared__ long long stg_v[kPjVals][kPjChunk];
    __shared__ unsigned long long red3[3][kPjThreads / kWarp];
    const int tid = threadIdx.x, lane = tid % kWarp, w = tid / kWarp;
    const int P = A.nparts;
    long long kmin = 0;
    const bool direct = ht_is_direct(A.H, &kmin);
    const uint32_t gmask = (1u << A.shift) - 1u;
    unsigned long long joined = 0, passed = 0;
    long long sum = 0;
    for (long long c = blockIdx.x; c < A.nchunks; c += gridDim.x) {
        for (int i = tid; i < P; i += kPjThreads) hist[i] = 0;
        __syncthreads();
        uint32_t g[kPjRowsPerThread], rank[kPjRowsPerThread];
        int64_t v[kPjRowsPerThread][kPjVals];
        int64_t sv[kPjRowsPerThread];
        const long long r0 = c * kPjChunk + tid;
        // every column the thread's rows need (loads in flight together), then their build slots
        bool ok[kPjRowsPerThread];
        uint64_t key[kPjRowsPerThread];
#pragma unroll
        for (int j = 0; j < kPjRowsPerThread; ++j) {
            const long long r = r0 + static_cast<long long>(j) * kPjThreads;
            ok[j] = r < A.n;
            key[j] = 0;
            sv[j] = 0;
#pragma unroll
            for (int a = 0; a < kPjVals; ++a) v[j][a] = 0;
            if (ok[j]) {
                for (int q = 0; q < A.ncond; ++q) {
                    const PjCond& cd = A.cond[q];
                    const uint64_t x = static_cast<uint64_t>(ldg_typed(cd.p, cd.type, r));
                    ok[j] = ok[j] && (((x - static_cast<uint64_t>(cd.lo)) <= cd.span) != (cd.negate != 0));
                }
                key[j] = static_cast<uint64_t>(ldg_typed(A.fk.p, A.fk.type, r));
#pragma unroll
                for (int a = 0; a < kPjVals; ++a)
                    if (a < A.nval) v[j][a] = pj_prod(A.f[a], r);
                if (A.has_sum) sv[j] = pj_prod(A.fs, r);
            }
        }
        uint4 sl[kPjRowsPerThread];
#pragma unroll
        for (int j = 0; j < kPjRowsPerThread; ++j)
            sl[j] = ok[j] ? ht_match(A.H, direct, kmin, key[j]) : make_uint4(0u, 0u, 0u, 0u);
        const uint32_t P_u = static_cast<uint32_t>(P);
#pragma unroll
        for (int j = 0; j < kPjRowsPerThread; ++j) {
            g[j] = 0xFFFFFFFFu;
            passed += ok[j] ? 1u : 0u;
            if (!sl[j].w) continue;
            joined += sl[j].w;
            sum += sv[j] * static_cast<long long>(sl[j].w);
            if (sl[j].z & kDirectGroup) {
                const uint32_t gid = sl[j].z & ~kDirectGroup;
                if ((gid >> A.shift) < P_u) {
                    g[j] = gid;
                    rank[j] = atomicAdd(&hist[gid >> A.shift], 1u);
                } else {  // (not expected: dense ids stay below the partitions' span) straight to L2
                    unsigned long long* ga = A.S.acc + static_cast<long long>(gid) * A.S.nacc;
                    red_add_u64(&ga[0], 1ULL);
#pragma unroll
                    for (int a = 0; a < kPjVals; ++a)
                        if (a < A.nval) red_add_u64(&ga[a + 1], static_cast<unsigned long long>(v[j][a]));
                }
            } else {
                pj_add_chain(A, sl[j], v[j]);
            }
        }
        __syncthreads();
        // partition starts: exclusive scan of the P counts (each thread a run of them)
        constexpr int kPer = kPjMaxParts / kPjThreads;
        uint32_t loc[kPer], tot = 0;
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            const int p = tid * kPer + i;
            loc[i] = p < P ? hist[p] : 0u;
            tot += loc[i];
        }
        uint32_t incl = tot;
#pragma unroll
        for (int o = 1; o < kWarp; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == kWarp - 1) wsum[w] = incl;
        __syncthreads();
        uint32_t before = 0, total = 0;
#pragma unroll
        for (int i = 0; i < kPjThreads / kWarp; ++i) {
            before += i < w ? wsum[i] : 0u;
            total += wsum[i];
        }
        uint32_t run = before + incl - tot;
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            const int p = tid * kPer + i;
            if (p < P) start[p] = run;
            run += loc[i];
        }
        if (tid == 0) start[P] = total;
        __syncthreads();
        uint16_t* seg = A.seg + c * static_cast<long long>(P + 1);
        for (int p = tid; p <= P; p += kPjThreads) seg[p] = static_cast<uint16_t>(start[p]);
#pragma unroll
        for (int j = 0; j < kPjRowsPerThread; ++j) {
            if (g[j] == 0xFFFFFFFFu) continue;
            const uint32_t pos = start[g[j] >> A.shift] + rank[j];
            stg_g[pos] = static_cast<uint16_t>(g[j] & gmask);
#pragma unroll
            for (int a = 0; a < kPjVals; ++a)
                if (a < A.nval) stg_v[a][pos] = v[j][a];
        }
        __syncthreads();
        const long long base = c * kPjChunk;
        for (uint32_t i = tid; i < total; i += kPjThreads) A.rec_g[base + i] = stg_g[i];
        for (int a = 0; a < A.nval; ++a) {
            long long* dst = A.rec_v + static_cast<long long>(a) * A.nchunks * kPjChunk + base;
            for (uint32_t i = tid; i < total; i += kPjThreads) dst[i] = stg_v[a][i];
        }
        __syncthreads();
    }
    // the plan's counts and ungrouped sum; the last block publishes them
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        joined += __shfl_xor_sync(0xffffffffu, joined, o);
        passed += __shfl_xor_sync(0xffffffffu, passed, o);
        sum += __shfl_xor_sync(0xffffffffu, sum, o);
    }
    if (lane == 0) {
        red3[0][w] = joined;
        red3[1][w] = static_cast<unsigned long long>(sum);
        red3[2][w] = passed;
    }
    __syncthreads();
    if (tid != 0) return;
    unsigned long long t[3] = {0, 0, 0};
    for (int i = 0; i < kPjThreads / kWarp; ++i)
        for (int k = 0; k < 3; ++k) t[k] += red3[k][i];
    for (int k = 0; k < 3; ++k)
        if (t[k]) atomicAdd(&A.acc[k], t[k]);
    __threadfence();
    if (atomicAdd(&A.acc[3], 1ULL) != static_cast<unsigned long long>(gridDim.x) - 1ULL) return;
    __threadfence();
    if (A.d_num_joined) *A.d_num_joined = static_cast<int64_t>(atomicAdd(&A.acc[0], 0ULL));
    if (A.d_sum) *A.d_sum = static_cast<int64_t>(atomicAdd(&A.acc[1], 0ULL));
    if (A.d_num_rows) *A.d_num_rows = static_cast<int64_t>(atomicAdd(&A.acc[2], 0ULL));
}

// Work item i of the aggregation: partition i % P, slice i / P of the chunks,
// with P the partitions that hold groups (from the device group count) and as
// many slices per partition as the grid has blocks for.
__global__ void __launch_bounds__(kPjAggThreads) k_pj_agg(const __grid_constant__ PartJoinArgs A) {
    extern __shared__ __align__(16) unsigned long long tab[];
    const int tid = threadIdx.x, lane = tid % kWarp, w = tid / kWarp;
    constexpr int kWarps = kPjAggThreads / kWarp;
    const GroupSpec& S = A.S;
    const int nacc = S.nacc;
    const long long G = *S.d_dense_n;
    const long long kg = 1LL << A.shift;
    const long long P = std::min<long long>((G + kg - 1) / kg, A.nparts);
    if (P <= 0) return;
    const long long nsplit = (static_cast<long long>(gridDim.x) + P - 1) / P;
    const long long items = P * nsplit;
    const long long stride_rec = A.nchunks * kPjChunk;
    for (long long item = blockIdx.x; item < items; item += gridDim.x) {
        const long long p = item % P, sp = item / P;
        const long long c0 = A.nchunks * sp / nsplit, c1 = A.nchunks * (sp + 1) / nsplit;
        for (long long i = tid; i < kg * nacc; i += kPjAggThreads) tab[i] = 0;
        __syncthreads();
        for (long long cb = c0 + static_cast<long long>(w) * kWarp; cb < c1; cb += static_cast<long long>(kWarps) * kWarp) {
            const long long c = cb + lane;
            uint32_t s = 0, len = 0;
            if (c < c1) {
                const uint16_t* sg = A.seg + c * (A.nparts + 1) + p;
                s = sg[0];
                len = static_cast<uint32_t>(sg[1]) - s;
            }
            uint32_t incl = len;
#pragma unroll
            for (int o = 1; o < kWarp; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const uint32_t total = __shfl_sync(0xffffffffu, incl, kWarp - 1);
            const uint32_t excl = incl - len;
            // kPjAggUnroll records per lane in flight: owners and loads first, then the table updates
            for (uint32_t i0 = 0; i0 < total; i0 += kWarp * kPjAggUnroll) {
                uint32_t gg[kPjAggUnroll];
                unsigned long long vv[kPjAggUnroll][kPjVals];
                bool act[kPjAggUnroll];
#pragma unroll
                for (int u = 0; u < kPjAggUnroll; ++u) {
                    const uint32_t i = i0 + u * kWarp + lane;
                    // owner lane: the last lane whose records start at or before i
                    int own = 0;
#pragma unroll
                    for (int b = 16; b > 0; b >>= 1) {
                        const uint32_t e = __shfl_sync(0xffffffffu, excl, (own + b) & (kWarp - 1));
                        if (own + b < kWarp && e <= i) own += b;
                    }
                    const uint32_t os = __shfl_sync(0xffffffffu, s, own);
                    const uint32_t oe = __shfl_sync(0xffffffffu, excl, own);
                    act[u] = i < total;
                    gg[u] = 0;
#pragma unroll
                    for (int a = 0; a < kPjVals; ++a) vv[u][a] = 0;
                    if (act[u]) {
                        const long long idx = (cb + own) * kPjChunk + os + (i - oe);
                        gg[u] = A.rec_g[idx];
#pragma unroll
                        for (int a = 0; a < kPjVals; ++a)
                            if (a < A.nval) vv[u][a] = static_cast<unsigned long long>(A.rec_v[a * stride_rec + idx]);
                    }
                }
#pragma unroll
                for (int u = 0; u < kPjAggUnroll; ++u) {
                    if (!act[u]) continue;
                    unsigned long long* t = tab + static_cast<long long>(gg[u]) * nacc;
                    atomicAdd(&t[0], 1ULL);
#pragma unroll
                    for (int a = 0; a < kPjVals; ++a)
                        if (a < A.nval) atomicAdd(&t[a + 1], vv[u][a]);
                }
            }
        }
        __syncthreads();
        const long long g0 = p * kg;
        for (long long g = tid; g < kg && g0 + g < G; g += kPjAggThreads) {
            const unsigned long long* t = tab + g * nacc;
            if (!t[0]) continue;
            unsigned long long* ga = S.acc + (g0 + g) * nacc;
            for (int a = 0; a < nacc; ++a) red_add_u64(&ga[a], t[a]);
        }
        __syncthreads();
    }
}

// ---- host ---------------------------------------------------------------------

static bool pj_factor_of(const ProdForm& pf, int k, const ScanGeom& G, const tqp_table* F, PjFactor* out) {
    out->kind = pf.kind[k];
    out->a = pf.a[k];
    out->b = pf.b[k];
    out->p = nullptr;
    out->type = 0;
    if (pf.kind[k] == kFacConst) return true;
    for (int c = 0; c < F->num_cols; ++c)
        if (G.col[c].slot >= 0 && G.col[c].soff == pf.soff[k]) {
            out->p = static_cast<const unsigned char*>(F->cols[c].data);
            out->type = F->cols[c].type;
            return true;
        }
    return false;
}

// Scratch of the partitioned path for n fact rows and `nparts` partitions.
static size_t pj_scratch_bytes(long long n, int nparts, int nval) {
    const long long nchunks = (n + kPjChunk - 1) / kPjChunk;
    const size_t recs = static_cast<size_t>(nchunks) * kPjChunk;
    return recs * 2 + 256 + recs * 8 * static_cast<size_t>(nval) + 256 +
           static_cast<size_t>(nchunks) * (nparts + 1) * 2 + 256;
}

// Lower the fused probe's arguments (built for the staged engine, so that
// their closed forms refer to staged columns) into the partitioned kernels'
// and launch them.  Returns TQP_ERR_UNSUPPORTED, with nothing launched and no
// scratch kept, when the plan falls outside what the path covers.
tqp_status launch_part_join(tqp_ctx* ctx, const PlanJoinArgs& J, const tqp_table* F, long long maxg,
                            unsigned long long* acc_words, cudaStream_t stream) {
    if (!J.dgs || !J.pjfast || !J.H.meta) return TQP_ERR_UNSUPPORTED;
    const int nval = J.S.nacc - 1;
    if (nval < 0 || nval > kPjVals || J.S.minmax) return TQP_ERR_UNSUPPORTED;
    int shift = 16;
    while (shift > 0 && (1LL << shift) * J.S.nacc * 8 > kPjTableBytes) --shift;
    const long long parts = (std::max<long long>(maxg, 1) + (1LL << shift) - 1) >> shift;
    if (parts > kPjMaxParts) return TQP_ERR_UNSUPPORTED;
    PartJoinArgs A;
    memset(&A, 0, sizeof(A));
    A.n = F->num_rows;
    A.ncond = J.ncond;
    for (int q = 0; q < J.ncond; ++q) {
        const Cond& cd = J.cond[q];
        A.cond[q] = PjCond{static_cast<const unsigned char*>(F->cols[cd.col].data), F->cols[cd.col].type, cd.negate,
                           cd.lo, cd.span};
    }
    A.fk = PjCol{static_cast<const unsigned char*>(F->cols[J.fk_col].data), F->cols[J.fk_col].type, 0};
    A.nval = nval;
    for (int a = 0; a < nval; ++a)
        for (int k = 0; k < 2; ++k)
            if (!pj_factor_of(J.pacc[a], k, J.G, F, &A.f[a][k])) return TQP_ERR_UNSUPPORTED;
    A.has_sum = J.has_sum;
    for (int k = 0; k < 2; ++k) {
        A.fs[k] = PjFactor{nullptr, 0, kFacConst, 0, k == 0 ? 0 : 1};
        if (J.has_sum && !pj_factor_of(J.psum, k, J.G, F, &A.fs[k])) return TQP_ERR_UNSUPPORTED;
    }
    A.shift = shift;
    A.nparts = static_cast<int32_t>(parts);
    A.H = J.H;
    A.next = J.next;
    A.dgs = J.dgs;
    A.S = J.S;
    A.nchunks = (A.n + kPjChunk - 1) / kPjChunk;
    const size_t used = ctx->used;
    const size_t recs = static_cast<size_t>(A.nchunks) * kPjChunk;
    A.rec_g = static_cast<uint16_t*>(arena_alloc(ctx, recs * 2));
    A.rec_v = static_cast<long long*>(arena_alloc(ctx, std::max<size_t>(recs * 8 * nval, 8)));
    A.seg = static_cast<uint16_t*>(arena_alloc(ctx, static_cast<size_t>(A.nchunks) * (parts + 1) * 2));
    if (!A.rec_g || !A.rec_v || !A.seg) {
        ctx->used = used;  // not enough scratch: the fused probe runs instead
        return TQP_ERR_UNSUPPORTED;
    }
    A.acc = acc_words;
    A.d_num_joined = J.d_num_joined;
    A.d_sum = J.d_sum;
    A.d_num_rows = J.d_num_rows;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pj_scatter, kPjThreads, 0) != cudaSuccess || occ < 1)
        occ = 1;
    const long long sblocks = std::max<long long>(1, std::min<long long>(A.nchunks, static_cast<long long>(occ) * ctx->num_sms));
    k_pj_scatter<<<static_cast<unsigned>(sblocks), kPjThreads, 0, stream>>>(A);
    TQP_CUDA(cudaGetLastError());
    const size_t tab_bytes = static_cast<size_t>(1LL << shift) * J.S.nacc * 8;
    static SmemFlags attr_done;
    TQP_TRY(allow_smem(ctx, reinterpret_cast<const void*>(k_pj_agg), attr_done));
    int aocc = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&aocc, k_pj_agg, kPjAggThreads, tab_bytes) != cudaSuccess ||
        aocc < 1)
        aocc = 1;
    k_pj_agg<<<static_cast<unsigned>(aocc * ctx->num_sms), kPjAggThreads, tab_bytes, stream>>>(A);
    TQP_CUDA(cudaGetLastError());
    return TQP_OK;
}

size_t part_join_scratch_bytes(long long n, long long maxg, int nacc) {
    int shift = 16;
    while (shift > 0 && (1LL << shift) * nacc * 8 > kPjTableBytes) --shift;
    const long long parts = (std::max<long long>(maxg, 1) + (1LL << shift) - 1) >> shift;
    return pj_scratch_bytes(n, static_cast<int>(std::min<long long>(parts, kPjMaxParts)), nacc - 1);
}

}  // namespace tqp
