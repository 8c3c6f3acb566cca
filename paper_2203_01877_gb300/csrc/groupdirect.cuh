// Group-by for few groups without the staged scan engine (the aggregation
// of Section 5.4, one output row per distinct key tuple, for the shape where
// the key domain is small, e.g. the six (flag, status) groups of the
// scan-aggregate query).
//
// A warp takes 32 quads of rows at a time (four consecutive rows per lane,
// 128 rows per step).  The columns a step reads are fetched one step ahead
// with asynchronous 16- and 4-byte copies (cp.async) into a per-warp slot in
// shared memory, so their memory latency overlaps the previous step's
// arithmetic; the lane then reads its four values of a column with one
// vector load from the slot.  Rows are added into lane-private accumulator
// tables in shared memory ([slot][acc][lane] per warp: no two lanes share an
// address, no atomics), with the four rows of a lane that share a group
// folded first.  The warp's keys live in a list of kDirSlots entries held in
// registers (identical in every lane).  When a step brings more distinct keys
// than the list holds, the warp flushes its tables into the global table and
// starts a new list; rows that still do not fit go to the global table one
// by one.  The last, partial steps read global memory directly.
//
// Dense ids: a first pass reduces each key column's [min, max]; when the
// product of the ranges is at most kDirSlots, a row's slot is its mixed-radix
// index sum_i (x_i - min_i) * stride_i -- no key packing, no list lookup --
// and the flush rebuilds each used slot's packed key from its index.
#pragma once

#include "finalize.cuh"

namespace tqp {

constexpr int kDirThreads = 256;
constexpr int kDirMinBlocks = 2;
constexpr int kDirSlots = 8;                    // keys per warp list
constexpr int kDirAcc = 4;                      // count + three sums
constexpr int kDirConds = 4;
constexpr int kDirKeys = TQP_MAX_GROUP_COLS;
constexpr int kDirSums = kDirAcc - 1;
constexpr int kDirWarpWords = kDirSlots * kDirAcc * 32;
constexpr int kDirTableBytes = (kDirThreads / 32) * kDirWarpWords * 8;  // 64 KB
constexpr int kDirPrefCols = 8;          // distinct columns a step reads
constexpr int kDirLaneBytes = 128;       // their bytes per lane (four rows)
constexpr int kDirSlotBytes = 32 * kDirLaneBytes;
constexpr int kDirDenseOff = kDirTableBytes + (kDirThreads / 32) * kDirSlotBytes;
constexpr int kDirSmemBytes = kDirDenseOff + 128;  // 96 KB + the dense-id parameters

// Dense ids of the CTA (computed once from the key ranges).
struct DirDense {
    long long kmin[kDirKeys];
    int32_t stride[kDirKeys];
    int32_t range[kDirKeys];
    int32_t P;      // slots in use: the product of the ranges
    int32_t dense;  // 1: ids are mixed-radix indices
};
static_assert(sizeof(DirDense) <= 128, "dense parameters");
// the last CTA finalizes the table in the (then unused) lane tables and slots
static_assert(kDirSmemBytes >= 2 * kSmallCap * (8 + 4), "finalize scratch");

// A column fetched ahead: its block in a warp slot starts at `off` and holds
// the four values of every lane (esize 8: [half][lane][16 B]; 4: [lane][16 B];
// 1: [lane][4 B]).
struct DirPref {
    const unsigned char* p;
    int32_t type;
    int32_t off;
};

struct DirCol {
    const unsigned char* p;
    int32_t type;
    int32_t soff;  // byte offset of its block in a warp slot (GroupDirectArgs::pref)
};

// A range condition on a column: a row passes iff ((x - lo) <= span) != negate
// (32-bit arithmetic for 32- and 8-bit columns, as in the staged scans).
struct DirCond {
    const unsigned char* p;
    int32_t type;
    int32_t negate;
    int64_t lo;
    uint64_t span;
    int32_t soff;
    int32_t pad;
};

// One affine factor a * x + b of a closed-form sum (kind as in ProdForm).
struct DirFactor {
    const unsigned char* p;
    int32_t type;
    int32_t kind;
    int64_t a;
    int64_t b;
    int32_t soff;
    int32_t pad;
};

struct GroupDirectArgs {
    long long n;
    int32_t ncond, ngc, nsum, kw32;
    DirCond cond[kDirConds];
    DirCol key[kDirKeys];
    DirFactor f[kDirSums][2];
    int32_t npref;
    int32_t pad;
    DirPref pref[kDirPrefCols];
    GroupSpec S;
    int* err;
    // key ranges from the first pass, as [2 i] = max of ~enc(x) and [2 i + 1]
    // = max of enc(x), enc(x) = x ^ 2^63 (so the first is ~enc(min)): either
    // reduced into kmeta, or one record of 2 kDirKeys words per range block
    // in kpart (nparts records); both nullptr: no key columns
    const unsigned long long* kmeta;
    const unsigned long long* kpart;
    int32_t nparts;
    int32_t fin;              // 1: the last CTA finalizes the table into O
    unsigned int* done;       // CTAs finished (zeroed by the range pass when fin)
    GroupOut O;
};

// Shape of the kernel's query.  In the generic kernel every member returns -1
// (decided at run time from the arguments: the column types, the expression
// kinds, the counts); a kernel compiled for one query shape at run time
// (jit.cu) returns that shape's values, so the per-step dispatch on them
// folds away.  Factor i is factor i % 2 of sum i / 2.
struct DirAnySpec {
    static constexpr __device__ int ncond() { return -1; }
    static constexpr __device__ int cond_type(int) { return -1; }
    static constexpr __device__ int ngc() { return -1; }
    static constexpr __device__ int key_type(int) { return -1; }
    static constexpr __device__ int nsum() { return -1; }
    static constexpr __device__ int fac_type(int) { return -1; }
    static constexpr __device__ int fac_kind(int) { return -1; }
    // an earlier factor reading the same column (its values are reused), or -1
    static constexpr __device__ int fac_same(int) { return -1; }
    // 1: sum a multiplies by its second factor; 0: that factor is the constant 1
    static constexpr __device__ int mul(int) { return -1; }
};

// The shape's value where it fixes one (s >= 0), else the run-time one.
__device__ __forceinline__ constexpr int sp_or(int s, int r) { return s >= 0 ? s : r; }

// ---- asynchronous copies into the warp slot ----
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Fetch quad q (four rows, all in the table) of every prefetched column into the slot.
__device__ __forceinline__ void dir_prefetch(const GroupDirectArgs& A, unsigned char* slot, long long q, int lane) {
#pragma unroll
    for (int c = 0; c < kDirPrefCols; ++c) {
        if (c < A.npref) {
            const DirPref& pc = A.pref[c];
            unsigned char* d = slot + pc.off;
            if (pc.type == TQP_I64) {
                const unsigned char* g = pc.p + q * 32;
                cp_async16(d + lane * 16, g);
                cp_async16(d + 512 + lane * 16, g + 16);
            } else if (pc.type == TQP_I32) {
                cp_async16(d + lane * 16, pc.p + q * 16);
            } else {
                cp_async4(d + lane * 4, pc.p + q * 4);
            }
        }
    }
    cp_async_commit();
}

// The lane's four values of a prefetched column (block at byte `soff` of the slot).
__device__ __forceinline__ void dir_slot4(const unsigned char* slot, int soff, int type, int lane, int64_t (&x)[4]) {
    const unsigned char* d = slot + soff;
    if (type == TQP_I64) {
        const longlong2 a = *reinterpret_cast<const longlong2*>(d + lane * 16);
        const longlong2 b = *reinterpret_cast<const longlong2*>(d + 512 + lane * 16);
        x[0] = a.x;
        x[1] = a.y;
        x[2] = b.x;
        x[3] = b.y;
    } else if (type == TQP_I32) {
        const int4 v = *reinterpret_cast<const int4*>(d + lane * 16);
        x[0] = v.x;
        x[1] = v.y;
        x[2] = v.z;
        x[3] = v.w;
    } else {
        const unsigned w = *reinterpret_cast<const unsigned*>(d + lane * 4);
#pragma unroll
        for (int j = 0; j < 4; ++j) x[j] = (w >> (8 * j)) & 0xFFu;
    }
}

// x[j] = row 4 q + j of a column: from the warp slot (kSlot: the step was
// prefetched) or from global memory, rows from `n` on reading as 0.
template <bool kSlot>
__device__ __forceinline__ void dir_load4(const GroupDirectArgs& A, const unsigned char* slot, int soff,
                                          const unsigned char* p, int type, long long q, int lane, int64_t (&x)[4]) {
    if constexpr (kSlot) {
        dir_slot4(slot, soff, type, lane, x);
    } else {
        const long long n = A.n;
#pragma unroll
        for (int j = 0; j < 4; ++j) x[j] = 4 * q + j < n ? ldg_typed(p, type, 4 * q + j) : 0;
    }
}

// x <- the factor's affine form of the column values already in x.
__device__ __forceinline__ void dir_apply_kind(int kind, const DirFactor& f, int64_t (&x)[4]) {
    if (kind == kFacPlain) return;
    const uint64_t b = static_cast<uint64_t>(f.b);
    if (kind == kFacAdd) {
#pragma unroll
        for (int j = 0; j < 4; ++j) x[j] = static_cast<int64_t>(static_cast<uint64_t>(x[j]) + b);
    } else if (kind == kFacRsub) {
#pragma unroll
        for (int j = 0; j < 4; ++j) x[j] = static_cast<int64_t>(b - static_cast<uint64_t>(x[j]));
    } else {
        const uint64_t a = static_cast<uint64_t>(f.a);
#pragma unroll
        for (int j = 0; j < 4; ++j) x[j] = static_cast<int64_t>(static_cast<uint64_t>(x[j]) * a + b);
    }
}

// Factor i (of sum i / 2) for the step's rows; raw[i] keeps the column values
// for a later factor of the same column (SP::fac_same).
template <bool kSlot, class SP>
__device__ __forceinline__ void dir_factor_sp(const GroupDirectArgs& A, const unsigned char* slot, int i, long long q,
                                              int lane, int64_t (&raw)[2 * kDirSums][4], int64_t (&x)[4]) {
    const DirFactor& f = A.f[i / 2][i % 2];
    const int kind = sp_or(SP::fac_kind(i), f.kind);
    if (kind == kFacConst) {
#pragma unroll
        for (int j = 0; j < 4; ++j) x[j] = f.b;
        return;
    }
    const int same = SP::fac_same(i);
    if (same >= 0) {
#pragma unroll
        for (int j = 0; j < 4; ++j) raw[i][j] = raw[same][j];
    } else {
        dir_load4<kSlot>(A, slot, f.soff, f.p, sp_or(SP::fac_type(i), f.type), q, lane, raw[i]);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) x[j] = raw[i][j];
    dir_apply_kind(kind, f, x);
}

template <bool kSlot>
__device__ __forceinline__ void dir_factor(const GroupDirectArgs& A, const unsigned char* slot, const DirFactor& f,
                                           long long q, int lane, int64_t (&x)[4]) {
    const int kind = f.kind;
    if (kind == kFacConst) {
#pragma unroll
        for (int j = 0; j < 4; ++j) x[j] = f.b;
        return;
    }
    dir_load4<kSlot>(A, slot, f.soff, f.p, f.type, q, lane, x);
    if (kind == kFacPlain) return;
    const uint64_t b = static_cast<uint64_t>(f.b);
    if (kind == kFacAdd) {
#pragma unroll
        for (int j = 0; j < 4; ++j) x[j] = static_cast<int64_t>(static_cast<uint64_t>(x[j]) + b);
    } else if (kind == kFacRsub) {
#pragma unroll
        for (int j = 0; j < 4; ++j) x[j] = static_cast<int64_t>(b - static_cast<uint64_t>(x[j]));
    } else {
        const uint64_t a = static_cast<uint64_t>(f.a);
#pragma unroll
        for (int j = 0; j < 4; ++j) x[j] = static_cast<int64_t>(static_cast<uint64_t>(x[j]) * a + b);
    }
}

// Accumulator combines (kMM: some accumulator is a MIN/MAX code, combined
// by unsigned maximum; otherwise every accumulator is a sum).
template <bool kMM>
__device__ __forceinline__ unsigned long long acc_combine(int kind, unsigned long long x, unsigned long long y) {
    if constexpr (kMM) return kind != kAccSum ? (x > y ? x : y) : x + y;
    else return x + y;
}

template <bool kMM>
__device__ __forceinline__ unsigned long long warp_combine(int kind, unsigned long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = acc_combine<kMM>(kind, x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}

// Into the global table: a reduction (sums) or an atomic maximum (codes).
template <bool kMM>
__device__ __forceinline__ void acc_store(int kind, unsigned long long* p, unsigned long long x) {
    if (kMM && kind != kAccSum) atomicMax(p, x);
    else red_add_u64(p, x);
}

// Kind of accumulator a (0 is the count).
__device__ __forceinline__ int acc_kind_of(const GroupSpec& S, int a) { return a == 0 ? kAccSum : S.acc_kind[a - 1]; }

// Every listed key's lane partials into the global table; the warp's tables are zero afterwards.
template <bool kMM>
__device__ __forceinline__ void dir_flush(const GroupDirectArgs& A, unsigned long long* area,
                                          const uint64_t (&dk)[kDirSlots], int nused, int lane) {
    __syncwarp();
    const GroupSpec& S = A.S;
    uint64_t mine = 0;
#pragma unroll
    for (int d = 0; d < kDirSlots; ++d)
        if (d == lane) mine = dk[d];
    const long long gl = lane < nused ? gtab_slot(S, mine, A.err) : -1;
    for (int d = 0; d < nused; ++d) {
        const long long g = __shfl_sync(0xffffffffu, gl, d);
#pragma unroll
        for (int a = 0; a < kDirAcc; ++a) {
            if (a < S.nacc) {
                unsigned long long* p = area + (d * kDirAcc + a) * 32 + lane;
                const int kind = acc_kind_of(S, a);
                const unsigned long long x = warp_combine<kMM>(kind, *p);
                *p = 0;
                if (lane == 0 && x && g >= 0) acc_store<kMM>(kind, &S.acc[g * S.nacc + a], x);
            }
        }
    }
    __syncwarp();
}

// Dense ids, after every warp of the CTA has finished: the CTA's partials of
// each used slot into the global table (its packed key rebuilt from the slot
// index).  Warp w takes the (slot, accumulator) pairs w, w + 8, ...: each
// lane sums its column over the eight warps' tables, the warp sums the
// lanes, and one reduction per pair and CTA goes to L2.
template <bool kMM>
__device__ __forceinline__ void dir_flush_dense_cta(const GroupDirectArgs& A, const DirDense& Dn,
                                                    unsigned long long* tables, int lane, int w) {
    const GroupSpec& S = A.S;
    __shared__ long long gslot[kDirSlots];
    static_assert(kDirSlots <= kDirThreads / 32, "one warp per slot");
    if (w < kDirSlots) {  // warp d: the global entry of slot d, if some row reached it
        const int d = w;
        long long g = -1;
        if (d < Dn.P) {
            unsigned long long c = 0;  // lane l: the count of slot d over the eight warps' lane l
            for (int v = 0; v < kDirThreads / 32; ++v) c += tables[v * kDirWarpWords + (d * kDirAcc) * 32 + lane];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
            if (c && lane == 0) {
                uint64_t key = 0;
                for (int i = 0; i < A.ngc; ++i) {
                    const long long x = Dn.kmin[i] + (d / Dn.stride[i]) % Dn.range[i];
                    const int b = S.key_bits[i];
                    const uint64_t e = enc_key(x, b);
                    key = b == 64 ? e : ((key << b) | e);
                }
                g = gtab_slot(S, key, A.err);
            }
        }
        if (lane == 0) gslot[d] = g;
    }
    __syncthreads();
    const int npairs = Dn.P * S.nacc;
    for (int pr = w; pr < npairs; pr += kDirThreads / 32) {
        const int d = pr / S.nacc, a = pr % S.nacc;
        if (gslot[d] < 0) continue;  // (warp-uniform) no row reached slot d
        const int kind = acc_kind_of(S, a);
        unsigned long long x = 0;
        for (int v = 0; v < kDirThreads / 32; ++v)
            x = acc_combine<kMM>(kind, x, tables[v * kDirWarpWords + (d * kDirAcc + a) * 32 + lane]);
        x = warp_combine<kMM>(kind, x);
        if (lane == 0 && x) acc_store<kMM>(kind, &S.acc[gslot[d] * S.nacc + a], x);
    }
}

// Rows of a lane (pass bits `ok`, slots id[j]) into its lane tables: rows
// with the same slot folded first, so that the read-add-writes of the
// remaining rows touch distinct addresses and issue together instead of
// forming one dependent chain through shared memory.
template <bool kMM>
__device__ __forceinline__ void dir_rmw(const GroupDirectArgs& A, unsigned long long* area, uint32_t ok,
                                        const int (&id)[4], int64_t (&val)[kDirSums][4], int lane) {
    uint32_t act = ok;
    unsigned long long cnt[4] = {1, 1, 1, 1};
#pragma unroll
    for (int j = 1; j < 4; ++j) {
        bool done = false;
#pragma unroll
        for (int k = 0; k < j; ++k) {
            if (!done && ((act >> k) & 1u) && ((act >> j) & 1u) && id[k] == id[j]) {
                cnt[k] += cnt[j];
#pragma unroll
                for (int a = 0; a < kDirSums; ++a)
                    val[a][k] = static_cast<int64_t>(acc_combine<kMM>(
                        acc_kind_of(A.S, a + 1), static_cast<unsigned long long>(val[a][k]),
                        static_cast<unsigned long long>(val[a][j])));
                act &= ~(1u << j);
                done = true;
            }
        }
    }
    const int nacc = A.S.nacc;
    unsigned long long* p[4];
#pragma unroll
    for (int j = 0; j < 4; ++j)  // (rows outside `act` are not touched: their ids may be anything)
        p[j] = area + (static_cast<unsigned>(id[j]) < static_cast<unsigned>(kDirSlots) ? id[j] : 0) * (kDirAcc * 32) + lane;
#pragma unroll
    for (int a = 0; a < kDirAcc; ++a) {
        if (a < nacc) {
            unsigned long long old[4];
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if ((act >> j) & 1u) old[j] = p[j][a * 32];
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if ((act >> j) & 1u)
                    p[j][a * 32] = a == 0 ? old[j] + cnt[j]
                                          : acc_combine<kMM>(acc_kind_of(A.S, a), old[j],
                                                             static_cast<unsigned long long>(val[a - 1][j]));
        }
    }
}

// The four rows of every lane (pass bits `ok`) into the lane tables: ids from
// the warp's key list (extended with new keys), then dir_rmw.  False, with
// nothing added, when the list would overflow.
template <bool kMM>
__device__ __forceinline__ bool dir_lane_step(const GroupDirectArgs& A, unsigned long long* area,
                                              uint64_t (&dk)[kDirSlots], int& nused, uint32_t ok,
                                              const uint64_t (&key)[4], int64_t (&val)[kDirSums][4], int lane) {
    int id[4];
    bool miss = false;
    const bool kw32 = A.kw32 != 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        id[j] = -1;
        if (kw32) {
            const uint32_t k = static_cast<uint32_t>(key[j]);
#pragma unroll
            for (int d = 0; d < kDirSlots; ++d)
                if (d < nused && k == static_cast<uint32_t>(dk[d])) id[j] = d;
        } else {
#pragma unroll
            for (int d = 0; d < kDirSlots; ++d)
                if (d < nused && key[j] == dk[d]) id[j] = d;
        }
        miss |= ((ok >> j) & 1u) && id[j] < 0;
    }
    if (__any_sync(0xffffffffu, miss)) {  // new keys: extend the list (rare after the first steps)
        uint64_t ndk[kDirSlots];
        int nn = nused;
        int nid[4];
#pragma unroll
        for (int d = 0; d < kDirSlots; ++d) ndk[d] = dk[d];
#pragma unroll
        for (int j = 0; j < 4; ++j) nid[j] = id[j];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            bool m = ((ok >> j) & 1u) && nid[j] < 0;
            while (__any_sync(0xffffffffu, m)) {
                if (nn == kDirSlots) return false;  // the list is unchanged: nothing was added
                const int src = __ffs(__ballot_sync(0xffffffffu, m)) - 1;
                const uint64_t k = __shfl_sync(0xffffffffu, key[j], src);
#pragma unroll
                for (int d = 0; d < kDirSlots; ++d)
                    if (d == nn) ndk[d] = k;
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (((ok >> i) & 1u) && nid[i] < 0 && key[i] == k) nid[i] = nn;
                ++nn;
                m = ((ok >> j) & 1u) && nid[j] < 0;
            }
        }
#pragma unroll
        for (int d = 0; d < kDirSlots; ++d) dk[d] = ndk[d];
#pragma unroll
        for (int j = 0; j < 4; ++j) id[j] = nid[j];
        nused = nn;
    }
    dir_rmw<kMM>(A, area, ok, id, val, lane);
    return true;
}

// One warp step: the quad q of every lane.  kSlot: every lane's quad holds
// four rows of the table and sits in the warp slot; otherwise quads at or
// past the end hold none and are read from global memory.
template <bool kSlot, bool kDense, bool kMM, class SP>
__device__ __forceinline__ void dir_step(const GroupDirectArgs& A, const DirDense& Dn, unsigned long long* area,
                                         unsigned char* slot, uint64_t (&dk)[kDirSlots], int& nused, long long q,
                                         int lane, long long next = -1) {
    const GroupSpec& S = A.S;
    const long long n = A.n;
    uint32_t ok = 0xFu;
    long long qq = q;
    if (!kSlot) {
        const long long nq = (n + 3) / 4;
        qq = q < nq ? q : 0;
        ok = 0;
        if (q < nq)
#pragma unroll
            for (int j = 0; j < 4; ++j) ok |= static_cast<uint32_t>(4 * q + j < n) << j;
    }
    const int ncond = sp_or(SP::ncond(), A.ncond);
#pragma unroll
    for (int c = 0; c < kDirConds; ++c) {
        if (c < ncond) {
            const DirCond& cd = A.cond[c];
            const int ctype = sp_or(SP::cond_type(c), cd.type);
            int64_t x[4];
            dir_load4<kSlot>(A, slot, cd.soff, cd.p, ctype, qq, lane, x);
            uint32_t m = 0;
            if (ctype == TQP_I64) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    m |= static_cast<uint32_t>(static_cast<uint64_t>(x[j]) - static_cast<uint64_t>(cd.lo) <= cd.span) << j;
            } else {
                const uint32_t lo = static_cast<uint32_t>(cd.lo), sp = static_cast<uint32_t>(cd.span);
#pragma unroll
                for (int j = 0; j < 4; ++j) m |= static_cast<uint32_t>(static_cast<uint32_t>(x[j]) - lo <= sp) << j;
            }
            ok &= cd.negate ? ~m : m;
        }
    }
    if (!__any_sync(0xffffffffu, ok != 0)) {
        if (kSlot && next >= 0) {
            __syncwarp();
            dir_prefetch(A, slot, next, lane);
        }
        return;
    }
    uint64_t key[4] = {0, 0, 0, 0};
    int id[4] = {0, 0, 0, 0};
    const int ngc = sp_or(SP::ngc(), A.ngc);
#pragma unroll
    for (int i = 0; i < kDirKeys; ++i) {
        if (i < ngc) {
            int64_t x[4];
            dir_load4<kSlot>(A, slot, A.key[i].soff, A.key[i].p, sp_or(SP::key_type(i), A.key[i].type), qq, lane, x);
            const int b = S.key_bits[i];
            if constexpr (kDense) {  // mixed-radix slot index (every key lies in its column's range)
                const long long lo = Dn.kmin[i];
                const int st = Dn.stride[i];
#pragma unroll
                for (int j = 0; j < 4; ++j) id[j] += static_cast<int>(x[j] - lo) * st;
            } else {
              if (b == 8) {
#pragma unroll
                for (int j = 0; j < 4; ++j) key[j] = (key[j] << 8) | (static_cast<uint64_t>(x[j]) & 0xFFu);
            } else if (b == 32) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    key[j] = (key[j] << 32) | static_cast<uint64_t>(static_cast<uint32_t>(x[j]) ^ 0x80000000u);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) key[j] = static_cast<uint64_t>(x[j]) ^ 0x8000000000000000ull;
            }
            }
        }
    }
    int64_t val[kDirSums][4];
    int64_t raw[2 * kDirSums][4];
    const int nsum = sp_or(SP::nsum(), A.nsum);
#pragma unroll
    for (int a = 0; a < kDirSums; ++a) {
        if (a < nsum) {
            dir_factor_sp<kSlot, SP>(A, slot, 2 * a, qq, lane, raw, val[a]);
            const int mul = SP::mul(a);
            if (mul == 1 || (mul < 0 && (A.f[a][1].kind != kFacConst || A.f[a][1].b != 1))) {
                int64_t y[4];
                dir_factor_sp<kSlot, SP>(A, slot, 2 * a + 1, qq, lane, raw, y);
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    val[a][j] = static_cast<int64_t>(static_cast<uint64_t>(val[a][j]) * static_cast<uint64_t>(y[j]));
            }
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) val[a][j] = 0;
        }
    }
    if constexpr (kMM) {  // MIN/MAX accumulators take their order-preserving codes
#pragma unroll
        for (int a = 0; a < kDirSums; ++a) {
            const int kind = acc_kind_of(S, a + 1);
            if (a < nsum && kind != kAccSum)
#pragma unroll
                for (int j = 0; j < 4; ++j) val[a][j] = static_cast<int64_t>(acc_encode(kind, val[a][j]));
        }
    }
    if (kSlot && next >= 0) {  // every slot value is in registers: refill the slot with the next step
        __syncwarp();
        dir_prefetch(A, slot, next, lane);
    }
    if constexpr (kDense) {
        dir_rmw<kMM>(A, area, ok, id, val, lane);
        return;
    }
    if (dir_lane_step<kMM>(A, area, dk, nused, ok, key, val, lane)) return;
    dir_flush<kMM>(A, area, dk, nused, lane);  // list full: flush and start a new one
    nused = 0;
    if (dir_lane_step<kMM>(A, area, dk, nused, ok, key, val, lane)) return;
    // more distinct keys in this step than a list holds: row by row into the global table
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (!((ok >> j) & 1u)) continue;
        const long long g = gtab_slot(S, key[j], A.err);
        if (g < 0) continue;
        red_add_u64(&S.acc[g * S.nacc], 1ULL);
#pragma unroll
        for (int a = 1; a <= kDirSums; ++a)
            if (a < S.nacc)
                acc_store<kMM>(acc_kind_of(S, a), &S.acc[g * S.nacc + a], static_cast<unsigned long long>(val[a - 1][j]));
    }
}

// Dense-id parameters from the encoded key bounds (one thread per CTA):
// ea[i] = ~enc(min_i), eb[i] = enc(max_i).
__device__ __forceinline__ void dir_dense_init(const GroupDirectArgs& A, const unsigned long long* ea,
                                               const unsigned long long* eb, bool have, DirDense* Dn) {
    Dn->dense = 0;
    Dn->P = 1;
    if (A.ngc > 0 && !have) return;
    long long P = 1;
    for (int i = A.ngc - 1; i >= 0; --i) {
        // encoded bounds compare as unsigned; rows exist, so elo <= ehi
        const unsigned long long elo = ~ea[i], ehi = eb[i];
        if (ehi < elo || ehi - elo >= static_cast<unsigned long long>(kDirSlots)) return;
        const unsigned long long r = ehi - elo + 1;
        Dn->kmin[i] = static_cast<long long>(elo ^ (1ULL << 63));
        Dn->range[i] = static_cast<int32_t>(r);
        Dn->stride[i] = static_cast<int32_t>(P);
        P *= static_cast<long long>(r);
        if (P > kDirSlots) return;
    }
    Dn->P = static_cast<int32_t>(P);
    Dn->dense = 1;
}

// Every thread of a CTA (kDirThreads): the key bounds, reduced from the range
// blocks' records (one record per thread: a single round of loads), then
// thread 0 derives the dense-id parameters.
__device__ __forceinline__ void dir_dense_setup(const GroupDirectArgs& A, DirDense* Dn, int lane, int w) {
    __shared__ unsigned long long red[kDirThreads / 32][2 * kDirKeys];
    unsigned long long v[2 * kDirKeys];
#pragma unroll
    for (int k = 0; k < 2 * kDirKeys; ++k) v[k] = 0;
    const bool have = A.kmeta || A.kpart;
    if (A.kpart) {
        for (int p = threadIdx.x; p < A.nparts; p += kDirThreads)
#pragma unroll
            for (int k = 0; k < 2 * kDirKeys; ++k)
                if (k < 2 * A.ngc) {
                    const unsigned long long x = A.kpart[p * 2 * kDirKeys + k];
                    v[k] = x > v[k] ? x : v[k];
                }
    } else if (A.kmeta && threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < 2 * kDirKeys; ++k)
            if (k < 2 * A.ngc) v[k] = A.kmeta[k];
    }
#pragma unroll
    for (int k = 0; k < 2 * kDirKeys; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long x = __shfl_xor_sync(0xffffffffu, v[k], o);
            v[k] = x > v[k] ? x : v[k];
        }
        if (lane == 0) red[w][k] = v[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long ea[kDirKeys], eb[kDirKeys];
#pragma unroll
        for (int i = 0; i < kDirKeys; ++i) {
            ea[i] = eb[i] = 0;
            for (int u = 0; u < kDirThreads / 32; ++u) {
                ea[i] = red[u][2 * i] > ea[i] ? red[u][2 * i] : ea[i];
                eb[i] = red[u][2 * i + 1] > eb[i] ? red[u][2 * i + 1] : eb[i];
            }
        }
        dir_dense_init(A, ea, eb, have, Dn);
    }
}

// The warp's grid-stride loop: 32 quads per step; a step whose quads all lie
// within the table is fetched into the warp slot one step ahead.
template <bool kDense, bool kMM, class SP>
__device__ __forceinline__ void dir_loop(const GroupDirectArgs& A, const DirDense& Dn, unsigned long long* area,
                                         unsigned char* slot, int lane, int w, long long vb, long long vg) {
    uint64_t dk[kDirSlots];
#pragma unroll
    for (int d = 0; d < kDirSlots; ++d) dk[d] = 0;
    int nused = 0;
    const long long nq = (A.n + 3) / 4;
    const long long nfull = A.n / 4;  // quads with four rows
    const long long stride = vg * kDirThreads;
    long long base = vb * kDirThreads + w * 32;
    bool have = base + 32 <= nfull;  // the slot receives step `base`
    if (have) dir_prefetch(A, slot, base + lane, lane);
    for (; base < nq; base += stride) {
        if (have) {
            const long long next = base + stride;
            const bool nhave = next + 32 <= nfull;
            cp_async_wait_all();
            __syncwarp();
            // dir_step moves the step's values to registers, then refills the slot
            dir_step<true, kDense, kMM, SP>(A, Dn, area, slot, dk, nused, base + lane, lane, nhave ? next + lane : -1);
            have = nhave;
        } else {
            dir_step<false, kDense, kMM, SP>(A, Dn, area, slot, dk, nused, base + lane, lane);
        }
    }
    if constexpr (!kDense) dir_flush<kMM>(A, area, dk, nused, lane);  // dense: the CTA flushes once
}

// One CTA of the direct group-by: block vb of vg blocks working on this table
// (kMM: the kernel for tables with MIN/MAX accumulators).
template <bool kMM, class SP = DirAnySpec>
__device__ __forceinline__ void group_direct_block(const GroupDirectArgs& A, unsigned char* smem, long long vb,
                                                   long long vg) {
    const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
    unsigned long long* area = reinterpret_cast<unsigned long long*>(smem) + w * kDirWarpWords;
    unsigned char* slot = smem + kDirTableBytes + w * kDirSlotBytes;
    DirDense* Dn = reinterpret_cast<DirDense*>(smem + kDirDenseOff);
    for (int i = lane; i < kDirWarpWords; i += 32) area[i] = 0;
    dir_dense_setup(A, Dn, lane, w);
    __syncthreads();
    if (Dn->dense) {
        dir_loop<true, kMM, SP>(A, *Dn, area, slot, lane, w, vb, vg);
        __syncthreads();
        dir_flush_dense_cta<kMM>(A, *Dn, reinterpret_cast<unsigned long long*>(smem), lane, w);
    } else {
        dir_loop<false, kMM, SP>(A, *Dn, area, slot, lane, w, vb, vg);
    }
    if (!A.fin) return;
    // the last CTA to finish finalizes the table (every CTA's adds are
    // ordered before its count by the fence)
    __shared__ int last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(A.done, 1u) == static_cast<unsigned int>(vg - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    finalize_small_block(A.S, A.O, smem);
}

// First pass: [min, max] of every key column (encoded as the kmeta words;
// zeroed before the launch).  Each column is read in 16-byte chunks, four
// chunks per thread in flight, and reduced in its own width: four bytes per
// instruction for uint8 (SIMD byte min/max), 32-bit for int32; the ragged
// end is read element by element.
__device__ __forceinline__ void dir_enc_update(long long x, unsigned long long& mx, unsigned long long& mn) {
    const unsigned long long e = static_cast<unsigned long long>(x) ^ (1ULL << 63);
    mx = e > mx ? e : mx;
    mn = ~e > mn ? ~e : mn;
}

__device__ __forceinline__ void group_direct_range_block(const GroupDirectArgs& A, unsigned long long* kmeta,
                                                         unsigned long long* kpart, long long vb, long long vg) {
    __shared__ unsigned long long red[kDirThreads / 32][2];
    const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
    const long long n = A.n;
    const long long tid = vb * blockDim.x + threadIdx.x;
    const long long nth = vg * blockDim.x;
    for (int i = 0; i < A.ngc; ++i) {
        const int type = A.key[i].type;
        const int es = type == TQP_I64 ? 8 : (type == TQP_I32 ? 4 : 1);
        const uint4* p = reinterpret_cast<const uint4*>(A.key[i].p);
        const long long nchunk = n * es / 16;  // whole 16-byte chunks
        unsigned long long mx = 0, mn = 0;
        long long c = tid;
        if (type == TQP_U8) {
            unsigned lo4 = 0xFFFFFFFFu, hi4 = 0;
            for (; c + 3 * nth < nchunk; c += 4 * nth) {
                uint4 v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] = __ldg(p + c + u * nth);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    lo4 = __vminu4(__vminu4(lo4, v[u].x), __vminu4(v[u].y, __vminu4(v[u].z, v[u].w)));
                    hi4 = __vmaxu4(__vmaxu4(hi4, v[u].x), __vmaxu4(v[u].y, __vmaxu4(v[u].z, v[u].w)));
                }
            }
            for (; c < nchunk; c += nth) {
                const uint4 v = __ldg(p + c);
                lo4 = __vminu4(__vminu4(lo4, v.x), __vminu4(v.y, __vminu4(v.z, v.w)));
                hi4 = __vmaxu4(__vmaxu4(hi4, v.x), __vmaxu4(v.y, __vmaxu4(v.z, v.w)));
            }
            if (lo4 != 0xFFFFFFFFu || hi4 != 0) {  // at least one chunk seen
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    dir_enc_update((lo4 >> (8 * k)) & 0xFFu, mx, mn);
                    dir_enc_update((hi4 >> (8 * k)) & 0xFFu, mx, mn);
                }
            }
        } else if (type == TQP_I32) {
            int lo = INT_MAX, hi = INT_MIN;
            bool seen = false;
            for (; c + 3 * nth < nchunk; c += 4 * nth) {
                uint4 v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] = __ldg(p + c + u * nth);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    lo = min(lo, min(min(static_cast<int>(v[u].x), static_cast<int>(v[u].y)),
                                     min(static_cast<int>(v[u].z), static_cast<int>(v[u].w))));
                    hi = max(hi, max(max(static_cast<int>(v[u].x), static_cast<int>(v[u].y)),
                                     max(static_cast<int>(v[u].z), static_cast<int>(v[u].w))));
                }
                seen = true;
            }
            for (; c < nchunk; c += nth) {
                const uint4 v = __ldg(p + c);
                lo = min(lo, min(min(static_cast<int>(v.x), static_cast<int>(v.y)),
                                 min(static_cast<int>(v.z), static_cast<int>(v.w))));
                hi = max(hi, max(max(static_cast<int>(v.x), static_cast<int>(v.y)),
                                 max(static_cast<int>(v.z), static_cast<int>(v.w))));
                seen = true;
            }
            if (seen) {
                dir_enc_update(lo, mx, mn);
                dir_enc_update(hi, mx, mn);
            }
        } else {
            for (; c < nchunk; c += nth) {
                const uint4 v = __ldg(p + c);
                dir_enc_update(static_cast<long long>((static_cast<unsigned long long>(v.y) << 32) | v.x), mx, mn);
                dir_enc_update(static_cast<long long>((static_cast<unsigned long long>(v.w) << 32) | v.z), mx, mn);
            }
        }
        for (long long r = nchunk * 16 / es + tid; r < n; r += nth) dir_enc_update(ldg_typed(A.key[i].p, type, r), mx, mn);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long a = __shfl_xor_sync(0xffffffffu, mx, o), b = __shfl_xor_sync(0xffffffffu, mn, o);
            mx = a > mx ? a : mx;
            mn = b > mn ? b : mn;
        }
        if (lane == 0) {
            red[w][0] = mn;
            red[w][1] = mx;
        }
        __syncthreads();
        if (threadIdx.x < 2) {
            unsigned long long v = 0;
            for (int k = 0; k < static_cast<int>(blockDim.x) / 32; ++k) v = red[k][threadIdx.x] > v ? red[k][threadIdx.x] : v;
            if (kpart) kpart[vb * 2 * kDirKeys + 2 * i + threadIdx.x] = v;
            else atomicMax(&kmeta[2 * i + threadIdx.x], v);
        }
        __syncthreads();
    }
}

// The single-call form of the first pass: block 0 also clears the group
// table and the CTA counter of the direct kernel that follows.
__device__ __forceinline__ void group_direct_prep_block(const GroupDirectArgs& A, unsigned long long* kpart,
                                                        long long vb, long long vg) {
    if (vb == 0) {
        const GroupSpec& S = A.S;
        for (long long i = threadIdx.x; i <= S.cap; i += blockDim.x) S.keys[i] = kEmptyKey;
        for (long long i = threadIdx.x; i < (S.cap + 1) * S.nacc; i += blockDim.x) S.acc[i] = 0;
        if (threadIdx.x == 0) {
            *S.ndistinct = 0;
            if (A.done) *A.done = 0;
        }
    }
    if (A.ngc > 0) group_direct_range_block(A, nullptr, kpart, vb, vg);
}

}  // namespace tqp
