// Group-by for few groups without staging (the aggregation of Section 5.4,
// one output row per distinct key tuple, for the shape where the key domain
// is small, e.g. the six (flag, status) groups of the scan-aggregate query).
//
// Every thread reads four consecutive rows of each column with one vector
// load (16 bytes of int32, two 16-byte pairs of int64, 4 bytes of uint8), so
// a warp covers 128 consecutive rows per step and nothing is staged through
// shared memory.  Rows are added into lane-private accumulator tables in
// shared memory ([slot][acc][lane] per warp: no two lanes share an address,
// no atomics), with the four rows of a lane that share a group folded first.
// The warp's keys live in a list of kDirSlots entries held in registers
// (identical in every lane).  When a step brings more distinct keys than the
// list holds, the warp flushes its tables into the global table and starts a
// new list; rows that still do not fit go to the global table one by one.
// With few threads' worth of state per SM the kernel runs two CTAs of eight
// warps per SM, and the accumulators reach the global table once per warp.
#pragma once

#include "group.cuh"

namespace tqp {

constexpr int kDirThreads = 256;
constexpr int kDirMinBlocks = 2;
constexpr int kDirSlots = 8;                    // keys per warp list
constexpr int kDirAcc = 4;                      // count + three sums
constexpr int kDirConds = 4;
constexpr int kDirKeys = TQP_MAX_GROUP_COLS;
constexpr int kDirSums = kDirAcc - 1;
constexpr int kDirWarpWords = kDirSlots * kDirAcc * 32;
constexpr int kDirSmemBytes = (kDirThreads / 32) * kDirWarpWords * 8;  // 64 KB

struct DirCol {
    const unsigned char* p;
    int32_t type;
    int32_t pad;
};

// A range condition on a column: a row passes iff ((x - lo) <= span) != negate
// (32-bit arithmetic for 32- and 8-bit columns, as in the staged scans).
struct DirCond {
    const unsigned char* p;
    int32_t type;
    int32_t negate;
    int64_t lo;
    uint64_t span;
};

// One affine factor a * x + b of a closed-form sum (kind as in ProdForm).
struct DirFactor {
    const unsigned char* p;
    int32_t type;
    int32_t kind;
    int64_t a;
    int64_t b;
};

struct GroupDirectArgs {
    long long n;
    int32_t ncond, ngc, nsum, kw32;
    DirCond cond[kDirConds];
    DirCol key[kDirKeys];
    DirFactor f[kDirSums][2];
    GroupSpec S;
    int* err;
};

// x[j] = row 4 q + j of a column.  kFull: all four rows exist (one vector
// load of the 16-byte aligned column); otherwise rows from `n` on read as 0.
template <bool kFull>
__device__ __forceinline__ void dir_load4(const unsigned char* p, int type, long long q, long long n,
                                          int64_t (&x)[4]) {
    if constexpr (kFull) {
        if (type == TQP_I64) {
            const longlong2* v = reinterpret_cast<const longlong2*>(p) + 2 * q;
            const longlong2 a = __ldg(v), b = __ldg(v + 1);
            x[0] = a.x;
            x[1] = a.y;
            x[2] = b.x;
            x[3] = b.y;
        } else if (type == TQP_I32) {
            const int4 v = __ldg(reinterpret_cast<const int4*>(p) + q);
            x[0] = v.x;
            x[1] = v.y;
            x[2] = v.z;
            x[3] = v.w;
        } else {
            const unsigned w = __ldg(reinterpret_cast<const unsigned*>(p) + q);
#pragma unroll
            for (int j = 0; j < 4; ++j) x[j] = (w >> (8 * j)) & 0xFFu;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) x[j] = 4 * q + j < n ? ldg_typed(p, type, 4 * q + j) : 0;
    }
}

template <bool kFull>
__device__ __forceinline__ void dir_factor(const DirFactor& f, long long q, long long n, int64_t (&x)[4]) {
    const int kind = f.kind;
    if (kind == kFacConst) {
#pragma unroll
        for (int j = 0; j < 4; ++j) x[j] = f.b;
        return;
    }
    dir_load4<kFull>(f.p, f.type, q, n, x);
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

// Every listed key's lane partials into the global table; the warp's tables are zero afterwards.
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
                unsigned long long x = *p;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                *p = 0;
                if (lane == 0 && x && g >= 0) red_add_u64(&S.acc[g * S.nacc + a], x);
            }
        }
    }
    __syncwarp();
}

// The four rows of every lane (pass bits `ok`) into the lane tables: ids from
// the warp's key list (extended with new keys), rows of a lane with the same
// id folded, then one read-add-write per (distinct id, accumulator).  False,
// with nothing added, when the list would overflow.
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
    // fold rows of this lane that share a group
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
                for (int a = 0; a < kDirSums; ++a) val[a][k] += val[a][j];
                act &= ~(1u << j);
                done = true;
            }
        }
    }
    const int nacc = A.S.nacc;
    unsigned long long* p[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) p[j] = area + (id[j] < 0 ? 0 : id[j]) * (kDirAcc * 32) + lane;
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
                    p[j][a * 32] = old[j] + (a == 0 ? cnt[j] : static_cast<unsigned long long>(val[a - 1][j]));
        }
    }
    return true;
}

// One warp step: the quad q of every lane (kFull: every lane's quad holds
// four rows of the table; otherwise quads at or past nq hold none).
template <bool kFull>
__device__ __forceinline__ void dir_step(const GroupDirectArgs& A, unsigned long long* area, uint64_t (&dk)[kDirSlots],
                                         int& nused, long long q, int lane) {
    const GroupSpec& S = A.S;
    const long long n = A.n;
    uint32_t ok = 0xFu;
    long long qq = q;
    if (!kFull) {
        const long long nq = (n + 3) / 4;
        qq = q < nq ? q : 0;
        ok = 0;
        if (q < nq)
#pragma unroll
            for (int j = 0; j < 4; ++j) ok |= static_cast<uint32_t>(4 * q + j < n) << j;
    }
#pragma unroll
    for (int c = 0; c < kDirConds; ++c) {
        if (c < A.ncond) {
            const DirCond& cd = A.cond[c];
            int64_t x[4];
            dir_load4<kFull>(cd.p, cd.type, qq, n, x);
            uint32_t m = 0;
            if (cd.type == TQP_I64) {
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
    if (!__any_sync(0xffffffffu, ok != 0)) return;
    uint64_t key[4] = {0, 0, 0, 0};
#pragma unroll
    for (int i = 0; i < kDirKeys; ++i) {
        if (i < A.ngc) {
            int64_t x[4];
            dir_load4<kFull>(A.key[i].p, A.key[i].type, qq, n, x);
            const int b = S.key_bits[i];
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
    int64_t val[kDirSums][4];
#pragma unroll
    for (int a = 0; a < kDirSums; ++a) {
        if (a < A.nsum) {
            dir_factor<kFull>(A.f[a][0], qq, n, val[a]);
            if (A.f[a][1].kind != kFacConst || A.f[a][1].b != 1) {
                int64_t y[4];
                dir_factor<kFull>(A.f[a][1], qq, n, y);
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    val[a][j] = static_cast<int64_t>(static_cast<uint64_t>(val[a][j]) * static_cast<uint64_t>(y[j]));
            }
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) val[a][j] = 0;
        }
    }
    if (dir_lane_step(A, area, dk, nused, ok, key, val, lane)) return;
    dir_flush(A, area, dk, nused, lane);  // list full: flush and start a new one
    nused = 0;
    if (dir_lane_step(A, area, dk, nused, ok, key, val, lane)) return;
    // more distinct keys in this step than a list holds: row by row into the global table
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (!((ok >> j) & 1u)) continue;
        const long long g = gtab_slot(S, key[j], A.err);
        if (g < 0) continue;
        red_add_u64(&S.acc[g * S.nacc], 1ULL);
#pragma unroll
        for (int a = 1; a <= kDirSums; ++a)
            if (a < S.nacc) red_add_u64(&S.acc[g * S.nacc + a], static_cast<unsigned long long>(val[a - 1][j]));
    }
}

// One CTA of the direct group-by: warps take 32 quads at a time in a
// grid-stride loop (warp-uniform trip count); steps whose 32 quads all lie
// within the table take the vector-load path.
__device__ __forceinline__ void group_direct_block(const GroupDirectArgs& A, unsigned char* smem) {
    const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
    unsigned long long* area = reinterpret_cast<unsigned long long*>(smem) + w * kDirWarpWords;
    for (int i = lane; i < kDirWarpWords; i += 32) area[i] = 0;
    __syncwarp();
    uint64_t dk[kDirSlots];
#pragma unroll
    for (int d = 0; d < kDirSlots; ++d) dk[d] = 0;
    int nused = 0;
    const long long nq = (A.n + 3) / 4;
    const long long nfull = A.n / 4;  // quads with four rows
    const long long stride = static_cast<long long>(gridDim.x) * kDirThreads;
    for (long long base = static_cast<long long>(blockIdx.x) * kDirThreads + w * 32; base < nq; base += stride) {
        if (base + 32 <= nfull) dir_step<true>(A, area, dk, nused, base + lane, lane);
        else dir_step<false>(A, area, dk, nused, base + lane, lane);
    }
    dir_flush(A, area, dk, nused, lane);
}

}  // namespace tqp
