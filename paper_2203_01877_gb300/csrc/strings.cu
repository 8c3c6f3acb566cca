// String columns, IN and LIKE: the pre-pass that evaluates a scan's set and
// pattern predicates (paper Section 4.1 string representation, Section 5's
// IN / LIKE expressions).
//
// A string column is an (n x m) byte array, each string right-padded with 0.
// The pre-pass evaluates every IN / LIKE / NOT LIKE predicate of one scan in
// a single launch and writes one byte per row (1: all of them hold); the scan
// itself then filters on that byte column like on any uint8 column, so the
// staged scans, the group-bys and the plans need no string code.
//   * a warp takes 32 consecutive rows; for a string column it copies the 32
//     strings (32 m contiguous bytes, 16-byte aligned) into shared memory with
//     vector loads, and each lane then reads its own string from there;
//   * LIKE: the greedy wildcard matcher (advance on a literal or `_`, remember
//     the last `%` and resume after it on a mismatch), linear in practice;
//   * IN: binary search in the sorted, deduplicated values (int64 numbers, or
//     m-byte strings compared bytewise);
//   * the values and patterns travel in the kernel parameters and are copied
//     to shared memory once per block.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "host.h"

namespace tqp {

constexpr int kStrThreads = 256;
constexpr int kStrWarps = kStrThreads / kWarp;
constexpr int kStrMaxWidth = 255;
// LIKE program flags: the first / last segment is anchored to the string's
// start / end; the pattern has no `%` (the one segment is the whole string);
// the greedy matcher on the raw pattern instead (a segment over 32 bytes).
constexpr int kLikeStart = 1, kLikeEnd = 2, kLikeExact = 4, kLikeGreedy = 8;
constexpr int kLikeMaxSeg = 32;

struct StrPred {
    const unsigned char* col;  // column data (device)
    int32_t type;              // TQP_CHAR or a numeric type
    int32_t width;             // string width (TQP_CHAR)
    int32_t op;                // TQP_IN, TQP_LIKE or TQP_NOT_LIKE
    int32_t off;               // byte offset of the values / pattern in the blob (8-aligned)
    int32_t count;             // IN: values; LIKE: pattern bytes
    int32_t nseg;              // LIKE: segments between `%`s
    int32_t flags;             // LIKE: kLike* flags
    int32_t prog;              // LIKE: byte offset of the segment lengths, then 256 masks per segment
    int32_t pad;
};

struct StrLaunch {
    int64_t n;
    unsigned char* out;        // n bytes
    int32_t npred;
    int32_t blob_bytes;
    int32_t stage_bytes;       // per warp: 32 strings of the widest string column (16-byte multiple)
    int32_t pad;
    StrPred p[TQP_MAX_PREDS];
    alignas(16) unsigned char blob[TQP_MAX_SET_BYTES];
};
static_assert(sizeof(StrLaunch) <= 32764, "kernel parameters are limited to 32764 bytes");

// LIKE on s[0, n) with pattern p[0, m): `%` any sequence, `_` one byte.
__device__ __forceinline__ bool like_greedy(const unsigned char* s, int n, const unsigned char* p, int m) {
    int si = 0, pi = 0, star = -1, mark = 0;
    while (si < n) {
        if (pi < m && p[pi] != '%' && (p[pi] == '_' || p[pi] == s[si])) {
            ++si;
            ++pi;
        } else if (pi < m && p[pi] == '%') {
            star = pi++;
            mark = si;
        } else if (star >= 0) {
            pi = star + 1;
            si = ++mark;
        } else {
            return false;
        }
    }
    while (pi < m && p[pi] == '%') ++pi;
    return pi == m;
}

// LIKE by segments: the pattern split at its `%`s into segments (`_` a
// one-byte wildcard inside them), each with a table of 256 masks: bit j of
// mask[c] is set when byte c may stand at the segment's position j.  An
// anchored first / last segment must match at the string's start / end; the
// segments between are found leftmost-first with the Shift-And recurrence
// (D = ((D << 1) | 1) & mask[c] per string byte), and each search starts where
// the previous segment's match ended (the leftmost choice leaves the most
// room for the rest, so it finds a match whenever one exists).
__device__ __forceinline__ bool seg_at(const unsigned char* s, int p, int len, const uint32_t* mk) {
    for (int j = 0; j < len; ++j)
        if (!((mk[s[p + j]] >> j) & 1u)) return false;
    return true;
}

__device__ bool like_segments(const unsigned char* s, int n, const StrPred& q, const unsigned char* blob) {
    const int32_t* lens = reinterpret_cast<const int32_t*>(blob + q.prog);
    const uint32_t* masks = reinterpret_cast<const uint32_t*>(blob + q.prog + ((q.nseg * 4 + 15) / 16) * 16);
    if (q.flags & kLikeExact) return n == lens[0] && seg_at(s, 0, lens[0], masks);
    int pos = 0, first = 0, last = q.nseg;
    if (q.flags & kLikeStart) {
        if (lens[0] > n || !seg_at(s, 0, lens[0], masks)) return false;
        pos = lens[0];
        first = 1;
    }
    int limit = n;  // the middle segments must end by here
    if (q.flags & kLikeEnd) {
        last = q.nseg - 1;
        limit = n - lens[last];
        if (limit < pos || !seg_at(s, limit, lens[last], masks + 256 * last)) return false;
    }
    for (int k = first; k < last; ++k) {
        const uint32_t* mk = masks + 256 * k;
        const uint32_t hit = 1u << (lens[k] - 1);
        uint32_t D = 0;
        int i = pos;
        for (; i < limit; ++i) {
            D = ((D << 1) | 1u) & mk[s[i]];
            if (D & hit) break;
        }
        if (i >= limit) return false;
        pos = i + 1;
    }
    return true;
}

// Bytewise comparison of two m-byte strings.
__device__ __forceinline__ int str_cmp(const unsigned char* a, const unsigned char* b, int m) {
    for (int i = 0; i < m; ++i)
        if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
    return 0;
}

__global__ void __launch_bounds__(kStrThreads) k_str_prepass(const __grid_constant__ StrLaunch L) {
    extern __shared__ __align__(16) unsigned char ssm[];
    unsigned char* blob = ssm;                                           // the values and patterns
    unsigned char* stage = ssm + ((L.blob_bytes + 15) / 16) * 16;        // per warp: 32 strings
    for (int i = threadIdx.x; i < L.blob_bytes; i += blockDim.x) blob[i] = L.blob[i];
    __syncthreads();
    const int lane = threadIdx.x % kWarp, w = threadIdx.x / kWarp;
    unsigned char* my = stage + w * L.stage_bytes;
    const long long groups = (L.n + kWarp - 1) / kWarp;
    for (long long g = static_cast<long long>(blockIdx.x) * kStrWarps + w; g < groups;
         g += static_cast<long long>(gridDim.x) * kStrWarps) {
        const long long r0 = g * kWarp, row = r0 + lane;
        const int rows = static_cast<int>(L.n - r0 < kWarp ? L.n - r0 : kWarp);
        bool pass = lane < rows;
        for (int k = 0; k < L.npred; ++k) {
            if (!__any_sync(0xffffffffu, pass)) break;
            const StrPred& q = L.p[k];
            if (q.type == TQP_CHAR) {
                const int m = q.width;
                // the group's strings: rows * m bytes from a 16-byte aligned start
                const unsigned char* src = q.col + r0 * m;
                const int bytes = rows * m;
                __syncwarp();
                for (int i = lane; i < bytes / 16; i += kWarp)
                    reinterpret_cast<uint4*>(my)[i] = __ldg(reinterpret_cast<const uint4*>(src) + i);
                for (int i = (bytes / 16) * 16 + lane; i < bytes; i += kWarp) my[i] = __ldg(src + i);
                __syncwarp();
                if (pass) {
                    const unsigned char* s = my + lane * m;
                    if (q.op == TQP_IN) {
                        const unsigned char* v = blob + q.off;
                        int lo = 0, hi = q.count;  // first value >= s
                        while (lo < hi) {
                            const int mid = (lo + hi) / 2;
                            if (str_cmp(v + mid * m, s, m) < 0) lo = mid + 1;
                            else hi = mid;
                        }
                        pass = lo < q.count && str_cmp(v + lo * m, s, m) == 0;
                    } else {
                        int n = 0;
                        if ((m & 3) == 0) {  // four bytes at a time: the first zero byte of a word
                            const uint32_t* sw = reinterpret_cast<const uint32_t*>(s);
                            n = m;
                            for (int i = 0; i < m / 4; ++i) {
                                const uint32_t x = sw[i];
                                const uint32_t z = (x - 0x01010101u) & ~x & 0x80808080u;  // lowest set bit: first zero byte
                                if (z) {
                                    n = 4 * i + (__ffs(z) - 1) / 8;
                                    break;
                                }
                            }
                        } else {
                            while (n < m && s[n]) ++n;
                        }
                        const bool hit = (q.flags & kLikeGreedy) ? like_greedy(s, n, blob + q.off, q.count)
                                                                 : like_segments(s, n, q, blob);
                        pass = q.op == TQP_LIKE ? hit : !hit;
                    }
                }
            } else if (pass) {  // IN on a numeric column
                const int64_t x = ldg_typed(q.col, q.type, row);
                const int64_t* v = reinterpret_cast<const int64_t*>(blob + q.off);
                int lo = 0, hi = q.count;
                while (lo < hi) {
                    const int mid = (lo + hi) / 2;
                    if (v[mid] < x) lo = mid + 1;
                    else hi = mid;
                }
                pass = lo < q.count && v[lo] == x;
            }
        }
        if (lane < rows) L.out[row] = pass ? 1 : 0;
    }
}

static bool is_set_op(int op) { return op == TQP_IN || op == TQP_LIKE || op == TQP_NOT_LIKE; }

bool has_set_preds(const tqp_table* t, const tqp_pred* preds, int32_t npreds) {
    for (int i = 0; i < npreds && i < TQP_MAX_PREDS && preds; ++i) {
        if (is_set_op(preds[i].op)) return true;
        if (preds[i].col >= 0 && preds[i].col < t->num_cols && t->cols[preds[i].col].type == TQP_CHAR) return true;
    }
    return false;
}

tqp_status str_prepass(tqp_ctx* ctx, const tqp_table* t, const tqp_pred* preds, int32_t npreds, cudaStream_t st,
                       StrLowered* out, bool check_only) {
    out->active = false;
    out->t = *t;
    out->npreds = npreds;
    if (npreds < 0 || npreds > TQP_MAX_PREDS)
        return fail(TQP_ERR_INVALID_ARG, "npreds %d outside [0, %d]", npreds, TQP_MAX_PREDS);
    if (npreds > 0 && !preds) return fail(TQP_ERR_INVALID_ARG, "preds is NULL");
    for (int i = 0; i < npreds; ++i) out->preds[i] = preds[i];
    if (!has_set_preds(t, preds, npreds)) return TQP_OK;
    std::vector<unsigned char> lb(sizeof(StrLaunch), 0);
    StrLaunch* L = reinterpret_cast<StrLaunch*>(lb.data());
    std::vector<int> cols;
    int nkeep = 0;
    size_t used = 0;
    int maxw = 0;
    for (int i = 0; i < npreds; ++i) {
        const tqp_pred& p = preds[i];
        if (p.col < 0 || p.col >= t->num_cols)
            return fail(TQP_ERR_INVALID_ARG, "predicate %d: column %d out of range", i, p.col);
        const tqp_column& c = t->cols[p.col];
        const bool str = c.type == TQP_CHAR;
        if (!is_set_op(p.op)) {
            if (str)
                return fail(TQP_ERR_INVALID_ARG, "predicate %d: string column %d takes IN / LIKE / NOT LIKE only", i,
                            p.col);
            out->preds[nkeep++] = p;
            continue;
        }
        if (!str && p.op != TQP_IN)
            return fail(TQP_ERR_INVALID_ARG, "predicate %d: LIKE on numeric column %d", i, p.col);
        if (p.hi < 0 || (p.hi > 0 && p.lo == 0))
            return fail(TQP_ERR_INVALID_ARG, "predicate %d: bad value list (lo %lld, hi %lld)", i, (long long)p.lo,
                        (long long)p.hi);
        if (p.op != TQP_IN && p.hi > kStrMaxWidth)
            return fail(TQP_ERR_INVALID_ARG, "predicate %d: LIKE pattern longer than %d bytes", i, kStrMaxWidth);
        StrPred& q = L->p[L->npred++];
        q.col = static_cast<const unsigned char*>(c.data);
        q.type = c.type;
        q.width = str ? c.scale : 0;
        maxw = std::max(maxw, q.width);
        q.op = p.op;
        q.off = static_cast<int32_t>(used);
        const unsigned char* src = reinterpret_cast<const unsigned char*>(static_cast<uintptr_t>(p.lo));
        std::vector<unsigned char> data;
        if (p.op != TQP_IN) {  // the pattern
            data.assign(src, src + p.hi);
            q.count = static_cast<int32_t>(p.hi);
        } else if (str) {      // m-byte strings, sorted and deduplicated
            const int m = c.scale;
            std::vector<std::string> v;
            for (long long k = 0; k < p.hi; ++k) v.emplace_back(reinterpret_cast<const char*>(src) + k * m, m);
            std::sort(v.begin(), v.end(), [](const std::string& a, const std::string& b) {
                return memcmp(a.data(), b.data(), a.size()) < 0;
            });
            v.erase(std::unique(v.begin(), v.end()), v.end());
            for (const std::string& x : v) data.insert(data.end(), x.begin(), x.end());
            q.count = static_cast<int32_t>(v.size());
        } else {               // int64 numbers, sorted and deduplicated
            std::vector<int64_t> v(reinterpret_cast<const int64_t*>(src), reinterpret_cast<const int64_t*>(src) + p.hi);
            std::sort(v.begin(), v.end());
            v.erase(std::unique(v.begin(), v.end()), v.end());
            data.resize(v.size() * 8);
            if (!v.empty()) memcpy(data.data(), v.data(), data.size());
            q.count = static_cast<int32_t>(v.size());
        }
        if (used + data.size() > static_cast<size_t>(TQP_MAX_SET_BYTES))
            return fail(TQP_ERR_UNSUPPORTED, "IN / LIKE values take more than %d bytes", TQP_MAX_SET_BYTES);
        if (!data.empty()) memcpy(L->blob + used, data.data(), data.size());
        used = (used + data.size() + 15) / 16 * 16;
        if (p.op != TQP_IN) {  // the segment program, when it fits (else the greedy matcher)
            std::vector<std::vector<unsigned char>> segs;
            std::vector<unsigned char> cur;
            bool any_pct = false;
            for (unsigned char ch : data) {
                if (ch == '%') {
                    any_pct = true;
                    if (!cur.empty()) segs.push_back(cur);
                    cur.clear();
                } else {
                    cur.push_back(ch);
                }
            }
            if (!cur.empty() || !any_pct) segs.push_back(cur);
            q.nseg = static_cast<int32_t>(segs.size());
            q.flags = any_pct ? 0 : kLikeExact;
            if (any_pct && data.front() != '%') q.flags |= kLikeStart;
            if (any_pct && data.back() != '%') q.flags |= kLikeEnd;
            bool fits = true;
            for (const auto& g : segs) fits = fits && g.size() <= static_cast<size_t>(kLikeMaxSeg);
            const size_t hdr = (segs.size() * 4 + 15) / 16 * 16;
            const size_t prog_bytes = hdr + segs.size() * 256 * 4;
            if (!fits || used + prog_bytes > static_cast<size_t>(TQP_MAX_SET_BYTES)) {
                q.flags = kLikeGreedy;
            } else {
                q.prog = static_cast<int32_t>(used);
                int32_t* lens = reinterpret_cast<int32_t*>(L->blob + used);
                uint32_t* masks = reinterpret_cast<uint32_t*>(L->blob + used + hdr);
                for (size_t k = 0; k < segs.size(); ++k) {
                    lens[k] = static_cast<int32_t>(segs[k].size());
                    for (size_t j = 0; j < segs[k].size(); ++j)
                        for (int c = 0; c < 256; ++c)
                            if (segs[k][j] == '_' || segs[k][j] == c) masks[k * 256 + c] |= 1u << j;
                }
                used += prog_bytes;
            }
        }
        cols.push_back(p.col);
    }
    TQP_TRY(check_device_cols(t, cols, "IN / LIKE"));
    if (t->num_cols + 1 > TQP_MAX_COLS)
        return fail(TQP_ERR_UNSUPPORTED, "IN / LIKE need a free column slot (the table has %d of %d)", t->num_cols,
                    TQP_MAX_COLS);
    if (check_only) {  // the other predicates, as the scan will take them; nothing allocated or launched
        out->npreds = nkeep;
        return TQP_OK;
    }
    // the pass column, then the table with it appended and the predicate on it
    const long long n = t->num_rows;
    unsigned char* pass = nullptr;
    if (n > 0) {
        pass = static_cast<unsigned char*>(arena_alloc(ctx, static_cast<size_t>((n + 15) / 16 * 16)));
        if (!pass) return arena_oom(ctx, static_cast<size_t>((n + 15) / 16 * 16));
        L->n = n;
        L->out = pass;
        L->blob_bytes = static_cast<int32_t>(used);
        L->stage_bytes = (kWarp * maxw + 15) / 16 * 16;
        static SmemFlags attr;
        TQP_TRY(allow_smem(ctx, reinterpret_cast<const void*>(k_str_prepass), attr));
        const size_t smem = (used + 15) / 16 * 16 + static_cast<size_t>(kStrWarps) * L->stage_bytes;
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_str_prepass, kStrThreads, smem) != cudaSuccess ||
            occ < 1)
            occ = 1;
        const long long groups = (n + kWarp - 1) / kWarp;
        const long long want = (groups + kStrWarps - 1) / kStrWarps;
        const int grid = static_cast<int>(std::min<long long>(want, static_cast<long long>(ctx->num_sms) * occ));
        k_str_prepass<<<grid, kStrThreads, smem, st>>>(*L);
        TQP_CUDA(cudaGetLastError());
    }
    out->cols.assign(t->cols, t->cols + t->num_cols);
    tqp_column pc;
    pc.data = pass;
    pc.type = TQP_U8;
    pc.scale = 0;
    out->cols.push_back(pc);
    out->t.num_cols = t->num_cols + 1;
    out->t.cols = out->cols.data();
    tqp_pred eq;
    eq.col = t->num_cols;
    eq.op = TQP_EQ;
    eq.lo = 1;
    eq.hi = 0;
    out->preds[nkeep++] = eq;
    out->npreds = nkeep;
    out->active = true;
    return TQP_OK;
}

}  // namespace tqp
