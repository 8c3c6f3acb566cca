// Stable LSD radix sort of (uint64 key, uint32 value) pairs, 8-bit digits.
//
// Used where an operator needs an order the hash table does not give: the
// group-by output (keys ascending, paper Section 5.4 / Algorithm 3's sort)
// and the join's build-side runs of equal keys.  Per pass:
//   upsweep   per-tile digit histograms (shared-memory counters);
//   scan      one block per digit: exclusive scan over tiles, plus the
//             digit's base (sum of all smaller digits' totals);
//   downsweep each warp ranks its own contiguous slice with __match_any_sync
//             peers and per-warp digit bases, so equal digits keep input
//             order (stability) and stores land in ascending position order.
// The item count lives in device memory (it is usually produced by a kernel);
// grids are sized for an upper bound and tiles past the count exit at once.
#include "host.h"

namespace tqp {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / kWarp;
constexpr int kSortItems = 16;                          // per thread
constexpr int kSortTile = kSortThreads * kSortItems;    // 4096
constexpr int kSortSlice = kSortTile / kSortWarps;      // 512 per warp

__global__ void __launch_bounds__(kSortThreads) k_rs_upsweep(const uint64_t* __restrict__ keys,
                                                             const long long* __restrict__ n_ptr, int shift,
                                                             uint32_t* __restrict__ hist, long long ntiles,
                                                             unsigned long long* __restrict__ digit_tot) {
    __shared__ uint32_t cnt[256];
    const long long n = *n_ptr;
    const long long tile = blockIdx.x;
    const long long base = tile * kSortTile;
    cnt[threadIdx.x] = 0;
    __syncthreads();
    if (base < n) {
        for (int i = 0; i < kSortItems; ++i) {
            const long long idx = base + i * kSortThreads + threadIdx.x;
            if (idx < n) atomicAdd(&cnt[(keys[idx] >> shift) & 0xFF], 1u);
        }
    }
    __syncthreads();
    const uint32_t c = cnt[threadIdx.x];
    hist[static_cast<long long>(threadIdx.x) * ntiles + tile] = c;
    if (c) atomicAdd(&digit_tot[threadIdx.x], static_cast<unsigned long long>(c));
}

__global__ void __launch_bounds__(1024) k_rs_scan(uint32_t* __restrict__ hist, long long ntiles,
                                                  const unsigned long long* __restrict__ digit_tot) {
    __shared__ unsigned long long wsum[32];
    __shared__ unsigned long long carry_sm;
    const int d = blockIdx.x;
    const int lane = threadIdx.x % kWarp, w = threadIdx.x / kWarp;
    // base of digit d = totals of all smaller digits
    unsigned long long b = threadIdx.x < static_cast<unsigned>(d) ? digit_tot[threadIdx.x] : 0ULL;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(0xffffffffu, b, o);
    if (lane == 0) wsum[w] = b;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long s = 0;
        for (int i = 0; i < 32; ++i) s += wsum[i];
        carry_sm = s;
    }
    __syncthreads();
    unsigned long long carry = carry_sm;
    uint32_t* row = hist + static_cast<long long>(d) * ntiles;
    for (long long off = 0; off < ntiles; off += 1024) {
        const long long i = off + threadIdx.x;
        const unsigned long long v = i < ntiles ? row[i] : 0u;
        unsigned long long incl = v;
#pragma unroll
        for (int o = 1; o < kWarp; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        __syncthreads();
        if (lane == kWarp - 1) wsum[w] = incl;
        __syncthreads();
        unsigned long long before = 0, total = 0;
        for (int j = 0; j < 32; ++j) {
            const unsigned long long x = wsum[j];
            before += (j < w) ? x : 0ULL;
            total += x;
        }
        if (i < ntiles) row[i] = static_cast<uint32_t>(carry + before + incl - v);
        carry += total;
    }
}

__global__ void __launch_bounds__(kSortThreads) k_rs_downsweep(const uint64_t* __restrict__ kin,
                                                               const uint32_t* __restrict__ vin,
                                                               uint64_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                               const long long* __restrict__ n_ptr, int shift,
                                                               const uint32_t* __restrict__ hist, long long ntiles) {
    __shared__ uint32_t wcnt[kSortWarps][256];
    const long long n = *n_ptr;
    const long long tile = blockIdx.x;
    const long long base = tile * kSortTile;
    if (base >= n) return;
    const int lane = threadIdx.x % kWarp, w = threadIdx.x / kWarp;
    for (int d = lane; d < 256; d += kWarp) wcnt[w][d] = 0;
    __syncwarp();
    const long long s0 = base + static_cast<long long>(w) * kSortSlice;
    // phase 1: per-warp digit counts of the warp's slice
    for (int i = 0; i < kSortSlice / kWarp; ++i) {
        const long long idx = s0 + i * kWarp + lane;
        const int dg = idx < n ? static_cast<int>((kin[idx] >> shift) & 0xFF) : 256;
        const uint32_t peers = __match_any_sync(0xffffffffu, dg);
        if (dg < 256 && lane == __ffs(peers) - 1) wcnt[w][dg] += __popc(peers);
    }
    __syncthreads();
    // phase 2: per-warp bases = global tile offset + counts of earlier warps
    {
        const int d = threadIdx.x;  // 256 threads, one digit each
        uint32_t run = hist[static_cast<long long>(d) * ntiles + tile];
        for (int ww = 0; ww < kSortWarps; ++ww) {
            const uint32_t c = wcnt[ww][d];
            wcnt[ww][d] = run;
            run += c;
        }
    }
    __syncthreads();
    // phase 3: stable scatter
    const uint32_t lt = lanemask_lt();
    for (int i = 0; i < kSortSlice / kWarp; ++i) {
        const long long idx = s0 + i * kWarp + lane;
        uint64_t k = 0;
        uint32_t v = 0;
        int dg = 256;
        if (idx < n) {
            k = kin[idx];
            v = vin[idx];
            dg = static_cast<int>((k >> shift) & 0xFF);
        }
        const uint32_t peers = __match_any_sync(0xffffffffu, dg);
        if (dg < 256) {
            const uint32_t pos = wcnt[w][dg] + __popc(peers & lt);
            kout[pos] = k;
            vout[pos] = v;
        }
        __syncwarp();
        if (dg < 256 && lane == __ffs(peers) - 1) wcnt[w][dg] += __popc(peers);
        __syncwarp();
    }
}

// Scratch needed by radix_sort_pairs for up to n_max items.
size_t radix_sort_scratch(long long n_max) {
    const long long ntiles = (n_max + kSortTile - 1) / kSortTile;
    return 256 * sizeof(unsigned long long) + static_cast<size_t>(256) * ntiles * sizeof(uint32_t) + 256;
}

// Sort bits [begin_bit, end_bit) of the keys.  Buffers (k0, v0) hold the
// input; (k1, v1) are a second buffer of the same size.  *result_in_1 tells
// which buffer holds the sorted output.
tqp_status radix_sort_pairs(uint64_t* k0, uint32_t* v0, uint64_t* k1, uint32_t* v1, const long long* d_n,
                            long long n_max, int begin_bit, int end_bit, void* scratch, cudaStream_t stream,
                            bool* result_in_1) {
    *result_in_1 = false;
    if (n_max <= 0 || end_bit <= begin_bit) return TQP_OK;
    const long long ntiles = (n_max + kSortTile - 1) / kSortTile;
    unsigned long long* digit_tot = static_cast<unsigned long long*>(scratch);
    uint32_t* hist = reinterpret_cast<uint32_t*>(digit_tot + 256);
    bool in1 = false;
    for (int shift = begin_bit; shift < end_bit; shift += 8) {
        uint64_t* ki = in1 ? k1 : k0;
        uint32_t* vi = in1 ? v1 : v0;
        uint64_t* ko = in1 ? k0 : k1;
        uint32_t* vo = in1 ? v0 : v1;
        TQP_CUDA(cudaMemsetAsync(digit_tot, 0, 256 * sizeof(unsigned long long), stream));
        k_rs_upsweep<<<static_cast<unsigned>(ntiles), kSortThreads, 0, stream>>>(ki, d_n, shift, hist, ntiles,
                                                                                 digit_tot);
        k_rs_scan<<<256, 1024, 0, stream>>>(hist, ntiles, digit_tot);
        k_rs_downsweep<<<static_cast<unsigned>(ntiles), kSortThreads, 0, stream>>>(ki, vi, ko, vo, d_n, shift, hist,
                                                                                   ntiles);
        TQP_CUDA(cudaGetLastError());
        in1 = !in1;
    }
    *result_in_1 = in1;
    return TQP_OK;
}

}  // namespace tqp
