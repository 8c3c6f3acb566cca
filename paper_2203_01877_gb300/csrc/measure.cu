// Measurement kernels: the roofline of the joined aggregation.
//
// The joined aggregation adds each probe row's count and value into a
// per-key (or per-group) accumulator table held in L2 with fire-and-forget
// 8-byte reductions (red.global.add.u64).  Its bound is the rate at which
// the L2 completes such reductions at random addresses, not DRAM bandwidth;
// tqp_measure_l2_red measures that rate for a given table size, reductions
// per row and occupancy, so the kernel can be reported against it.  (The
// paper has no counterpart: this is a measurement entry point.)
#include "host.h"

namespace tqp {

// Row i adds 1 to word (k * adds + 0) and i to words (k * adds + j), j >= 1,
// of key k = mix64(i ^ seed) mod nkeys: uniformly random keys, every row's
// words adjacent (one 16-byte accumulator entry for adds = 2).
__global__ void k_measure_l2_red(unsigned long long* __restrict__ table, long long nkeys, long long rows, int adds,
                                 unsigned long long seed) {
    const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < rows; i += stride) {
        const unsigned long long k = mix64(static_cast<unsigned long long>(i) ^ seed) % static_cast<unsigned long long>(nkeys);
        unsigned long long* a = table + k * static_cast<unsigned long long>(adds);
        red_add_u64(&a[0], 1ULL);
        for (int j = 1; j < adds; ++j) red_add_u64(&a[j], static_cast<unsigned long long>(i));
    }
}

}  // namespace tqp

using namespace tqp;

extern "C" tqp_status tqp_measure_l2_red(int device, unsigned long long* d_table, int64_t table_words, int64_t rows,
                                         int32_t adds_per_row, int32_t blocks_per_sm, int32_t threads,
                                         void* stream) {
    clear_error();
    if (!d_table || table_words < 1 || rows < 0 || adds_per_row < 1 || adds_per_row > 8 || table_words < adds_per_row)
        return fail(TQP_ERR_INVALID_ARG, "tqp_measure_l2_red: bad table, row or add counts");
    if (threads < 32 || threads > 1024 || threads % 32 != 0 || blocks_per_sm < 1 || blocks_per_sm > 32)
        return fail(TQP_ERR_INVALID_ARG, "tqp_measure_l2_red: bad launch shape");
    DeviceGuard g(device);
    if (!g.ok) return fail(TQP_ERR_CUDA, "cannot select device %d", device);
    int sms = 0;
    TQP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    if (rows == 0) return TQP_OK;
    k_measure_l2_red<<<sms * blocks_per_sm, threads, 0, static_cast<cudaStream_t>(stream)>>>(
        d_table, table_words / adds_per_row, rows, adds_per_row, 0x9E3779B97F4A7C15ULL);
    TQP_CUDA(cudaGetLastError());
    return TQP_OK;
}
