// Measurement kernels: the ceiling of the staged scans and the roofline of
// the joined aggregation.
//
// The joined aggregation adds each probe row's count and value into a
// per-key (or per-group) accumulator table held in L2 with fire-and-forget
// 8-byte reductions (red.global.add.u64).  Its bound is the rate at which
// the L2 completes such reductions at random addresses, not DRAM bandwidth;
// tqp_measure_l2_red measures that rate for a given table size, reductions
// per row and occupancy, so the kernel can be reported against it.  (The
// paper has no counterpart: this is a measurement entry point.)
#include "host.h"
#include "engine.cuh"

namespace tqp {

// The staged scan engine with a body that only reads what was staged: every
// 16-byte word of every stage once, folded into a checksum so nothing is
// elided.  Its rate is the ceiling of every scan body on the same columns and
// launch shape (tqp_measure_scan_rate).
struct ScanRateArgs {
    ScanGeom G;
    EngineCtl ctl;
    unsigned long long* out;  // checksum (added)
    int64_t pad;
};

struct ScanRateBody {
    static constexpr int kMinBlocks = 1;
    static constexpr int kSmemBytes = 128;
    const ScanRateArgs& A;
    unsigned int acc = 0;
    __device__ ScanRateBody(const ScanRateArgs& a, unsigned char*) : A(a) {}
    __device__ void pass1(const ScanGeom& G, const TileView& v, int cw, int lane) {
        const uint4* s = reinterpret_cast<const uint4*>(v.stage);
        const int words = G.stage_bytes / 16;
        for (int i = cw * kWarp + lane; i < words; i += kConsumers) {
            const uint4 x = s[i];
            acc += x.x ^ x.y ^ x.z ^ x.w;
        }
    }
    __device__ void chunk_end(const ScanGeom&, long long, long long, long long, int, int) {}
    __device__ void finish(const ScanGeom&, int, int lane) {
        unsigned int x = acc;  // one add per warp (not per thread, all to one word)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0 && x) atomicAdd(A.out, static_cast<unsigned long long>(x));
    }
};

__global__ void __launch_bounds__(kEngineThreads, 1) k_measure_scan(const __grid_constant__ ScanRateArgs P) {
    extern __shared__ __align__(128) unsigned char smem[];
    const ScanRateArgs& A = stage_args(P, smem + kHeaderBytes);
    ScanRateBody body(A, smem + kHeaderBytes + args_bytes<ScanRateArgs>());
    run_engine(A.G, A.ctl, body, smem, args_bytes<ScanRateArgs>());
}

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

extern "C" tqp_status tqp_measure_scan_rate(tqp_ctx* ctx, const tqp_table* t, int32_t tile_rows, int32_t stages,
                                            int32_t ctas_per_sm, unsigned long long* d_out, void* stream) {
    clear_error();
    TQP_TRY(check_ctx(ctx));
    TQP_TRY(check_table(t, "tqp_measure_scan_rate"));
    if (!d_out) return fail(TQP_ERR_INVALID_ARG, "d_out is NULL");
    if (t->num_cols > kMaxStaged) return fail(TQP_ERR_INVALID_ARG, "at most %d columns", kMaxStaged);
    if (stages < 2 || stages > kMaxStages || ctas_per_sm < 1 || ctas_per_sm > 2)
        return fail(TQP_ERR_INVALID_ARG, "stages must be in [2, %d] and ctas_per_sm in [1, 2]", kMaxStages);
    std::vector<int> cols;
    for (int c = 0; c < t->num_cols; ++c) cols.push_back(c);
    TQP_TRY(check_numeric_cols(t, cols, "tqp_measure_scan_rate"));
    TQP_TRY(check_device_cols(t, cols, "tqp_measure_scan_rate"));
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(TQP_ERR_CUDA, "cannot select device %d", ctx->device);
    arena_reset(ctx);
    ScanRateArgs A;
    memset(&A, 0, sizeof(A));
    const tqp_tuning tu{tile_rows, stages, ctas_per_sm, 1};
    size_t smem = 0;
    const int body = ScanRateBody::kSmemBytes + args_bytes<ScanRateArgs>();
    TQP_TRY(make_geom(ctx, t, cols, tu, body, &A.G, &smem));
    if (A.G.ntiles == 0) return TQP_OK;
    if (smem * ctas_per_sm > 227u * 1024u)
        return fail(TQP_ERR_UNSUPPORTED, "%d CTAs of %zu bytes do not fit one SM", ctas_per_sm, smem);
    static SmemFlags attr;
    TQP_TRY(allow_smem(ctx, reinterpret_cast<const void*>(k_measure_scan), attr));
    unsigned long long* ticket = static_cast<unsigned long long*>(arena_alloc(ctx, 256));
    if (!ticket) return arena_oom(ctx, 256);
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    TQP_CUDA(cudaMemsetAsync(ticket, 0, 256, st));
    const int grid = engine_grid(ctx, reinterpret_cast<const void*>(k_measure_scan), smem, A.G.ntiles, ctas_per_sm);
    A.ctl.ticket = ticket;
    A.ctl.err = ctx->d_err;
    A.ctl.wait_cap = ctx->wait_cap;
    A.ctl.chunk_tiles = (A.G.ntiles + grid - 1) / grid;
    A.ctl.nchunks = (A.G.ntiles + A.ctl.chunk_tiles - 1) / A.ctl.chunk_tiles;
    A.out = d_out;
    k_measure_scan<<<static_cast<unsigned>(A.ctl.nchunks), kEngineThreads, smem, st>>>(A);
    TQP_CUDA(cudaGetLastError());
    return TQP_OK;
}

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
