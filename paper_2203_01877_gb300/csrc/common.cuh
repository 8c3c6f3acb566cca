// Device-side building blocks shared by the libtqp kernels (sm_103a).
//
//  * inline-PTX wrappers for mbarriers and bulk asynchronous (TMA engine)
//    global->shared copies,
//  * bounded spin waits that latch an error instead of hanging,
//  * typed column loads widened to int64,
//  * the postfix expression evaluator (register stack, no local memory),
//  * packed group keys and integer hashing.
#pragma once

#ifdef __CUDACC_RTC__
// Runtime compilation of query-specialised kernels (jit.cu): the fixed-width
// types and limits without the host headers.
typedef signed char int8_t;
typedef unsigned char uint8_t;
typedef short int16_t;
typedef unsigned short uint16_t;
typedef int int32_t;
typedef unsigned int uint32_t;
typedef long long int64_t;
typedef unsigned long long uint64_t;
typedef unsigned long long uintptr_t;
typedef unsigned long size_t;
#define INT_MAX 2147483647
#define INT_MIN (-INT_MAX - 1)
#define LLONG_MIN (-9223372036854775807LL - 1)
#else
#include <climits>
#include <cstdint>
#include <cuda_runtime.h>
#endif

#include "../../include/tqp.h"

namespace tqp {

constexpr int kWarp = 32;

// ---- error latch ---------------------------------------------------------
// Every device-side error goes to one int in scratch: the first one wins.
__device__ __forceinline__ void latch_error(int* err, int code) {
    if (err) atomicCAS(err, 0, code);
}
__device__ __forceinline__ int read_error(const int* err) {
    return err ? *(volatile const int*)err : 0;
}

// ---- relaxed gpu-scope 64-bit load/store (look-back status words) --------
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// ---- shared-memory addresses and mbarriers -------------------------------
// Fire-and-forget 64-bit add to global memory (a RED, no value returned).
// Accumulator pointers often come from shared memory (staged kernel
// arguments), where the compiler cannot tell that they address global memory
// and would otherwise emit a generic atomic that returns the old value.
__device__ __forceinline__ void red_add_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "l"(v));
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Arrive once and announce `bytes` of asynchronous transactions.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// Non-blocking test of phase completion (never suspends the thread, so a
// bounded number of polls is a bounded time).
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with parity `parity` to complete; false after `cap`
// polls (each poll sleeps at most ~256 ns, so cap = 2^22 is about a second).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long cap) {
    for (long long i = 0; i < cap; ++i) {
        if (mbar_test_wait(bar, parity)) return true;
        if (i >= 16) __nanosleep(i < 1024 ? 32 : 256);
    }
    return false;
}

// L2 policy for data read exactly once: evicted first, so streaming a large
// table does not push hash tables, masks and accumulators out of L2.
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// Bulk asynchronous copy global -> shared (TMA engine, non-tensor form).
// dst, src 16-byte aligned; bytes a positive multiple of 16.  Completion is
// signalled as transaction bytes on `bar`; `policy` is an L2 cache policy.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
        : "memory");
}

// Sum of a signed 64-bit value over the lanes in `peers` (every lane of
// `peers` calls this with the same mask): three 21/21/22-bit limbs, each
// summed exactly in 32 bits by the warp reduction unit, recombined mod 2^64.
__device__ __forceinline__ long long group_sum_i64(uint32_t peers, long long x) {
    const unsigned lo = static_cast<unsigned>(x) & 0x1FFFFFu;
    const unsigned mid = static_cast<unsigned>(x >> 21) & 0x1FFFFFu;
    const int hi = static_cast<int>(x >> 42);
    const unsigned slo = __reduce_add_sync(peers, lo);
    const unsigned smid = __reduce_add_sync(peers, mid);
    const int shi = __reduce_add_sync(peers, hi);
    return static_cast<long long>(static_cast<unsigned long long>(slo) + (static_cast<unsigned long long>(smid) << 21) +
                                  (static_cast<unsigned long long>(static_cast<long long>(shi)) << 42));
}

// Named barrier over `nthreads` threads (id 1..15; 0 is __syncthreads).
__device__ __forceinline__ void named_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Warp-aggregated ticket: the lanes with `want` get consecutive positions
// from `counter` with one atomic per warp (all 32 lanes must call it).
__device__ __forceinline__ long long warp_claim(unsigned long long* counter, bool want) {
    const uint32_t m = __ballot_sync(0xffffffffu, want);
    unsigned long long base = 0;
    if ((threadIdx.x % kWarp) == 0 && m) base = atomicAdd(counter, static_cast<unsigned long long>(__popc(m)));
    base = __shfl_sync(0xffffffffu, base, 0);
    return want ? static_cast<long long>(base + __popc(m & lanemask_lt())) : -1;
}

// ---- typed loads ------------------------------------------------------------
__device__ __forceinline__ int esize_of(int type) { return type == TQP_I64 ? 8 : (type == TQP_I32 ? 4 : 1); }

__device__ __forceinline__ int64_t load_typed(const unsigned char* base, int type, int64_t i) {
    switch (type) {
        case TQP_I32: return static_cast<int64_t>(reinterpret_cast<const int32_t*>(base)[i]);
        case TQP_I64: return reinterpret_cast<const int64_t*>(base)[i];
        default: return static_cast<int64_t>(base[i]);
    }
}

__device__ __forceinline__ int64_t ldg_typed(const unsigned char* base, int type, int64_t i) {
    switch (type) {
        case TQP_I32: return static_cast<int64_t>(__ldg(reinterpret_cast<const int32_t*>(base) + i));
        case TQP_I64: return __ldg(reinterpret_cast<const long long*>(base) + i);
        default: return static_cast<int64_t>(__ldg(base + i));
    }
}

// ---- integer hashing ----------------------------------------------------------
// 64-bit finaliser (the SplitMix64 / MurMur3 fmix64 style mix): every input
// bit affects every output bit, so masked low bits index a table well.
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z ^= z >> 33;
    z *= 0xff51afd7ed558ccdULL;
    z ^= z >> 33;
    z *= 0xc4ceb9fe1a85ec53ULL;
    z ^= z >> 33;
    return z;
}

}  // namespace tqp
