// Radix-partitioned joined aggregation: the join -> group-by of a plan with
// the aggregation moved from L2 atomics into shared memory.
//
// The paper's hash join (Section 5.3) leaves partitioned joins for build
// sides beyond on-chip capacity as future work.  Here the partitioning is on
// the probe side, by the joined row's dense group id: every aggregate update
// of a joined row otherwise costs random 8-byte reductions in L2, whose rate
// (about 2.1e11 per second on GB300, measured by tqp_measure_l2_red) bounds
// the fused probe no matter how the table is laid out.  Two kernels, neither
// waiting on another CTA:
//
//   k_pj_scatter  per chunk of kPjChunk fact rows: evaluate the predicates,
//                 probe the build table, and for a row whose key has one build
//                 row (the slot holds that row's dense group id) compute its
//                 aggregate values; a shared-memory counting sort groups the
//                 chunk's joined rows by partition (group id >> shift), and the
//                 chunk is written out contiguously -- its records in
//                 partition order plus each partition's start (seg).  Rows of
//                 keys with several build rows add to their groups directly
//                 (L2 reductions, one per build row and accumulator).
//   k_pj_agg      per (partition, slice of chunks): the partition's 2^shift
//                 groups as a shared-memory table; every record of the slice
//                 is added with shared-memory atomics, then each non-empty
//                 group is added to the global group table once.
//
// Results are the exact integer sums of the plan (addition commutes), so
// they equal the fused probe's bit for bit.
#pragma once

#include "group.cuh"
#include "join.cuh"

namespace tqp {

constexpr int kPjThreads = 256;
constexpr int kPjRowsPerThread = 8;
constexpr int kPjChunk = kPjThreads * kPjRowsPerThread;  // rows per chunk (record offsets fit 16 bits)
constexpr int kPjMaxParts = 1024;
constexpr int kPjVals = 2;                                // sums per record (after the implicit count)
constexpr int kPjAggThreads = 512;
constexpr int kPjAggUnroll = 8;                           // records per lane in flight in k_pj_agg
constexpr int kPjTableBytes = 96 * 1024;                  // shared-memory group table of k_pj_agg
constexpr int kPjConds = TQP_MAX_PREDS;

struct PjCol {
    const unsigned char* p;
    int32_t type;
    int32_t pad;
};

// a row passes iff ((u64)(x - lo) <= span) != negate
struct PjCond {
    const unsigned char* p;
    int32_t type;
    int32_t negate;
    int64_t lo;
    uint64_t span;
};

// one affine factor a * x + b (kind as in ProdForm); p = nullptr: the constant b
struct PjFactor {
    const unsigned char* p;
    int32_t type;
    int32_t kind;
    int64_t a;
    int64_t b;
};

struct PartJoinArgs {
    long long n;          // fact rows
    int32_t ncond;
    int32_t nval;         // sums per record: S.nacc - 1 (<= kPjVals)
    int32_t has_sum;      // ungrouped SUM over joined rows
    int32_t shift;        // group g belongs to partition g >> shift
    int32_t nparts;       // partitions the scatter sorts into (groups <= nparts << shift)
    int32_t pad;
    PjCond cond[kPjConds];
    PjCol fk;
    PjFactor f[kPjVals][2];  // sum a = f[a][0] * f[a][1]
    PjFactor fs[2];          // the ungrouped sum
    JoinHT H;
    const uint32_t* next;    // chained build: next dim row of the same key
    const uint32_t* dgs;     // dim row -> dense group id
    GroupSpec S;             // dense group accumulators (count first)
    long long nchunks;
    uint16_t* rec_g;         // [nchunks * kPjChunk]: group id within its partition
    long long* rec_v;        // [nval][nchunks * kPjChunk]: the record's sums
    uint16_t* seg;           // [nchunks][nparts + 1]: partition starts within the chunk
    unsigned long long* acc; // [0] joined, [1] sum, [2] passing fact rows, [3] finished scatter blocks (zeroed)
    int64_t* d_num_joined;
    int64_t* d_sum;
    int64_t* d_num_rows;
};

}  // namespace tqp
