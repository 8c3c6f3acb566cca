// A dimension table prepared once for many joined plans (tqp_dim_prepare):
// its chained hash table and the dense group id of every row, resident in a
// long-lived region of the context's arena.
#pragma once

#include "host.h"
#include "group.cuh"
#include "join.cuh"

struct tqp_dim {
    tqp_ctx* ctx = nullptr;
    size_t top_before = 0, top_after = 0;
    tqp::JoinHT H{};                   // slots, cap, key range (direct-mapped or hashed)
    uint32_t* next = nullptr;          // chain links
    uint32_t* dgs = nullptr;           // dim row -> dense group id
    unsigned long long* dkeys = nullptr;  // [groups + 1] packed key of each dense group
    long long* d_groups = nullptr;     // device copy of `groups` (the dense count)
    long long groups = 0;
    long long nrows = 0;
    int32_t key_col = 0;
    int32_t ngc = 0;
    int32_t group_cols[TQP_MAX_GROUP_COLS] = {0, 0, 0, 0};
    const void* key_data = nullptr;    // identity of the prepared table
};

namespace tqp {

// Validate that plan p may use p->prepared (same dimension, key and group
// columns as the preparation).
tqp_status check_prepared(const tqp_ctx* ctx, const tqp_plan* p);

// Claim, number and remap the dense group ids of D's rows for the key columns
// of S (dim column indices): dgs[n], dkeys[dmax + 1], dacc[(dmax + 1) * S.nacc]
// (accumulators of the claimed ids cleared) and ndistinct[2] ([1]: the dense
// count) are the caller's; the claim table is per-call scratch.  With H set,
// unique-key slots of H receive their row's dense id.
tqp_status dense_groups_launch(tqp_ctx* ctx, const tqp_table* D, const GroupSpec& S, long long maxg,
                               const JoinHT* H, uint32_t* dgs, unsigned long long* dkeys, unsigned long long* dacc,
                               unsigned long long* ndistinct, cudaStream_t stream);

}  // namespace tqp
