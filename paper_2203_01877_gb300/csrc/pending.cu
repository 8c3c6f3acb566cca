// Entry points whose kernels are not built yet: they report UNSUPPORTED.
#include "host.h"

using namespace tqp;

extern "C" {
tqp_status tqp_groupby_agg(tqp_ctx*, const tqp_table*, const tqp_pred*, int32_t, const int32_t*, int32_t,
                           const tqp_agg*, int32_t, int64_t*, int64_t*, double*, int64_t, int64_t*, void*) {
    return fail(TQP_ERR_UNSUPPORTED, "tqp_groupby_agg not built");
}
tqp_status tqp_hash_join(tqp_ctx*, const tqp_table*, int32_t, const tqp_table*, int32_t, int32_t*, int32_t*,
                         int64_t, int64_t*, void*) {
    return fail(TQP_ERR_UNSUPPORTED, "tqp_hash_join not built");
}
tqp_status tqp_run_plan(tqp_ctx*, const tqp_plan*, const tqp_result*, void*) {
    return fail(TQP_ERR_UNSUPPORTED, "tqp_run_plan not built");
}
tqp_status tqp_run_plans(tqp_ctx*, const tqp_plan*, const tqp_result*, int32_t, void*) {
    return fail(TQP_ERR_UNSUPPORTED, "tqp_run_plans not built");
}
}
