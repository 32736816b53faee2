// Split-precision tensor-core path (filled in below).
#include "lem_internal.h"

namespace lem {
struct SplitPlan {};
bool split_eligible(const lem_ctx*) { return false; }
lem_status split_prepare(lem_ctx*) { return fail(LEM_EINVAL, "split path not available"); }
lem_status split_step(lem_ctx*, double*, int) { return fail(LEM_EINVAL, "split path not available"); }
void split_destroy(lem_ctx* ctx) { delete ctx->split; ctx->split = nullptr; }
}  // namespace lem
