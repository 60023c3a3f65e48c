// Split-BF16 block-sparse product (tensor cores).  Not built yet: the call reports it.
#include "cq_internal.cuh"

cq_status cq_bsmm_split(cq_ctx *ctx, const TaskList *, double, const cq_pattern *,
                        const double *, const cq_pattern *, const double *, double,
                        const cq_pattern *, double *)
{
    return cq_fail(ctx, CQ_ERR_INVALID, "split-BF16 product not available in this build");
}
