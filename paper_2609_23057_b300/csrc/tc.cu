// Tensor-core forms of the fused step (placeholder until the tcgen05 kernel lands).
#include "tc.h"

namespace rtlb {
rtlb_status tc_prepare_tables(rtlb_ctx *c, const double *, int, cudaStream_t)
{
    if (c->opt.precision == RTLB_PREC_FP32) return RTLB_OK;
    c->err = "tensor-core precision forms are not built yet";
    return RTLB_E_UNSUPPORTED;
}
rtlb_status tc_step(rtlb_ctx *c, const StepParams &, cudaStream_t)
{
    c->err = "tensor-core precision forms are not built yet";
    return RTLB_E_UNSUPPORTED;
}
void tc_release(rtlb_ctx *) {}
}  // namespace rtlb
