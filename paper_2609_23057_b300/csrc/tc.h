// Tensor-core (tcgen05) forms of the fused step: operand tables and launch.
#pragma once
#include "rtlb_internal.h"

namespace rtlb {
// Converts the float64 phase tables into the MMA operand tables (bf16, and the
// low parts for the split form) when the context's precision needs them.
rtlb_status tc_prepare_tables(rtlb_ctx *c, const double *tables, int n_phase, cudaStream_t s);
// One step with the tensor-core kernel.
rtlb_status tc_step(rtlb_ctx *c, const StepParams &p, cudaStream_t s);
void tc_release(rtlb_ctx *c);
}  // namespace rtlb
