// Tensor-core (tcgen05) forms of the fused step: operand tables and launch.
#pragma once
#include "rtlb_internal.h"

namespace rtlb {
// True when a tensor-core kernel handles n directions in this precision
// (n in {8,16,32,64}; the operands must fit in shared memory of one CTA, or of
// a CTA pair for the split-table form).
bool tc_shape_ok(int n, int precision);
// Builds the bf16 operand tables (and low parts for the split form) and the
// per-tile class lists from the float64 tables and the device class array
// (may be NULL = class 0).  No-op for the FP32 precision.
rtlb_status tc_prepare(rtlb_ctx *c, const double *tables, int n_phase, const uint8_t *dev_cls, cudaStream_t s);
// One step: the tensor-core kernel over single-class tiles, the CUDA-core
// kernel over tiles that mix phase classes.
rtlb_status tc_step(rtlb_ctx *c, const StepParams &p, cudaStream_t s);
// Reads (synchronizing `s`) and clears the device error flag of the
// tensor-core kernel; RTLB_E_TIMEOUT when a bounded wait gave up.
rtlb_status tc_check_error(rtlb_ctx *c, cudaStream_t s);
int tc_mixed_tiles(const rtlb_ctx *c);
void tc_release(rtlb_ctx *c);
}  // namespace rtlb
