// Tensor-core (tcgen05) forms of the fused step: operand tables and launch.
#pragma once
#include <cuda.h>
#include <vector>

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

// For the multi-channel batch (single-CTA layout only, n <= 32):
bool tc_encode_state_map(CUtensorMap *m, const float *S, size_t nsites, int n);
bool tc_table_maps(const rtlb_ctx *c, CUtensorMap *zhi, CUtensorMap *zlo, const float **fwd);
bool tc_pure_tiles(const rtlb_ctx *c, std::vector<int> &out);      // tile | class << 24
void tc_mixed_list(const rtlb_ctx *c, const int **list, int *count);
}  // namespace rtlb
