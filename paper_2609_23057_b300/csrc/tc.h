// Tensor-core (tcgen05) forms of the fused step: operand tables and launch.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
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
// Arms the bounded-wait test hook for the next tensor-core launch (bf16-class
// kernels): CTA 0 leaves one state load unissued.  RTLB_E_STATE before the
// tables exist, RTLB_E_UNSUPPORTED for the FP8 kernel.
rtlb_status tc_arm_stall(rtlb_ctx *c);
int tc_mixed_tiles(const rtlb_ctx *c);
// True when the prepared form gathers bilinear streaming while loading (the
// bf16, bf16x2 and bf16x3 forms with nx % 128 == 0, n % 16 == 0 and room for
// four staging slots: n in {16, 32}): tc_step then takes StepParams with taps
// (S = the previous step's P).
bool tc_gather(const rtlb_ctx *c);
// Pair form and stage count of the prepared tensor-core form (false when none).
bool tc_form(const rtlb_ctx *c, int *pair, int *stages);
void tc_release(rtlb_ctx *c);

// Tensor-core reverse step of the adjoint (adj_tc.cu), 4n in {32, 64, 128}: reads
// nu^t (tensor map tmNu, direction-major) and S^t, writes nu^{t-1} pushed
// along the negated offsets (push = 1) or lambda^0 in place (push = 0), and
// adds the per-site gradient sums into g_alpha / g_beta, each [2][nsites]
// (one half per group of directions).  Tables: Z^T as bf16 hi and lo,
// [n_phase][4n][KP] (K padded with zeros to KP = 4n rounded up to 64), tensor
// maps with 4n-row boxes.  `tiles` lists
// single-class 128-site tiles sorted by class (tile | class << 24).
struct AdjTcLaunch {
    const float *S;
    const float4 *coef;
    const int *dirT;
    int bcbitsT;
    float *nu_out;
    double *g_alpha, *g_beta;
    const int *tiles;
    int n_tiles;
    int nx, nz, n;
    int push;
    int sm_count;
};
int adjoint_tc_stages(int n);   // 0 where the form does not exist (n not in {8, 16, 32})
cudaError_t launch_adjoint_step_tc(const CUtensorMap &tmNu, const CUtensorMap &tmZhi, const CUtensorMap &tmZlo,
                                   const AdjTcLaunch &a, cudaStream_t s);
int adjoint_step_tc_take_error();
// float32 2D tensor map (rows of `inner` floats, `outer` rows, row stride
// inner * 4 bytes), boxes of box_inner x box_outer, no swizzle, zero fill
bool tc_encode_f32_2d(CUtensorMap *m, const float *base, uint64_t inner, uint64_t outer, uint32_t box_inner,
                      uint32_t box_outer);
// bf16 table [n_phase][N4][KP] tensor map with boxes of 64 columns x box_rows rows
bool tc_encode_table_map(CUtensorMap *m, const __nv_bfloat16 *Z, int N4, int KP, int n_phase, int box_rows);

// For the multi-channel batch (single-CTA layout only, n <= 32):
bool tc_encode_state_map(CUtensorMap *m, const float *S, size_t nsites, int n);
bool tc_table_maps(const rtlb_ctx *c, CUtensorMap *zhi, CUtensorMap *zlo, const float **fwd);
bool tc_pure_tiles(const rtlb_ctx *c, std::vector<int> &out);      // tile | class << 24
void tc_mixed_list(const rtlb_ctx *c, const int **list, int *count);
}  // namespace rtlb
