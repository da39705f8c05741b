// Device code shared by the tensor-core step kernels (single lattice, CTA
// pair, and the multi-channel batch): tile geometry, warp roles, error codes
// and the converter routine.
#pragma once
#include <cuda_fp8.h>

#include "tc_ptx.cuh"

namespace rtlb {
namespace tccommon {

using namespace tcptx;

constexpr int kTileM = 128;
constexpr int kWarps = 18;
constexpr int kEpiWarps = 8;
constexpr int kConvWarp0 = 8;
constexpr int kConvWarps = 8;                       // two groups of four (one TMEM lane quadrant each)
constexpr int kProdWarp = 16;
constexpr int kMmaWarp = 17;
constexpr int kThreads = kWarps * 32;
constexpr int kDirsPerStage = 8;                    // directions per state chunk
constexpr int kStageBytes = kDirsPerStage * kTileM * 16;
constexpr int kHalfSites = 64;                      // sites per TMA box row (256 floats)
constexpr int kSmemLimit = 232448;                  // max dynamic smem per block


// Arguments of the tensor-core step kernels.
struct TcParams {
    const float4 *coef;  // {alpha_hi, alpha_lo, beta, emission}
    const int *dir;
    const float *inflow;
    float *S_new;
    const int *tiles;  // tile | class << 24
    const float *fwd;  // [n_phase][n] forward-block factors
    int n_tiles;
    int nx, nz, n;
    int bcbits;
    int *err;
    // test hook of the bounded waits: when nonzero, CTA 0 leaves the load of
    // its first staging slot unissued (nothing is then in flight for it), so
    // its converters' wait runs out and the launch reports a timeout
    int stall = 0;
};

enum ErrCode { kErrTimeoutProducer = 1, kErrTimeoutConverter = 2, kErrTimeoutMma = 4, kErrTimeoutEpilogue = 8 };


// Per-site coefficients {alpha_hi, alpha_lo, beta, e} of one tile row (zero
// past the end of the lattice).  Converters fetch them a tile ahead so the
// global-memory latency overlaps the previous tile's conversion.
__device__ __forceinline__ float4 load_coef(const float4 *coef, int site, int nsites)
{
    return site < nsites ? __ldg(coef + site) : make_float4(0.f, 0.f, 0.f, 0.f);
}

// Staging slots: each converter group owns a ring of its own, stages / 2
// slots (stages is even), and the producer fills group (j & 1)'s ring with
// slot j of every tile.  A slot therefore always has the same consumer, so a
// consumer never waits on a slot more than one phase ahead of what it has
// itself released (a shared ring fed to two groups could let one group pass a
// parity test a full phase early when the other group lags).
__device__ __forceinline__ int ring_slot(int grp, uint32_t local, int ring) { return grp * ring + (int)(local % (uint32_t)ring); }

// Converter work for one tile (one site row per thread, TMEM lane r).  The
// converter warps form two groups; each 64-wide K chunk of the A operand (16
// directions) comes in two staging slots of 8 directions, and group `grp`
// takes slot j = 2c + grp (its ring's next entry, counted in `gq`): it writes
// the float32 part (alpha_hi + alpha_lo + beta c_d) S~ of its directions into
// the TMEM accumulator, packs beta S~ to bf16 in registers and releases the
// slot, then waits for the MMA to free A chunk c and stores its half of the
// chunk's 128-byte rows.  Returns false when a bounded wait gave up.
template <bool ALO>
__device__ __forceinline__ bool convert_tile(const float4 cf, const float *fwd, int r, int lane, int grp, int n,
                                             int groups, int stages, uint32_t &gq, int i, uint32_t acc, uint8_t *sA,
                                             uint8_t *sAlo, const uint8_t *sStage, uint64_t *st_full,
                                             uint64_t *st_empty, uint64_t *a_empty, uint32_t a_chunk,
                                             volatile int *abort_flag, int *err)
{
    const int half = r / kHalfSites, hr = r % kHalfSites;
    const int C = (4 * n + 63) / 64;
    for (int c = 0; c < C; ++c) {
        const int j = 2 * c + grp;                   // this group's slot of chunk c
        const int d_beg = 8 * j;                     // its 8 directions (all < n when j < groups)
        const bool mine = j < groups;
        uint4 packed[4], packed_lo[4];
        if (mine) {
            float fw[8];
#pragma unroll
            for (int k = 0; k < 8; k += 4) {
                const float4 f = __ldg(reinterpret_cast<const float4 *>(fwd + d_beg + k));
                fw[k] = f.x;
                fw[k + 1] = f.y;
                fw[k + 2] = f.z;
                fw[k + 3] = f.w;
            }
            const int ring = stages / 2;
            const uint32_t local = gq++;
            const int s = ring_slot(grp, local, ring);
            if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(&st_full[s]), (local / (uint32_t)ring) & 1, abort_flag, err,
                                                   kErrTimeoutConverter)))
                return false;
            const float4 *stg = reinterpret_cast<const float4 *>(sStage + (size_t)s * kStageBytes) +
                                half * (kDirsPerStage * kHalfSites) + hr;
#pragma unroll
            for (int dl = 0; dl < kDirsPerStage; dl += 2) {
                const int d = d_beg + dl;
                float4 v0 = stg[dl * kHalfSites], v1 = stg[(dl + 1) * kHalfSites];
                v0.x += cf.w;                               // emission (I only)
                v1.x += cf.w;
                const float sv[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
                const float g0 = fmaf(cf.z, fw[dl], cf.y), g1 = fmaf(cf.z, fw[dl + 1], cf.y);
                float init[8], bs[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    init[k] = fmaf(cf.x, sv[k], (k < 4 ? g0 : g1) * sv[k]);   // exact float32 part
                    bs[k] = cf.z * sv[k];                                       // beta S~ (MMA operand)
                }
                tmem_st8(acc + 4 * d, init);
                uint4 hi;
                hi.x = pack_bf16(bs[0], bs[1]);
                hi.y = pack_bf16(bs[2], bs[3]);
                hi.z = pack_bf16(bs[4], bs[5]);
                hi.w = pack_bf16(bs[6], bs[7]);
                packed[dl >> 1] = hi;
                if (ALO) {
                    const __nv_bfloat162 *h2 = reinterpret_cast<const __nv_bfloat162 *>(&hi);
                    uint32_t *lw = reinterpret_cast<uint32_t *>(&packed_lo[dl >> 1]);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const float2 f = __bfloat1622float2(h2[k]);
                        lw[k] = pack_bf16(bs[2 * k] - f.x, bs[2 * k + 1] - f.y);
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&st_empty[s]));
        }
        // A chunk c is free once the previous tile's MMAs on it completed
        if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(&a_empty[c]), (i & 1) ^ 1, abort_flag, err, kErrTimeoutConverter)))
            return false;
        if (mine) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t gi = 4u * (uint32_t)grp + (uint32_t)k;
                const uint32_t off = c * a_chunk + r * 128u + ((gi ^ (uint32_t)(r & 7)) << 4);
                *reinterpret_cast<uint4 *>(sA + off) = packed[k];
                if (ALO) *reinterpret_cast<uint4 *>(sAlo + off) = packed_lo[k];
            }
        }
    }
    return true;
}

// UE8M0 exponent of a block whose largest |value| is amax (float32): the
// smallest e with amax / 2^e <= 448 (the largest finite e4m3), clamped to the
// scale range; zero and subnormal amax take the smallest scale.
__device__ __forceinline__ int block_exponent(float amax)
{
    const uint32_t bits = __float_as_uint(amax);
    const int ex = (int)((bits >> 23) & 0xFFu);
    if (ex == 0) return -127;
    const int e = ex - 127 - 8 + ((bits & 0x7FFFFFu) > 0x600000u ? 1 : 0);   // mantissa above 1.75
    return e < -127 ? -127 : e;
}

// Two e4m3 values (round to nearest even, saturating at +-448), first in the
// low byte.
__device__ __forceinline__ uint32_t e4m3x2(float lo, float hi)
{
    return (uint32_t)__nv_cvt_float2_to_fp8x2(make_float2(lo, hi), __NV_SATFINITE, __NV_E4M3);
}

}  // namespace tccommon

// 3xTF32 form (tc_tf32.cu), 4n <= 128: shared memory for a stage count and the
// launch (grid CTAs over p.tiles); tables are float32 [n_phase][4n][4n]
// holding tf32 values, tensor maps with 32-column x 4n-row boxes (SW128).
size_t tc_tf32_smem_bytes(int N4, int stages);
cudaError_t launch_step_tc_tf32(const CUtensorMap &tmS, const CUtensorMap &tmZhi, const CUtensorMap &tmZlo,
                                const tccommon::TcParams &p, int N4, int stages, int grid, cudaStream_t s);

// Split FP8 form (tc_fp8x.cu): state operand in two e4m3 terms, table in
// three (z8 [3][n_phase][4n][KP8], sfb [3][n_phase][4n][4n / 32]); TMEM
// columns it needs (<= 512), shared memory for a stage count, and the launch.
int tc_fp8x_tmem_columns(int N4, int n_phase);
size_t tc_fp8x_smem_bytes(int N4, int stages);
cudaError_t launch_step_tc_fp8x(const CUtensorMap &tmS, const CUtensorMap &tmZ, const tccommon::TcParams &p,
                                const uint8_t *sfb, int N4, int stages, int n_phase, int grid, cudaStream_t s);

// FP8 block-scaled form (tc_fp8.cu): TMEM columns it needs (D, A scales, the
// B scales of every class; must be <= 512), shared memory for a stage count,
// and the launch (grid CTAs over p.tiles, one class-sorted slice each).
int tc_fp8_tmem_columns(int N4, int n_phase);
size_t tc_fp8_smem_bytes(int N4, int stages);
cudaError_t launch_step_tc_fp8(const CUtensorMap &tmS, const CUtensorMap &tmZ, const tccommon::TcParams &p,
                               const uint8_t *sfb, int N4, int stages, int n_phase, int grid, cudaStream_t s);
}  // namespace rtlb
