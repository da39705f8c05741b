// Device code shared by the tensor-core step kernels (single lattice, CTA
// pair, and the multi-channel batch): tile geometry, warp roles, error codes
// and the converter routine.
#pragma once
#include <cuda_fp8.h>

#include "step_common.cuh"
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
// gather form (bilinear streaming): a staging slot holds four directions, each
// the window of the previous step's P that a 128-site row tile's taps read --
// two lattice rows of 129 sites, copied as one TMA box of {G sites x 4 floats,
// kGatherCols / G site groups, 2 rows} from the first multiple of G at or
// below the first tap, at a 128-byte aligned pitch (G =
// RTLB_TC_GATHER_SITES).  Measured at 2048^2, n = 32 (bf16): 1.337 ms per
// step with G = 4, 1.368 with G = 2, 1.346 with G = 8, 1.75 ms for three boxes
// of 43 sites x 2 rows per direction.
#ifndef RTLB_TC_GATHER_SITES
#define RTLB_TC_GATHER_SITES 4
#endif
constexpr int kGatherDirs = 4;
constexpr int kGatherSites = RTLB_TC_GATHER_SITES;                 // sites per TMA box row
constexpr int kGatherCols = (kTileM + 1 + kGatherSites - 1 + kGatherSites - 1) / kGatherSites * kGatherSites;
constexpr uint32_t kGatherBoxBytes = 2u * kGatherCols * 16u;
constexpr uint32_t kGatherDirBytes = (kGatherBoxBytes + 127u) & ~127u;
constexpr uint32_t kGatherStageBytes = kGatherDirs * kGatherDirBytes;
constexpr uint32_t kGatherStageTx = kGatherDirs * kGatherBoxBytes;   // bytes the TMA delivers per slot

// Byte offset of window row `row`, column `col` (0..128 from the first site
// the taps read, which sits `lead` sites after the box's first site).
__device__ __forceinline__ uint32_t gather_window_offset(int row, int col, int lead)
{
    return (uint32_t)row * (kGatherCols * 16u) + (uint32_t)(col + lead) * 16u;
}

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
    // gather form only: the previous step's P (direction-major, read at the
    // lattice edge, where taps take the ghost rule)
    const float *P = nullptr;
};

// Bilinear taps of every direction for the gather form, passed as a kernel
// parameter (__grid_constant__) so that the warp-uniform reads hit the
// constant cache: direction d reads P at (x - n0x[d] - bx, z - n0z[d] - bz)
// with weight w[d][bx + 2 bz] (the tap order of Eq. 34's stencil product).
constexpr int kTcMaxDirs = 64;
struct GatherTaps {
    float4 w[kTcMaxDirs];
    int8_t n0x[kTcMaxDirs], n0z[kTcMaxDirs];
    int reach_x = 0, reach_z = 0;   // largest |tap offset| over the directions, per axis
};

// Whether the window values serve every tap of the row tile starting at
// (x0, z) as they are: taps inside the lattice, or beyond a vacuum side,
// whose ghost value (zero) is what the TMA fills outside the lattice -- a
// source beyond two sides takes the top / bottom side's rule, and a tile
// within reach of any other side fails the test.  Uniform over the CTA.
__device__ __forceinline__ bool gather_interior_tile(const GatherTaps &gt, int bcbits, int nx, int nz, int x0, int z)
{
    const bool left = bc_of(bcbits, RTLB_SIDE_LEFT) != RTLB_BC_VACUUM && x0 < gt.reach_x;
    const bool right = bc_of(bcbits, RTLB_SIDE_RIGHT) != RTLB_BC_VACUUM && x0 + kTileM - 1 + gt.reach_x >= nx;
    const bool bottom = bc_of(bcbits, RTLB_SIDE_BOTTOM) != RTLB_BC_VACUUM && z < gt.reach_z;
    const bool top = bc_of(bcbits, RTLB_SIDE_TOP) != RTLB_BC_VACUUM && z + gt.reach_z >= nz;
    return !(left || right || bottom || top);
}

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

struct GatherGeom {
    int nx, nz, bcbits;
    const float4 *P, *inflow;   // the previous step's P; inflow [4][n]
};

// Gather form of convert_tile (bilinear streaming, Eq. 33-38).  The step's
// input is the previous step's post-collision field P; S~ of (site, d) is the
// four-tap sum of P, formed here from the two-row window that the producer
// staged for direction d (tap (bx, bz) at window row 1 - bz, column
// r + 1 - bx) -- the same sum, in the same order, as the two-pass form's
// gather kernel.  Outside the lattice the TMA fills zeros, the ghost value of
// a vacuum side; in a tile within reach of another side (`edge`) the group
// first writes the ghost values (inflow, or the periodic image) into the
// window's entries outside the lattice and meets on fill_bar[grp].  The taps
// come from `gt` (forward taps: n0 and n0 + 1 per axis).  Each 64-wide K chunk
// c (16 directions) comes in four slots of four directions; group grp takes
// slots 4c + 2 grp and 4c + 2 grp + 1 (its directions 16c + 8 grp ... + 7, the
// same as in convert_tile), so the A rows it writes are the same.  Requires
// n % 16 == 0 and tiles that are row segments (nx % 128 == 0); x, z: the
// coordinates of this thread's site; fq: this group's count of fill_bar
// phases.
template <bool ALO>
__device__ __forceinline__ bool convert_tile_gather(const float4 cf, const float *fwd, int r, int lane, int grp, int n,
                                                    int stages, uint32_t &gq, int i, uint32_t acc, uint8_t *sA,
                                                    uint8_t *sAlo, uint8_t *sStage, uint64_t *st_full,
                                                    uint64_t *st_empty, uint64_t *a_empty, uint64_t *fill_bar,
                                                    uint32_t &fq, uint32_t a_chunk, const GatherGeom g,
                                                    const GatherTaps &gt, bool edge, int x, int z,
                                                    volatile int *abort_flag, int *err)
{
    const int C = n / 16;
    const int ring = stages / 2;
    const size_t nsites = (size_t)g.nx * g.nz;
    for (int c = 0; c < C; ++c) {
        const int d_beg = 16 * c + 8 * grp;
        uint4 packed[4], packed_lo[4];
        float fw[8];
#pragma unroll
        for (int k = 0; k < 8; k += 4) {
            const float4 f = __ldg(reinterpret_cast<const float4 *>(fwd + d_beg + k));
            fw[k] = f.x;
            fw[k + 1] = f.y;
            fw[k + 2] = f.z;
            fw[k + 3] = f.w;
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t local = gq++;
            const int s = ring_slot(grp, local, ring);
            if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(&st_full[s]), (local / (uint32_t)ring) & 1, abort_flag, err,
                                                   kErrTimeoutConverter)))
                return false;
            uint8_t *stg = sStage + (size_t)s * kGatherStageBytes;
            if (edge) {
                // ghost values into the four windows' entries outside the lattice
                const int x0 = x - r;
#pragma unroll 1
                for (int e = 0; e < kGatherDirs; ++e) {
                    const int d = d_beg + 4 * h + e;
                    const int xs0 = x0 - gt.n0x[d] - 1, xe = xs0 - (xs0 & (kGatherSites - 1)), zs0 = z - gt.n0z[d] - 1;
                    float4 *win = reinterpret_cast<float4 *>(stg + e * kGatherDirBytes);
#pragma unroll 1
                    for (int idx = r; idx < 2 * kGatherCols; idx += kTileM) {
                        const int row = idx / kGatherCols, xs = xe + idx - row * kGatherCols, zs = zs0 + row;
                        if (xs < 0 || xs >= g.nx || zs < 0 || zs >= g.nz)
                            win[idx] = source_or_ghost(g.P + (size_t)d * nsites, g.inflow, g.bcbits, g.nx, g.nz, n, d, xs,
                                                       zs);
                    }
                }
                fence_proxy_async();                        // before the next TMA into this slot
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&fill_bar[grp]));
                if (!__all_sync(0xffffffffu,
                                mbar_wait(smem_u32(&fill_bar[grp]), (fq++) & 1, abort_flag, err, kErrTimeoutConverter)))
                    return false;
            }
#pragma unroll
            for (int dp = 0; dp < 2; ++dp) {
                const int dl = 4 * h + 2 * dp;              // within this group's eight directions
                float4 v[2];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int d = d_beg + dl + e;
                    const float4 w4 = gt.w[d];
                    const int n0x = gt.n0x[d];
                    const float w[4] = {w4.x, w4.y, w4.z, w4.w};
                    const uint8_t *win = stg + (2 * dp + e) * kGatherDirBytes;
                    const int lead = (x - r - n0x - 1) & (kGatherSites - 1);   // first tap after the box's first site
                    // tap (bx, bz): window row 1 - bz, column r + 1 - bx; the
                    // loads are unconditional (in the window), the sums skip
                    // zero weights
                    float4 tv[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        tv[k] = *reinterpret_cast<const float4 *>(win +
                                                                  gather_window_offset(1 - (k >> 1), r + 1 - (k & 1), lead));
                    float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (w[k] != 0.f) axpy4(a, w[k], tv[k]);
                    v[e] = a;
                }
                v[0].x += cf.w;                             // emission (I only)
                v[1].x += cf.w;
                const float sv[8] = {v[0].x, v[0].y, v[0].z, v[0].w, v[1].x, v[1].y, v[1].z, v[1].w};
                const float g0 = fmaf(cf.z, fw[dl], cf.y), g1 = fmaf(cf.z, fw[dl + 1], cf.y);
                float init[8], bs[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    init[k] = fmaf(cf.x, sv[k], (k < 4 ? g0 : g1) * sv[k]);
                    bs[k] = cf.z * sv[k];
                }
                tmem_st8(acc + 4 * (d_beg + dl), init);
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
        if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(&a_empty[c]), (i & 1) ^ 1, abort_flag, err, kErrTimeoutConverter)))
            return false;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t gi = 4u * (uint32_t)grp + (uint32_t)k;
            const uint32_t off = c * a_chunk + r * 128u + ((gi ^ (uint32_t)(r & 7)) << 4);
            *reinterpret_cast<uint4 *>(sA + off) = packed[k];
            if (ALO) *reinterpret_cast<uint4 *>(sAlo + off) = packed_lo[k];
        }
    }
    return true;
}

// Producer side of the gather form: issues the windows of staging slot j of
// the tile whose first site is site0 -- directions 4j ... 4j + 3, one box
// each, from the multiple of kGatherSites at or below the first site the taps
// read (nx % 128 == 0).  (An L2 prefetch of the windows a few slots ahead
// measured slower at every distance tried, 4 to 12 slots.)
__device__ __forceinline__ void gather_slot_loads(const CUtensorMap *tm, const GatherTaps &gt, int nx, int site0, int j,
                                                  uint32_t dst, uint32_t bar)
{
    const int z = site0 / nx, x0 = site0 - z * nx;
#pragma unroll
    for (int e = 0; e < kGatherDirs; ++e) {
        const int d = kGatherDirs * j + e;
        const int xs = x0 - gt.n0x[d] - 1;
        tma_load_4d(dst + e * kGatherDirBytes, tm, bar, 0, (xs - (xs & (kGatherSites - 1))) / kGatherSites,
                    z - gt.n0z[d] - 1, d);
    }
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
