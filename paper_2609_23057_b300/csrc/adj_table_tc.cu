// Tensor-core form of the adjoint's phase-table gradient:
//
//   dL/dZ_c[r][k] += sum over the sites of class c of (beta mu)[site][r] S~[site][k]
//
// (the reverse-mode counterpart of the scattering contraction of Eq. 11 / 25;
// beta mu and S~ = S^t + e come from the reverse step).  One GEMM per class
// with M = N = 4n and the sites as the reduction dimension K.
//
// Persistent kernel, one CTA per SM, each reducing a contiguous slice of
// 32-site chunks, with warp roles:
//   warps 0-15  converters: per chunk and class present (a pass), each warp
//               takes whole (operand, direction) rows of the staged chunk, one
//               site per lane (conflict-free shared-memory reads), splits the
//               four Stokes components into bf16 hi + lo and stores them as
//               8-byte pieces of two MN-major, 128-byte-swizzled operand
//               tiles, A (M = table index r) and B (N = k): a site is a K
//               index, its four components four consecutive M (N) values, so
//               no transpose is needed.  K holds the chunk's 32 sites as hi
//               (K 0..31) and then lo (K 32..63).
//   warp  16    producer: TMA loads of the chunk's rows of beta mu (or mu) and
//               S and of its coefficients into a ring of staging slots
//   warp  17    MMA issuer: the hi.hi, hi.lo and lo.hi products (two K = 16
//               steps each, float32-class) into the class's TMEM accumulator
// The operand tiles are double-buffered, so the conversion of one pass
// overlaps the MMAs of the previous one.  The class set of each chunk comes
// from a mask built once per call (k_adj_chunk_masks); a chunk whose sites mix
// classes is reduced once per class present with the other classes' sites
// zeroed in A.  At the end each CTA stores its float32 accumulators (plain
// stores, zeros for a class it did not see) into its own partial, and a second
// kernel adds the partials of all CTAs, in a fixed order, into a running sum
// kept as float32 pairs (no atomics, so the result is reproducible; float64
// arithmetic, which the per-CTA float64 slots of an earlier form used, costs
// about 30 us per step on this GPU).
//
// Needs 4n <= 128 and n_phase * 4n <= 512 TMEM columns; other shapes use the
// CUDA-core kernel.  Every wait is bounded (about 2 s): on timeout the CTA
// records an error code and skips the rest of its work.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "rtlb_internal.h"
#include "tc.h"
#include "tc_ptx.cuh"

namespace rtlb {
namespace {

using namespace tcptx;

constexpr int kChunk = 32;                       // sites per K chunk: hi and lo fill one 128-byte bf16 row
constexpr int kRows = 128;                       // operand rows (table index; zero beyond 4n)
constexpr int kConvWarps = 16;
constexpr int kProdWarp = 16, kMmaWarp = 17;
constexpr int kTT = 18 * 32;                     // threads
constexpr int kSlots = 4;                        // staging slots
constexpr uint32_t kTile = kRows * 128;          // one operand tile, 16 KB
constexpr uint32_t kBuf = 2 * kTile;             // A and B
constexpr uint32_t kRowBytes = kChunk * 16;      // one direction of one operand in a staging slot
constexpr uint32_t kStageS = 32 * kRowBytes;     // S rows follow the (up to) 32 beta mu rows
constexpr uint32_t kStageCoef = 2 * kStageS;     // coefficients {alpha_hi, alpha_lo, beta, e} of the 32 sites
constexpr uint32_t kStage = kStageCoef + kChunk * 16;
constexpr uint32_t kStageAligned = (kStage + 1023) / 1024 * 1024;
constexpr int kErrTableTimeout = 16;

// L2 prefetch of the beta mu and S rows of the next run of this many chunks
// (0 = none), issued once per run.  Measured on the 1024 x 256, n = 32
// workload (table kernel alone): 0 / 2 / 4 / 8 chunks gave 130.2 / 131.1 /
// 132.0 / 133.4 us, so none by default.
#ifndef RTLB_TABLE_PREFETCH_CHUNKS
#define RTLB_TABLE_PREFETCH_CHUNKS 0
#endif

__device__ int g_table_tc_err;

__global__ void k_adj_chunk_masks(const uint8_t *__restrict__ cls, int nsites, uint32_t *__restrict__ masks)
{
    const int nchunks = (nsites + kChunk - 1) / kChunk;
    for (int ch = blockIdx.x * blockDim.x + threadIdx.x; ch < nchunks; ch += gridDim.x * blockDim.x) {
        uint32_t m = 0u;
        const int end = min(nsites, (ch + 1) * kChunk);
        for (int s = ch * kChunk; s < end; ++s) m |= 1u << cls[s];
        masks[ch] = m;
    }
}

// Error-free float32 addition (TwoSum): s + err == a + b exactly.
__device__ __forceinline__ float two_sum(float a, float b, float &err)
{
    const float s = a + b;
    const float bp = s - a;
    err = (a - (s - bp)) + (b - bp);
    return s;
}

// acc (hi at [0, len), lo at [len, 2 len)) += sum over the partials p of
// part[p][j].  Float64 arithmetic is slow on this GPU, so the sums are kept
// as float32 pairs (hi + lo, TwoSum on every addition: about twice float32's
// precision).  A block takes 64 consecutive j (16 float4 columns); its 16
// slices of threads each sum every 16th partial (independent float4 loads)
// and the slices are combined in a fixed order, so the result does not
// depend on timing.  len is a multiple of 64 (n_phase * 4n * 4n, 4n >= 32).
constexpr int kFoldCols = 16, kFoldSlices = 16;
__global__ void __launch_bounds__(kFoldCols * kFoldSlices)
    k_adj_fold_partials(const float *__restrict__ part, int nparts, int len, float *__restrict__ acc)
{
    __shared__ float hi_s[kFoldSlices][kFoldCols * 4], lo_s[kFoldSlices][kFoldCols * 4];
    const int col = threadIdx.x % kFoldCols, slice = threadIdx.x / kFoldCols;
    for (int j0 = blockIdx.x * kFoldCols * 4; j0 < len; j0 += gridDim.x * kFoldCols * 4) {
        const int j = j0 + 4 * col;
        float h[4] = {0.f, 0.f, 0.f, 0.f}, l[4] = {0.f, 0.f, 0.f, 0.f};
        for (int p = slice; p < nparts; p += kFoldSlices) {
            const float4 v = *reinterpret_cast<const float4 *>(part + (size_t)p * len + j);
            const float x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float e;
                h[k] = two_sum(h[k], x[k], e);
                l[k] += e;
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            hi_s[slice][4 * col + k] = h[k];
            lo_s[slice][4 * col + k] = l[k];
        }
        __syncthreads();
        if (threadIdx.x < kFoldCols * 4) {
            const int jj = j0 + threadIdx.x;
            float H = acc[jj], L = acc[len + jj];
            for (int sl = 0; sl < kFoldSlices; ++sl) {
                float e;
                H = two_sum(H, hi_s[sl][threadIdx.x], e);
                L += e + lo_s[sl][threadIdx.x];
            }
            acc[jj] = H;
            acc[len + jj] = L;
        }
        __syncthreads();
    }
}

// out[j] += hi[j] + lo[j] in float64 (once per call).
__global__ void k_adj_table_finish(const float *__restrict__ acc, int len, double *__restrict__ out)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < len; j += gridDim.x * blockDim.x)
        out[j] += (double)acc[j] + (double)acc[len + j];
}

// TMA load of a chunk's rows of beta mu (or nu) or S.  With
// RTLB_TABLE_LOAD_KEEP the lines keep normal L2 priority (the reverse step
// that follows reads the same data), otherwise they are marked evict-first.
#ifndef RTLB_TABLE_LOAD_KEEP
#define RTLB_TABLE_LOAD_KEEP 1
#endif
__device__ __forceinline__ void load_rows(uint32_t dst, const CUtensorMap *map, uint32_t bar, int x)
{
#if RTLB_TABLE_LOAD_KEEP
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(0)
        : "memory");
#else
    tma_load_2d(dst, map, bar, x, 0);
#endif
}

// MN-major, 128-byte-swizzled operand tile of 128 MN values x 64 K values
// (bf16): K groups of 8 (2048 bytes each) hold two atoms of 64 MN values (8 K
// rows of 128 bytes, the 16-byte chunks of row k XOR k % 8).  Byte offset of
// the four MN values 4 d .. 4 d + 3 at K index k.
__device__ __forceinline__ uint32_t mn_off4(int d, int k)
{
    return (uint32_t)(k >> 3) * 2048u + (uint32_t)(d >> 4) * 1024u + (uint32_t)(k & 7) * 128u +
           ((uint32_t)(((d & 15) >> 1) ^ (k & 7)) << 4) + ((uint32_t)(d & 1) << 3);
}

// Descriptor of such a tile: leading byte offset 1024 (next MN atom), stride
// byte offset 2048 (next K group of 8), 128-byte swizzle.
__device__ __forceinline__ uint64_t mn_desc(uint32_t saddr)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(1024 >> 4) << 16) | ((uint64_t)(2048 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__global__ void __launch_bounds__(kTT, 1)
    k_adj_table_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmS,
                   const __grid_constant__ CUtensorMap tmC, const uint8_t *__restrict__ cls,
                   const uint32_t *__restrict__ chunk_mask, float *__restrict__ part, int nsites, int n,
                   int n_phase, uint32_t tcols, int beta_scale)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023u)) & 1023u);
    uint8_t *ops = smem;                                                 // [2] x (A, B) operand tiles
    uint8_t *stage = smem + 2 * kBuf;                                    // [kSlots] staging slots
    uint64_t *bars = reinterpret_cast<uint64_t *>(stage + kSlots * kStageAligned);
    uint64_t *st_full = bars;                  // [kSlots] TMA bytes landed
    uint64_t *st_empty = st_full + kSlots;     // [kSlots] every converter warp is done with the slot
    uint64_t *op_full = st_empty + kSlots;     // [2] every converter warp wrote its rows of the buffer
    uint64_t *done = op_full + 2;              // [2] the MMAs reading the buffer completed
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int N4 = 4 * n;
    int *err = &g_table_tc_err;

    // operand tiles start at zero: rows 4n .. 127 of A are never written
    for (uint32_t o = (uint32_t)tid * 16u; o < 2 * kBuf; o += kTT * 16u)
        *reinterpret_cast<uint4 *>(smem + o) = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) {
        for (int k = 0; k < kSlots; ++k) {
            mbar_init(smem_u32(&st_full[k]), 1);
            mbar_init(smem_u32(&st_empty[k]), kConvWarps);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&op_full[b]), kConvWarps);
            mbar_init(smem_u32(&done[b]), 1);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kMmaWarp) tmem_alloc(smem_u32(tmem_slot), tcols);
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int nchunks = (nsites + kChunk - 1) / kChunk;
    const int c_begin = (int)((long long)nchunks * blockIdx.x / gridDim.x);
    const int c_end = (int)((long long)nchunks * (blockIdx.x + 1) / gridDim.x);
    const uint32_t stage_tx = 2u * (uint32_t)n * kRowBytes + kChunk * 16u;
    unsigned seen = 0u;                            // classes with an accumulator (MMA thread and, at the end, everyone)
    bool ok = true;

    if (warp == kProdWarp) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            int it = 0;
            for (int ch = c_begin; ch < c_end && ok; ++ch, ++it) {
                const int slot = it % kSlots;
                if (it >= kSlots)
                    ok = mbar_wait(smem_u32(&st_empty[slot]), ((it / kSlots) - 1) & 1, abort_flag, err, kErrTableTimeout);
                if (!ok) break;
                const uint32_t fb = smem_u32(&st_full[slot]);
                const uint32_t base = smem_u32(stage + slot * kStageAligned);
                mbar_expect_tx(fb, stage_tx);
                load_rows(base, &tmA, fb, 4 * ch * kChunk);
                load_rows(base + kStageS, &tmS, fb, 4 * ch * kChunk);
                tma_load_2d(base + kStageCoef, &tmC, fb, 0, ch * kChunk);
                if (RTLB_TABLE_PREFETCH_CHUNKS > 0 && it % RTLB_TABLE_PREFETCH_CHUNKS == 0) {
                    // the next run of chunks into L2 together: each direction's
                    // rows of beta mu and S then come from DRAM as runs of
                    // RTLB_TABLE_PREFETCH_CHUNKS x 512 bytes
                    for (int k = RTLB_TABLE_PREFETCH_CHUNKS; k < 2 * RTLB_TABLE_PREFETCH_CHUNKS; ++k)
                        if (ch + k < c_end) {
                            tma_prefetch_2d(&tmA, 4 * (ch + k) * kChunk, 0);
                            tma_prefetch_2d(&tmS, 4 * (ch + k) * kChunk, 0);
                        }
                }
            }
            // every load issued has landed before the CTA leaves (bounded)
            for (int k = 0; k < kSlots && k < it; ++k) {
                const int i2 = it - 1 - k, slot = i2 % kSlots;
                const unsigned long long t0 = global_ns();
                while (!mbar_try(smem_u32(&st_full[slot]), (i2 / kSlots) & 1) && global_ns() - t0 < kTimeoutNs) {
                }
            }
        }
    } else if (warp == kMmaWarp) {
        // ---------------------------------------------------------- MMA issuer
        if (lane == 0) {
            // both operands MN-major (transpose bits 15 and 16)
            const uint32_t idesc = idesc_bf16(kRows, N4) | (1u << 15) | (1u << 16);
            uint32_t pass = 0;
            unsigned mask_next = c_begin < c_end ? chunk_mask[c_begin] : 0u;
            for (int ch = c_begin; ch < c_end && ok; ++ch) {
                const unsigned mask = mask_next;
                if (ch + 1 < c_end) mask_next = chunk_mask[ch + 1];
                for (int c = 0; c < n_phase && ok; ++c) {
                    if (!(mask & (1u << c))) continue;
                    const int b = (int)(pass & 1u);
                    ok = mbar_wait(smem_u32(&op_full[b]), (pass >> 1) & 1u, abort_flag, err, kErrTableTimeout);
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t acc = tmem + (uint32_t)(c * N4);
                    uint32_t accum = (seen >> c) & 1u;
                    const uint64_t a0 = mn_desc(smem_u32(ops + b * kBuf)), b0 = mn_desc(smem_u32(ops + b * kBuf + kTile));
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk) {
                        // 4096 bytes (two K groups) per K = 16 step; the lo half starts at K = 32 (8192 bytes)
                        const uint64_t ah = a0 + 256 * kk, al = a0 + 512 + 256 * kk, bh = b0 + 256 * kk,
                                       bl = b0 + 512 + 256 * kk;
                        mma_bf16(acc, ah, bh, idesc, accum);
                        mma_bf16(acc, ah, bl, idesc, 1u);
                        mma_bf16(acc, al, bh, idesc, 1u);
                        accum = 1u;
                    }
                    mma_commit(smem_u32(&done[b]));
                    seen |= 1u << c;
                    ++pass;
                }
            }
            // every MMA issued has completed before TMEM is read and freed
            if (pass > 0u) {
                const int b = (int)((pass - 1u) & 1u);
                const uint32_t par = ((pass - 1u) >> 1) & 1u;
                const unsigned long long t0 = global_ns();
                while (!mbar_try(smem_u32(&done[b]), par) && global_ns() - t0 < kTimeoutNs) {
                }
                if (!mbar_try(smem_u32(&done[b]), par)) ok = false;
            }
        }
    } else {
        // ----------------------------------------------------------- converter
        uint32_t pass = 0;
        const int tasks = 2 * n;                   // (operand, direction) rows per pass
        int it = 0;
        unsigned mask_next = c_begin < c_end ? chunk_mask[c_begin] : 0u;
        for (int ch = c_begin; ch < c_end && ok; ++ch, ++it) {
            const int slot = it % kSlots;
            const unsigned mask = mask_next;
            if (ch + 1 < c_end) mask_next = chunk_mask[ch + 1];
            const bool single = (mask & (mask - 1u)) == 0u;
            const int site = ch * kChunk + lane;
            const int my_cls = (!single && site < nsites) ? (int)__ldg(cls + site) : -1;
            ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&st_full[slot]), (it / kSlots) & 1, abort_flag, err,
                                                   kErrTableTimeout));
            if (!ok) break;
            const uint8_t *st = stage + slot * kStageAligned;
            const float4 cf = *reinterpret_cast<const float4 *>(st + kStageCoef + lane * 16);   // {., ., beta, e}
            for (int c = 0; c < n_phase && ok; ++c) {
                if (!(mask & (1u << c))) continue;
                const int b = (int)(pass & 1u);
                // the MMAs of the pass two before this one (same buffer) completed
                if (pass >= 2u)
                    ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&done[b]), ((pass >> 1) & 1u) ^ 1u, abort_flag,
                                                           err, kErrTableTimeout));
                if (!ok) break;
                uint8_t *A = ops + b * kBuf;
                const float keep = (single || my_cls == c) ? (beta_scale ? cf.z : 1.f) : 0.f;
                // up to four (operand, direction) rows per warp (2n <= 64 rows,
                // 16 warps)
#pragma unroll
                for (int jt = 0; jt < 4; ++jt) {
                    const int t = warp + kConvWarps * jt;
                    if (t >= tasks) break;
                    const int o = t >= n ? 1 : 0, d = t - o * n;
                    float4 x = *reinterpret_cast<const float4 *>(st + o * kStageS + d * kRowBytes + lane * 16);
                    if (o == 0) {
                        x.x *= keep;
                        x.y *= keep;
                        x.z *= keep;
                        x.w *= keep;
                    } else {
                        x.x += cf.w;                                   // S~: emission on I
                    }
                    const uint32_t hi0 = pack_bf16(x.x, x.y), hi1 = pack_bf16(x.z, x.w);
                    const uint32_t lo0 = pack_bf16(x.x - __uint_as_float(hi0 << 16), x.y - __uint_as_float(hi0 & 0xFFFF0000u));
                    const uint32_t lo1 = pack_bf16(x.z - __uint_as_float(hi1 << 16), x.w - __uint_as_float(hi1 & 0xFFFF0000u));
                    uint8_t *tile = A + (uint32_t)o * kTile;
                    const uint32_t off = mn_off4(d, lane);                 // K = site (hi)
                    *reinterpret_cast<uint2 *>(tile + off) = make_uint2(hi0, hi1);
                    *reinterpret_cast<uint2 *>(tile + off + 4u * 2048u) = make_uint2(lo0, lo1);   // K = 32 + site (lo)
                }
                fence_proxy_async();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&op_full[b]));
                seen |= 1u << c;
                ++pass;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&st_empty[slot]));
        }
    }

    // the MMA thread drained its MMAs; everyone agrees on the outcome
    const bool all_ok = __syncthreads_and(ok) != 0;
    tc_fence_after();
    if (all_ok && warp < kConvWarps) {
        // warps w, w + 4, w + 8, w + 12 read the same lanes (rows r), each a
        // quarter of the columns (16 at least)
        const int q = warp & 3, qp = warp >> 2;
        const int r = q * 32 + lane;
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        const int cw = N4 / 4 >= 16 ? N4 / 4 : 16;        // columns per quarter
        for (int c = 0; c < n_phase; ++c) {
            float *dst = part + ((size_t)blockIdx.x * n_phase + c) * (size_t)N4 * N4;
            for (int col = qp * cw; col < (qp + 1) * cw && col < N4; col += 16) {
                float v[16];
                if (seen & (1u << c)) {
                    tmem_ld16(tmem + lane_base + (uint32_t)(c * N4 + col), v);
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] = 0.f;
                }
                if (r < N4) {
                    float4 *o4 = reinterpret_cast<float4 *>(dst + (size_t)r * N4 + col);
#pragma unroll
                    for (int j = 0; j < 4; ++j) o4[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                }
            }
        }
    } else if (!all_ok && tid == 0) {
        atomicOr(&g_table_tc_err, kErrTableTimeout);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp) tmem_dealloc(tmem, tcols);
}

}  // namespace

bool adjoint_table_tc_supported(int n, int n_phase)
{
    const int N4 = 4 * n;
    return (N4 == 32 || N4 == 64 || N4 == 128) && n_phase * N4 <= 512;
}

cudaError_t launch_adjoint_chunk_masks(const uint8_t *cls, int nsites, uint32_t *masks, cudaStream_t s)
{
    const int nchunks = (nsites + kChunk - 1) / kChunk;
    k_adj_chunk_masks<<<std::min((nchunks + 255) / 256, 148 * 8), 256, 0, s>>>(cls, nsites, masks);
    return cudaGetLastError();
}

size_t adjoint_chunk_masks_bytes(int nsites) { return (size_t)((nsites + kChunk - 1) / kChunk) * sizeof(uint32_t); }

cudaError_t launch_adjoint_table_tc(const AdjointParams &p, double *slots, int nslots, cudaStream_t s)
{
    if (!p.chunk_mask || !p.table_part || !p.table_acc || p.n > 32) return cudaErrorInvalidValue;
    const int N4 = 4 * p.n, nsites = p.nx * p.nz;
    uint32_t tcols = 32;
    while (tcols < (uint32_t)(p.n_phase * N4)) tcols <<= 1;
    CUtensorMap tmA, tmS, tmC;
    if (!tc_encode_f32_2d(&tmA, p.beta_mu, (uint64_t)nsites * 4, (uint64_t)p.n, kChunk * 4, (uint32_t)p.n) ||
        !tc_encode_f32_2d(&tmS, p.S, (uint64_t)nsites * 4, (uint64_t)p.n, kChunk * 4, (uint32_t)p.n) ||
        !tc_encode_f32_2d(&tmC, reinterpret_cast<const float *>(p.coef), 4, (uint64_t)nsites, 4, kChunk))
        return cudaErrorInvalidValue;
    const size_t smem = 2 * (size_t)kBuf + kSlots * (size_t)kStageAligned + 128 + 1024;
    static bool attr = false;
    if (!attr) {
        const cudaError_t e = cudaFuncSetAttribute(k_adj_table_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int grid = std::min(nslots, (nsites + kChunk - 1) / kChunk);
    k_adj_table_tc<<<grid, kTT, smem, s>>>(tmA, tmS, tmC, p.cls, p.chunk_mask, p.table_part, nsites, p.n, p.n_phase,
                                          tcols, p.beta_scale);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the partials of this launch into the running float32-pair sum
    const int len = p.n_phase * N4 * N4;
    k_adj_fold_partials<<<std::min(len / (kFoldCols * 4), 148 * 8), kFoldCols * kFoldSlices, 0, s>>>(p.table_part, grid,
                                                                                                      len, p.table_acc);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_table_tc_finish(const float *acc, int len, double *slot0, cudaStream_t s)
{
    k_adj_table_finish<<<std::min((len + 255) / 256, 148 * 4), 256, 0, s>>>(acc, len, slot0);
    return cudaGetLastError();
}

// Nonzero when a table-gradient kernel gave up waiting since the last call
// (the flag is cleared).
int adjoint_table_tc_take_error()
{
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_table_tc_err, sizeof(int)) != cudaSuccess) return -1;
    if (v) {
        const int z = 0;
        cudaMemcpyToSymbol(g_table_tc_err, &z, sizeof(int));
    }
    return v;
}

}  // namespace rtlb
