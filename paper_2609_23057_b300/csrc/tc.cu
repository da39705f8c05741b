// Tensor-core (tcgen05) form of the fused collide+stream step.
//
// Per tile of 128 consecutive sites the scattering contraction of Eq. 11/25,
// Y[site][4n] = S~[site][4n] . Z_c^T, is one GEMM with M = 128, N = K = 4n.
// The state stays float32 in HBM; the tensor core sees bf16 operands and
// accumulates in float32 in tensor memory (TMEM):
//
//   D  <- alpha * S~                      (written into TMEM before the MMAs)
//   D  += (beta * S~)_bf16 . Z_bf16^T     (tcgen05.mma, K in steps of 16)
//   S_new(x + c_d, d) = D(x, d)           (epilogue: TMEM -> registers -> push)
//
// so the dominant alpha * S~ term (unscattered light) is kept exactly in
// float32 and only the scattered part passes through bf16.  BF16X3 adds the
// two cross terms of a hi+lo split of both operands.
//
// Persistent kernel, one CTA per SM, warp roles:
//   warps 0-7   epilogue   (TMEM lane quadrant = warp % 4, one site per thread,
//                           warps 4-7 take the second half of the directions)
//   warps 8-15  converter  (FP32 staging -> bf16 A operand in the 128-byte
//                           swizzled K-major layout, alpha * S~ -> TMEM; two
//                           groups of four take alternate staging slots)
//   warp  16    producer   (TMA loads of state chunks and of Z)
//   warp  17    MMA issuer (one thread; also allocates TMEM)
// Z (one phase class at a time) and the whole A operand of the current tile
// stay in shared memory; TMEM holds two accumulators so the epilogue of one
// tile overlaps the next tile's conversion and MMAs.  Tiles whose sites mix
// phase classes go to the CUDA-core kernel instead (tile-list mode).
//
// Every mbarrier wait is bounded (about 2 s); on timeout the CTA raises an
// abort flag, records an error code, drains its own TMA loads and MMAs,
// frees its TMEM and returns; the host reports RTLB_E_TIMEOUT.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <tuple>
#include <cmath>
#include <cstring>
#include <vector>

#include "step_common.cuh"
#include "tc.h"
#include "tc_ptx.cuh"
#include "tc_common.cuh"

namespace rtlb {

namespace {

using namespace tcptx;
using namespace tccommon;

struct TcState {
    int N4 = 0, KP = 0, C = 0, n_phase = 0;
    int mode = 1;                    // 1 bf16, 2 bf16 + table lo, 3 hi+lo both, 4 e4m3 block-scaled, 5 3xTF32,
                                     // 6 split e4m3 (state 2 terms, table 3 terms)
    bool pair = false;               // CTA-pair kernel (table rows split over two CTAs)
    __nv_bfloat16 *d_Zhi = nullptr;  // [n_phase][N4][KP]
    __nv_bfloat16 *d_Zlo = nullptr;
    uint8_t *d_Z8 = nullptr;         // FP8: [n_phase][N4][KP8] e4m3 (FP8X: [3][n_phase][N4][KP8], one per term)
    uint8_t *d_sfb = nullptr;        // FP8: [n_phase][N4][N4 / 32] UE8M0 block scales of the table (FP8X: [3][...])
    float *d_Zt_hi = nullptr;        // TF32X3: [n_phase][N4][N4] tf32 hi part (float32 container)
    float *d_Zt_lo = nullptr;        // TF32X3: tf32 lo part
    int *d_pure = nullptr;           // tile | class << 24, sorted by class (pairs: 2 per entry)
    int n_pure = 0;
    int *d_mixed = nullptr;          // tile indices
    int n_mixed = 0;
    float *d_fwd = nullptr;          // [n_phase][n] forward-block factors applied in float32
    int *d_err = nullptr;
    int *h_err = nullptr;
    CUtensorMap tmZhi{}, tmZlo{}, tmS[2]{};
    bool tmS_ready[2] = {false, false};
    const float *tmS_ptr[2] = {nullptr, nullptr};
    // gather form (bilinear streaming, single-CTA bf16 forms): window maps of
    // both state buffers, the taps; tiles ordered down 512-site column strips
    bool gather = false;
    GatherTaps gtaps{};
    CUtensorMap tmG[2]{};
    const float *tmG_ptr[2] = {nullptr, nullptr};
    int sm_count = 0;
    int stages = 0;
    size_t smem = 0;
    int stall_next = 0;              // test hook armed for the next launch (TcParams::stall)
};

// MODE 1: bf16 operands; 2: bf16 state operand, table as bf16 hi + lo (two
// MMAs); 3: both operands hi + lo (three MMAs).
template <int MODE, bool GATHER>
__global__ void __launch_bounds__(kThreads, 1)
    k_step_tc(const __grid_constant__ CUtensorMap tmS, const __grid_constant__ CUtensorMap tmZhi,
              const __grid_constant__ CUtensorMap tmZlo, TcParams p, int N4, int stages,
              const __grid_constant__ GatherTaps gt)
{
    // GATHER: tmS is the windows' map (see encode_gather_map), the staging
    // slots hold four directions' windows and the converters form S~ from them
    constexpr uint32_t stage_bytes = GATHER ? kGatherStageBytes : (uint32_t)kStageBytes;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023u)) & 1023u);
    constexpr bool ZLO = MODE >= 2, ALO = MODE == 3;
    const int C = (N4 + 63) / 64;                  // K chunks of 64
    const int n = p.n;
    const int nsites = p.nx * p.nz;
    const int groups = n / kDirsPerStage;          // state chunks per tile (n % 8 == 0)
    const uint32_t z_chunk = (uint32_t)N4 * 128u;  // bytes per K chunk of Z
    const uint32_t a_chunk = (uint32_t)kTileM * 128u;

    uint8_t *sZ = smem;
    uint8_t *sZlo = sZ + C * z_chunk;
    uint8_t *sA = sZlo + (ZLO ? C * z_chunk : 0);
    uint8_t *sAlo = sA + C * a_chunk;
    uint8_t *sStage = sAlo + (ALO ? C * a_chunk : 0);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sStage + (size_t)stages * stage_bytes);
    uint64_t *st_full = bars;
    uint64_t *st_empty = st_full + stages;
    uint64_t *a_empty = st_empty + stages;     // [C]
    uint64_t *t_ready = a_empty + C;           // [2]
    uint64_t *acc_full = t_ready + 2;          // [2]
    uint64_t *acc_empty = acc_full + 2;        // [2]
    uint64_t *z_full = acc_empty + 2;          // [1]
    uint64_t *drain = z_full + 1;              // [1]
    uint64_t *z_free = drain + 1;              // [1]  the resident table's last MMAs completed
    uint64_t *fill_bar = z_free + 1;           // [2]  gather form: a converter group's ghost fill done
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(fill_bar + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    int8_t *s_cx = reinterpret_cast<int8_t *>(tmem_slot + 2);   // [n]
    int8_t *s_cz = s_cx + kMaxDirs;                              // [n]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // 4n <= 128: the exact float32 part goes into its own TMEM region E (two
    // buffers after the two accumulators) and the MMAs start D from zero; the
    // epilogue adds E.  The tensor core rounds each instruction's float32 sum
    // toward zero, so an accumulator holding the unscattered light would lose
    // a fraction of an ulp of it per instruction, step after step.  At 4n =
    // 256 the two accumulators fill TMEM and the part is written into D.
    const bool sepE = N4 <= 128;
    const int need = sepE ? 4 * N4 : 2 * N4;
    const uint32_t tcols = need <= 32 ? 32u : (need <= 64 ? 64u : (need <= 128 ? 128u : (need <= 256 ? 256u : 512u)));

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(smem_u32(&st_full[s]), 1);
            mbar_init(smem_u32(&st_empty[s]), 4);
        }
        for (int c = 0; c < C; ++c) mbar_init(smem_u32(&a_empty[c]), 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&t_ready[b]), kConvWarps);
            mbar_init(smem_u32(&acc_full[b]), 1);
            mbar_init(smem_u32(&acc_empty[b]), kEpiWarps);
        }
        mbar_init(smem_u32(z_full), 1);
        mbar_init(smem_u32(drain), 1);
        mbar_init(smem_u32(z_free), 1);
        mbar_init(smem_u32(&fill_bar[0]), 4);
        mbar_init(smem_u32(&fill_bar[1]), 4);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int d = threadIdx.x; d < n; d += blockDim.x) {
        s_cx[d] = (int8_t)p.dir[d];
        s_cz[d] = (int8_t)p.dir[n + d];
    }
    if (warp == kMmaWarp) tmem_alloc(smem_u32(tmem_slot), tcols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    // contiguous slice of the (class-sorted) tile list for this CTA
    const int t_begin = (int)((long long)p.n_tiles * blockIdx.x / gridDim.x);
    const int t_end = (int)((long long)p.n_tiles * (blockIdx.x + 1) / gridDim.x);
    const int T = t_end - t_begin;

    if (warp == kProdWarp) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            const bool stall = p.stall != 0 && blockIdx.x == 0;
            int prev_cls = -1;
            uint32_t gq[2] = {0, 0}, zr = 0;
            bool ok = true;
            for (int i = 0; i < T && ok; ++i) {
                const int e = p.tiles[t_begin + i];
                const int tile = e & 0xFFFFFF, cls = e >> 24;
                if (cls != prev_cls) {
                    // the MMA thread signals z_free once per table switch, after
                    // the previous table's last MMAs (one phase per switch, so
                    // the wait cannot alias however far ahead this thread runs)
                    if (i > 0) ok = mbar_wait(smem_u32(z_free), (zr++) & 1, abort_flag, p.err, kErrTimeoutProducer);
                    if (!ok) break;
                    const uint32_t zb = smem_u32(z_full);
                    mbar_expect_tx(zb, (ZLO ? 2u : 1u) * C * z_chunk);
                    for (int c = 0; c < C; ++c) {
                        tma_load_3d(smem_u32(sZ + c * z_chunk), &tmZhi, zb, 64 * c, 0, cls);
                        if (ZLO) tma_load_3d(smem_u32(sZlo + c * z_chunk), &tmZlo, zb, 64 * c, 0, cls);
                    }
                    prev_cls = cls;
                }
                // keep the next tiles' state on its way into L2
                for (int ahead = (i == 0 ? 1 : RTLB_TC_PREFETCH_TILES); !GATHER && ahead <= RTLB_TC_PREFETCH_TILES;
                     ++ahead) {
                    if (i + ahead >= T) break;
                    const int nt = p.tiles[t_begin + i + ahead] & 0xFFFFFF;
                    for (int j = 0; j < groups; ++j)
                        for (int h = 0; h < kTileM / kHalfSites; ++h)
                            tma_prefetch_2d(&tmS, 4 * (nt * kTileM + h * kHalfSites), j * kDirsPerStage);
                }
                const int nslots = GATHER ? n / kGatherDirs : groups;
                for (int j = 0; j < nslots && ok; ++j) {
                    // gather form: slots 4c + 2 grp + {0, 1} go to group grp
                    const int gr = GATHER ? (j >> 1) & 1 : j & 1;
                    const uint32_t local = gq[gr]++;
                    const int s = ring_slot(gr, local, stages / 2);
                    ok = mbar_wait(smem_u32(&st_empty[s]), ((local / (uint32_t)(stages / 2)) & 1) ^ 1, abort_flag, p.err,
                                   kErrTimeoutProducer);
                    if (!ok) break;
                    if (stall && i == 0 && j == 0) continue;   // test hook: this load is never issued
                    const uint32_t fb = smem_u32(&st_full[s]);
                    if (GATHER) {
                        mbar_expect_tx(fb, kGatherStageTx);
                        gather_slot_loads(&tmS, gt, p.nx, tile * kTileM, j, smem_u32(sStage + (size_t)s * stage_bytes), fb);
                        continue;
                    }
                    mbar_expect_tx(fb, kStageBytes);
                    for (int h = 0; h < kTileM / kHalfSites; ++h)
                        tma_load_2d(smem_u32(sStage + (size_t)s * kStageBytes + h * (kStageBytes / 2)), &tmS, fb,
                                    4 * (tile * kTileM + h * kHalfSites), j * kDirsPerStage);
                    if (RTLB_TC_PREFETCH_SLOTS > 0) {
                        // the state chunk RTLB_TC_PREFETCH_SLOTS slots ahead, into L2
                        const int ahead = i * groups + j + RTLB_TC_PREFETCH_SLOTS;
                        const int ia = ahead / groups, ja = ahead - ia * groups;
                        if (ia < T) {
                            const int ta = p.tiles[t_begin + ia] & 0xFFFFFF;
                            for (int h = 0; h < kTileM / kHalfSites; ++h)
                                tma_prefetch_2d(&tmS, 4 * (ta * kTileM + h * kHalfSites), ja * kDirsPerStage);
                        }
                    }
                }
            }
            // drain: wait (bounded) for the loads this thread issued into each stage
            for (int gr = 0; gr < 2; ++gr)
                for (uint32_t k = 0; k < (uint32_t)(stages / 2) && k < gq[gr]; ++k) {
                    const uint32_t local = gq[gr] - 1 - k;
                    if (stall && gr == 0 && local == 0) continue;   // never issued
                    const int s = ring_slot(gr, local, stages / 2);
                    unsigned long long t0 = global_ns();
                    while (!mbar_try(smem_u32(&st_full[s]), (local / (uint32_t)(stages / 2)) & 1) &&
                           global_ns() - t0 < kTimeoutNs) {
                    }
                }
        }
    } else if (warp == kMmaWarp) {
        // ---------------------------------------------------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(kTileM, N4);
            int prev_cls = -1;
            uint32_t zl = 0;
            bool ok = true;
            bool issued = false;
            for (int i = 0; i < T && ok; ++i) {
                const int cls = p.tiles[t_begin + i] >> 24;
                const int b = i & 1;
                if (cls != prev_cls) {
                    ok = mbar_wait(smem_u32(z_full), zl & 1, abort_flag, p.err, kErrTimeoutMma);
                    ++zl;
                    prev_cls = cls;
                    if (!ok) break;
                }
                ok = mbar_wait(smem_u32(&t_ready[b]), (i >> 1) & 1, abort_flag, p.err, kErrTimeoutMma);
                if (!ok) break;
                tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(b * N4);
                for (int c = 0; c < C; ++c) {
                    const int ksteps = min(4, (N4 - 64 * c) / 16);
                    for (int kk = 0; kk < ksteps; ++kk) {
                        const uint32_t ao = c * a_chunk + kk * 32, zo = c * z_chunk + kk * 32;
                        const uint32_t acc_in = (sepE && c == 0 && kk == 0) ? 0u : 1u;   // E: the tile starts D from zero
                        mma_bf16(d_tmem, sw128_desc(smem_u32(sA + ao)), sw128_desc(smem_u32(sZ + zo)), idesc, acc_in);
                        if (ZLO) mma_bf16(d_tmem, sw128_desc(smem_u32(sA + ao)), sw128_desc(smem_u32(sZlo + zo)), idesc, 1u);
                        if (ALO) mma_bf16(d_tmem, sw128_desc(smem_u32(sAlo + ao)), sw128_desc(smem_u32(sZ + zo)), idesc, 1u);
                    }
                    mma_commit(smem_u32(&a_empty[c]));
                }
                mma_commit(smem_u32(&acc_full[b]));
                if (i + 1 < T && (p.tiles[t_begin + i + 1] >> 24) != cls) mma_commit(smem_u32(z_free));
                issued = true;
            }
            if (issued) {
                // drain: all MMAs this thread issued have completed before TMEM is freed
                mma_commit(smem_u32(drain));
                unsigned long long t0 = global_ns();
                while (!mbar_try(smem_u32(drain), 0) && global_ns() - t0 < kTimeoutNs) {
                }
            }
        }
        __syncwarp();
    } else if (warp >= kConvWarp0) {
        // ----------------------------------------------------------- converter
        const int q = warp & 3;
        const int grp = (warp - kConvWarp0) >> 2;  // staging-slot group
        const int r = q * 32 + lane;               // site row = TMEM lane
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        uint32_t gq = 0, fq = 0;   // staging slots consumed; ghost fills (gather form)
        bool ok = true;
        // tile entries two ahead, coefficients one ahead (see load_coef)
        int e_next = T > 0 ? p.tiles[t_begin] : 0, e_after = T > 1 ? p.tiles[t_begin + 1] : 0;
        float4 cf_next = T > 0 ? load_coef(p.coef, (e_next & 0xFFFFFF) * kTileM + r, nsites) : float4{};
        for (int i = 0; i < T && ok; ++i) {
            const int entry = e_next;
            const float4 cf = cf_next;
            const int b = i & 1;
            if (i + 1 < T) {
                e_next = e_after;
                cf_next = load_coef(p.coef, (e_next & 0xFFFFFF) * kTileM + r, nsites);
                if (i + 2 < T) e_after = p.tiles[t_begin + i + 2];
            }
            ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&acc_empty[b]), ((i >> 1) & 1) ^ 1, abort_flag, p.err,
                                                   kErrTimeoutConverter));
            if (!ok) break;
            tc_fence_after();
            const uint32_t acc = tmem + lane_base + (uint32_t)((sepE ? 2 * N4 : 0) + b * N4);   // E, else D
            if (GATHER) {
                const int site = (entry & 0xFFFFFF) * kTileM + r, z = site / p.nx, x = site - z * p.nx;
                const GatherGeom g{p.nx, p.nz, p.bcbits, reinterpret_cast<const float4 *>(p.P),
                                   reinterpret_cast<const float4 *>(p.inflow)};
                ok = convert_tile_gather<ALO>(cf, p.fwd + (size_t)(entry >> 24) * n, r, lane, grp, n, stages, gq, i, acc,
                                              sA, sAlo, sStage, st_full, st_empty, a_empty, fill_bar, fq, a_chunk, g, gt,
                                              !gather_interior_tile(gt, p.bcbits, p.nx, p.nz, x - r, z), x, z,
                                              abort_flag, p.err);
            } else {
                ok = convert_tile<ALO>(cf, p.fwd + (size_t)(entry >> 24) * n, r, lane, grp, n, groups, stages, gq, i,
                                       acc, sA, sAlo, sStage, st_full, st_empty, a_empty, a_chunk, abort_flag, p.err);
            }
            if (!ok) break;
            tmem_wait_st();
            fence_proxy_async();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&t_ready[b]));
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int q = warp & 3;
        const int dhalf = warp >> 2;                  // 0: first half of the directions, 1: second
        const int r = q * 32 + lane;
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        const int dn = n / 2, dbeg = dhalf * dn;
        float4 *out = reinterpret_cast<float4 *>(p.S_new);
        bool ok = true;
        for (int i = 0; i < T && ok; ++i) {
            const int tile = p.tiles[t_begin + i] & 0xFFFFFF;
            const int b = i & 1;
            const int site = tile * kTileM + r;
            const int z = site / p.nx, x = site - z * p.nx;
            const bool interior = site < nsites && x > 0 && x < p.nx - 1 && z > 0 && z < p.nz - 1;
            ok = __all_sync(0xffffffffu,
                            mbar_wait(smem_u32(&acc_full[b]), (i >> 1) & 1, abort_flag, p.err, kErrTimeoutEpilogue));
            if (!ok) break;
            tc_fence_after();
            const uint32_t acc = tmem + lane_base + (uint32_t)(b * N4);
            for (int d0 = dbeg; d0 < dbeg + dn; d0 += 4) {
                float v[16];
                tmem_ld16(acc + 4 * d0, v);
                if (sepE) {
                    float e[16];
                    tmem_ld16(acc + (uint32_t)(2 * N4) + 4 * d0, e);
#pragma unroll
                    for (int k = 0; k < 16; ++k) v[k] += e[k];
                }
                if (interior) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int d = d0 + k;
                        const long long t = (long long)d * nsites + site + s_cx[d] + (long long)s_cz[d] * p.nx;
                        const float4 val = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
#if RTLB_TC_STREAM_STORES
                        __stcs(&out[t], val);
#else
                        out[t] = val;
#endif
                    }
                } else if (site < nsites) {
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        push_store_xz(p.dir, p.inflow, p.bcbits, p.S_new, p.nx, p.nz, n, site, x, z, d0 + k,
                                   make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]));
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&acc_empty[b]));
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kMmaWarp) tmem_dealloc(tmem, tcols);
}

// Split-table form (MODE 2) on a CTA pair (cluster of 2, cta_group::2) for
// tables too large for one CTA's shared memory with their low parts (n = 64:
// 2 x 128 KB).  CTA r of the pair processes its own 128-site tile (A rows,
// TMEM init, epilogue exactly as above) and holds rows [r N/2, (r+1) N/2) of
// the table's hi and lo parts.  The even CTA issues M = 256 MMAs that read A
// from both CTAs and B halves from each; their commits are multicast to both
// CTAs' barriers.  The odd CTA's converter warps report a ready tile on a
// local barrier; one thread of its otherwise idle MMA warp forwards it to the
// even CTA with a single remote (cluster-scope release) arrive, which keeps
// that microsecond-long release off the converters' path.  Its producer
// forwards the completion of its half of the table the same way.
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1)
    k_step_tc_pair(const __grid_constant__ CUtensorMap tmS, const __grid_constant__ CUtensorMap tmZhi,
                   const __grid_constant__ CUtensorMap tmZlo, TcParams p, int N4, int stages)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const uint32_t rank = cluster_rank();
    const bool leader = rank == 0;
    const int C = (N4 + 63) / 64;
    const int NH = N4 / 2;                          // table rows held by this CTA
    const int n = p.n;
    const int nsites = p.nx * p.nz;
    const int groups = n / kDirsPerStage;
    const uint32_t z_chunk = (uint32_t)NH * 128u;
    const uint32_t a_chunk = (uint32_t)kTileM * 128u;

    uint8_t *sZ = smem;
    uint8_t *sZlo = sZ + C * z_chunk;
    uint8_t *sA = sZlo + C * z_chunk;
    uint8_t *sStage = sA + C * a_chunk;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sStage + (size_t)stages * kStageBytes);
    uint64_t *st_full = bars;
    uint64_t *st_empty = st_full + stages;
    uint64_t *a_empty = st_empty + stages;     // [C]   multicast commit from the even CTA
    uint64_t *t_ready = a_empty + C;           // [2]   used in the even CTA: 8 converter warps
    uint64_t *acc_full = t_ready + 2;          // [2]   multicast commit
    uint64_t *acc_empty = acc_full + 2;        // [2]   local epilogue warps
    uint64_t *z_full = acc_empty + 2;          // [1]   even CTA: own TMA + odd CTA's forward
    uint64_t *drain = z_full + 1;              // [1]   multicast commit
    uint64_t *z_free = drain + 1;              // [1]   multicast commit: the resident table is no longer read
    uint64_t *t_local = z_free + 1;            // [2]   odd CTA: its 4 converter warps, forwarded to the even CTA
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(t_local + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    int8_t *s_cx = reinterpret_cast<int8_t *>(tmem_slot + 2);
    int8_t *s_cz = s_cx + kMaxDirs;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t tcols = 512;                 // two N4 = 256 accumulators

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(smem_u32(&st_full[s]), 1);
            mbar_init(smem_u32(&st_empty[s]), 4);
        }
        for (int c = 0; c < C; ++c) mbar_init(smem_u32(&a_empty[c]), 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&t_ready[b]), kConvWarps + 1);   // local converter warps + the odd CTA's forward
            mbar_init(smem_u32(&t_local[b]), kConvWarps);
            mbar_init(smem_u32(&acc_full[b]), 1);
            mbar_init(smem_u32(&acc_empty[b]), kEpiWarps);
        }
        mbar_init(smem_u32(z_full), leader ? 2 : 1);
        mbar_init(smem_u32(drain), 1);
        mbar_init(smem_u32(z_free), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int d = threadIdx.x; d < n; d += blockDim.x) {
        s_cx[d] = (int8_t)p.dir[d];
        s_cz[d] = (int8_t)p.dir[n + d];
    }
    if (warp == kMmaWarp) tmem_alloc_pair(smem_u32(tmem_slot), tcols);
    tc_fence_before();
    __syncthreads();
    cluster_sync();                             // barriers of both CTAs initialized
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int ncl = (int)cluster_nclusters_x(), cid = (int)cluster_id_x();
    const int t_begin = (int)((long long)p.n_tiles * cid / ncl);
    const int t_end = (int)((long long)p.n_tiles * (cid + 1) / ncl);
    const int T = t_end - t_begin;
    // pair entries: tile_a | class << 24 at 2k, tile_b at 2k + 1
    auto my_tile = [&](int i) { return p.tiles[2 * (t_begin + i) + (int)rank] & 0xFFFFFF; };
    auto pair_cls = [&](int i) { return p.tiles[2 * (t_begin + i)] >> 24; };

    if (warp == kProdWarp) {
        if (lane == 0) {
            const bool stall = p.stall != 0 && blockIdx.x == 0;   // the even CTA of cluster 0
            int prev_cls = -1;
            uint32_t gq[2] = {0, 0}, zl = 0, zr = 0;
            bool ok = true;
            for (int i = 0; i < T && ok; ++i) {
                const int tile = my_tile(i), cls = pair_cls(i);
                if (cls != prev_cls) {
                    if (i > 0) ok = mbar_wait(smem_u32(z_free), (zr++) & 1, abort_flag, p.err, kErrTimeoutProducer);
                    if (!ok) break;
                    const uint32_t zb = smem_u32(z_full);
                    mbar_expect_tx(zb, 2u * C * z_chunk);
                    for (int c = 0; c < C; ++c) {
                        tma_load_3d(smem_u32(sZ + c * z_chunk), &tmZhi, zb, 64 * c, NH * (int)rank, cls);
                        tma_load_3d(smem_u32(sZlo + c * z_chunk), &tmZlo, zb, 64 * c, NH * (int)rank, cls);
                    }
                    if (!leader) {
                        // forward the completion of this half to the even CTA
                        ok = mbar_wait(zb, zl & 1, abort_flag, p.err, kErrTimeoutProducer);
                        if (!ok) break;
                        mbar_arrive_cluster(mapa(zb, 0));
                    }
                    ++zl;
                    prev_cls = cls;
                }
                for (int j = 0; j < groups && ok; ++j) {
                    const int gr = j & 1;
                    const uint32_t local = gq[gr]++;
                    const int s = ring_slot(gr, local, stages / 2);
                    ok = mbar_wait(smem_u32(&st_empty[s]), ((local / (uint32_t)(stages / 2)) & 1) ^ 1, abort_flag, p.err,
                                   kErrTimeoutProducer);
                    if (!ok) break;
                    if (stall && i == 0 && j == 0) continue;   // test hook: this load is never issued
                    const uint32_t fb = smem_u32(&st_full[s]);
                    mbar_expect_tx(fb, kStageBytes);
                    for (int h = 0; h < kTileM / kHalfSites; ++h)
                        tma_load_2d(smem_u32(sStage + (size_t)s * kStageBytes + h * (kStageBytes / 2)), &tmS, fb,
                                    4 * (tile * kTileM + h * kHalfSites), j * kDirsPerStage);
                    if (RTLB_TC_PAIR_PREFETCH_SLOTS > 0) {
                        // two staging slots per CTA hold ~32 KB in flight: the
                        // chunk a few slots ahead goes to L2 meanwhile
                        const int ahead = i * groups + j + RTLB_TC_PAIR_PREFETCH_SLOTS;
                        const int ia = ahead / groups, ja = ahead - ia * groups;
                        if (ia < T) {
                            const int ta = my_tile(ia);
                            for (int h = 0; h < kTileM / kHalfSites; ++h)
                                tma_prefetch_2d(&tmS, 4 * (ta * kTileM + h * kHalfSites), ja * kDirsPerStage);
                        }
                    }
                }
            }
            for (int gr = 0; gr < 2; ++gr)
                for (uint32_t k = 0; k < (uint32_t)(stages / 2) && k < gq[gr]; ++k) {
                    const uint32_t local = gq[gr] - 1 - k;
                    if (stall && gr == 0 && local == 0) continue;   // never issued
                    const int s = ring_slot(gr, local, stages / 2);
                    unsigned long long t0 = global_ns();
                    while (!mbar_try(smem_u32(&st_full[s]), (local / (uint32_t)(stages / 2)) & 1) &&
                           global_ns() - t0 < kTimeoutNs) {
                    }
                }
        }
    } else if (warp == kMmaWarp) {
        if (lane == 0 && leader) {
            const uint32_t idesc = idesc_bf16(2 * kTileM, N4);
            int prev_cls = -1;
            uint32_t zl = 0;
            bool ok = true;
            for (int i = 0; i < T && ok; ++i) {
                const int cls = pair_cls(i);
                const int b = i & 1;
                if (cls != prev_cls) {
                    ok = mbar_wait_cluster(smem_u32(z_full), zl & 1, abort_flag, p.err, kErrTimeoutMma);
                    ++zl;
                    prev_cls = cls;
                    if (!ok) break;
                }
                ok = mbar_wait_cluster(smem_u32(&t_ready[b]), (i >> 1) & 1, abort_flag, p.err, kErrTimeoutMma);
                if (!ok) break;
                tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(b * N4);
                for (int c = 0; c < C; ++c) {
                    for (int kk = 0; kk < 4; ++kk) {
                        const uint32_t ao = c * a_chunk + kk * 32, zo = c * z_chunk + kk * 32;
                        const uint64_t ad = sw128_desc(smem_u32(sA + ao));
                        mma_bf16_pair(d_tmem, ad, sw128_desc(smem_u32(sZ + zo)), idesc, 1u);
                        mma_bf16_pair(d_tmem, ad, sw128_desc(smem_u32(sZlo + zo)), idesc, 1u);
                    }
                    mma_commit_pair(smem_u32(&a_empty[c]), 0x3);
                }
                mma_commit_pair(smem_u32(&acc_full[b]), 0x3);
                if (i + 1 < T && pair_cls(i + 1) != cls) mma_commit_pair(smem_u32(z_free), 0x3);
            }
            // commit even when nothing was issued (it then arrives at once):
            // both CTAs wait on `drain` below whenever T > 0, also after an abort
            if (T > 0) mma_commit_pair(smem_u32(drain), 0x3);
        } else if (lane == 0) {
            // odd CTA: forward each tile's readiness (A rows in shared memory,
            // accumulator initialized in TMEM) to the even CTA.  One
            // cluster-scope release per tile, off the converter warps' path
            // (a release at cluster scope costs about a microsecond).
            for (int i = 0; i < T; ++i) {
                const int b = i & 1;
                if (!mbar_wait(smem_u32(&t_local[b]), (i >> 1) & 1, abort_flag, p.err, kErrTimeoutMma)) break;
                tc_fence_after();
                fence_proxy_async();
                tc_fence_before();
                mbar_arrive_cluster(mapa(smem_u32(&t_ready[b]), 0));
            }
        }
        __syncwarp();
    } else if (warp >= kConvWarp0) {
        const int q = warp & 3;
        const int grp = (warp - kConvWarp0) >> 2;
        const int r = q * 32 + lane;
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        uint32_t gq = 0;
        bool ok = true;
        // coefficients and classes fetched a tile ahead (see load_coef)
        float4 cf_next = T > 0 ? load_coef(p.coef, my_tile(0) * kTileM + r, nsites) : float4{};
        int cls_next = T > 0 ? pair_cls(0) : 0;
        for (int i = 0; i < T && ok; ++i) {
            const float4 cf = cf_next;
            const int cls = cls_next;
            const int b = i & 1;
            if (i + 1 < T) {
                cf_next = load_coef(p.coef, my_tile(i + 1) * kTileM + r, nsites);
                cls_next = pair_cls(i + 1);
            }
            ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&acc_empty[b]), ((i >> 1) & 1) ^ 1, abort_flag, p.err,
                                                   kErrTimeoutConverter));
            if (!ok) break;
            tc_fence_after();
            const uint32_t acc = tmem + lane_base + (uint32_t)(b * N4);
            ok = convert_tile<false>(cf, p.fwd + (size_t)cls * n, r, lane, grp, n, groups, stages, gq, i, acc, sA, sA,
                                     sStage, st_full, st_empty, a_empty, a_chunk, abort_flag, p.err);
            if (!ok) break;
            tmem_wait_st();
            fence_proxy_async();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(leader ? &t_ready[b] : &t_local[b]));
        }
    } else {
        const int q = warp & 3;
        const int dhalf = warp >> 2;
        const int r = q * 32 + lane;
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        const int dn = n / 2, dbeg = dhalf * dn;
        float4 *out = reinterpret_cast<float4 *>(p.S_new);
        bool ok = true;
        for (int i = 0; i < T && ok; ++i) {
            const int tile = my_tile(i);
            const int b = i & 1;
            const int site = tile * kTileM + r;
            const int z = site / p.nx, x = site - z * p.nx;
            const bool interior = site < nsites && x > 0 && x < p.nx - 1 && z > 0 && z < p.nz - 1;
            ok = __all_sync(0xffffffffu,
                            mbar_wait(smem_u32(&acc_full[b]), (i >> 1) & 1, abort_flag, p.err, kErrTimeoutEpilogue));
            if (!ok) break;
            tc_fence_after();
            const uint32_t acc = tmem + lane_base + (uint32_t)(b * N4);
            for (int d0 = dbeg; d0 < dbeg + dn; d0 += 4) {
                float v[16];
                tmem_ld16(acc + 4 * d0, v);
                if (interior) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int d = d0 + k;
                        const long long t = (long long)d * nsites + site + s_cx[d] + (long long)s_cz[d] * p.nx;
                        const float4 val = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
#if RTLB_TC_STREAM_STORES
                        __stcs(&out[t], val);
#else
                        out[t] = val;
#endif
                    }
                } else if (site < nsites) {
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        push_store_xz(p.dir, p.inflow, p.bcbits, p.S_new, p.nx, p.nz, n, site, x, z, d0 + k,
                                   make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]));
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&acc_empty[b]));
        }
    }

    // every MMA issued into this CTA's TMEM has completed (bounded wait, taken
    // after an abort too: the even CTA commits `drain` once whenever T > 0),
    // then both CTAs leave together and free the pair's TMEM
    if (warp == kMmaWarp && lane == 0 && T > 0) {
        unsigned long long t0 = global_ns();
        while (!mbar_try_cluster(smem_u32(drain), 0) && global_ns() - t0 < kTimeoutNs) {
        }
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync();
    tc_fence_after();
    if (warp == kMmaWarp) tmem_dealloc_pair(tmem, tcols);
}

// ------------------------------------------------------------------ host side

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void *ptr = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    }
    return fn;
}

bool encode_state_map(CUtensorMap *m, const float *S, size_t nsites, int n)
{
    auto fn = encode_fn();
    if (!fn) return false;
    // 2D view: x = float index within one direction plane (4 per site), y = direction
    cuuint64_t dims[2] = {(cuuint64_t)nsites * 4, (cuuint64_t)n};
    cuuint64_t strides[1] = {(cuuint64_t)nsites * 16};
    cuuint32_t box[2] = {(cuuint32_t)(kHalfSites * 4), (cuuint32_t)kDirsPerStage};
    cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(S), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Windows of the gather form: 4D view (the floats of kGatherSites sites, site
// group, row z, direction d) of the direction-major state (nx % 128 == 0),
// boxes of kGatherCols sites x 2 rows, zero outside the lattice.
bool encode_gather_map(CUtensorMap *m, const float *S, int nx, int nz, int n)
{
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[4] = {(cuuint64_t)(4 * kGatherSites), (cuuint64_t)(nx / kGatherSites), (cuuint64_t)nz,
                          (cuuint64_t)n};
    cuuint64_t strides[3] = {(cuuint64_t)(16 * kGatherSites), (cuuint64_t)nx * 16, (cuuint64_t)nx * nz * 16};
    cuuint32_t box[4] = {(cuuint32_t)(4 * kGatherSites), (cuuint32_t)(kGatherCols / kGatherSites), 2, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float *>(S), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool encode_z_map(CUtensorMap *m, const __nv_bfloat16 *Z, int N4, int KP, int n_phase, int box_rows)
{
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)KP, (cuuint64_t)N4, (cuuint64_t)n_phase};
    cuuint64_t strides[2] = {(cuuint64_t)KP * 2, (cuuint64_t)N4 * KP * 2};
    cuuint32_t box[3] = {64, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16 *>(Z), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// tf32 table [n_phase][N4][N4] (float32 containers), boxes of 32 values (one
// SW128 row of 128 bytes) x N4 rows
bool encode_zt_map(CUtensorMap *m, const float *Zt, int N4, int n_phase)
{
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)N4, (cuuint64_t)N4, (cuuint64_t)n_phase};
    cuuint64_t strides[2] = {(cuuint64_t)N4 * 4, (cuuint64_t)N4 * N4 * 4};
    cuuint32_t box[3] = {32, (cuuint32_t)N4, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(Zt), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Nearest tf32 value (10 stored mantissa bits, ties to even) of a float32.
float tf32_round(float x)
{
    uint32_t b;
    std::memcpy(&b, &x, 4);
    if ((b & 0x7F800000u) != 0x7F800000u) b = (b + 0x0FFFu + ((b >> 13) & 1u)) & 0xFFFFE000u;
    float r;
    std::memcpy(&r, &b, 4);
    return r;
}

// e4m3 table [n_phase][N4][KP8] bytes, boxes of 128 bytes (one SW128 row) x N4 rows
bool encode_z8_map(CUtensorMap *m, const uint8_t *Z8, int N4, int KP8, int n_phase)
{
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)KP8, (cuuint64_t)N4, (cuuint64_t)n_phase};
    cuuint64_t strides[2] = {(cuuint64_t)KP8, (cuuint64_t)N4 * KP8};
    cuuint32_t box[3] = {128, (cuuint32_t)N4, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<uint8_t *>(Z8), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// UE8M0 exponent of a table block whose largest |value| is amax (float64):
// the smallest e with amax / 2^e <= 448, within [-127, 127]; -127 for zero.
int table_block_exponent(double amax)
{
    if (!(amax > 0.0)) return -127;
    int E2;
    const double f = std::frexp(amax, &E2);   // amax = f 2^E2, f in [0.5, 1)
    const int e = (E2 - 1) - 8 + (2.0 * f > 1.75 ? 1 : 0);
    return std::max(-127, std::min(127, e));
}

TcState *state_of(rtlb_ctx *c) { return static_cast<TcState *>(c->tc); }

void free_tables(TcState *t)
{
    cudaFree(t->d_Zhi);
    cudaFree(t->d_Zlo);
    cudaFree(t->d_Z8);
    cudaFree(t->d_sfb);
    t->d_Z8 = t->d_sfb = nullptr;
    cudaFree(t->d_Zt_hi);
    cudaFree(t->d_Zt_lo);
    t->d_Zt_hi = t->d_Zt_lo = nullptr;
    cudaFree(t->d_fwd);
    cudaFree(t->d_pure);
    cudaFree(t->d_mixed);
    t->d_fwd = nullptr;
    t->d_Zhi = t->d_Zlo = nullptr;
    t->d_pure = t->d_mixed = nullptr;
    t->n_pure = t->n_mixed = 0;
}

size_t smem_bytes(int N4, int mode, int stages, bool gather = false)
{
    const int C = (N4 + 63) / 64;
    size_t b = (size_t)C * N4 * 128 * (mode >= 2 ? 2 : 1) + (size_t)C * kTileM * 128 * (mode == 3 ? 2 : 1) +
               (size_t)stages * (gather ? kGatherStageBytes : (uint32_t)kStageBytes) + (size_t)(2 * stages + C + 11) * 8 + 16 + 2 * kMaxDirs;
    return b + 1024;  // alignment slack
}

size_t smem_bytes_pair(int N4, int stages)
{
    const int C = (N4 + 63) / 64;
    size_t b = (size_t)C * (N4 / 2) * 128 * 2 + (size_t)C * kTileM * 128 + (size_t)stages * kStageBytes +
               (size_t)(2 * stages + C + 11) * 8 + 16 + 2 * kMaxDirs;
    return b + 1024;
}

int mode_of(int precision)
{
    if (precision == RTLB_PREC_FP8) return 4;
    if (precision == RTLB_PREC_TF32X3) return 5;
    if (precision == RTLB_PREC_FP8X) return 6;
    return precision == RTLB_PREC_BF16X3 ? 3 : (precision == RTLB_PREC_BF16X2 ? 2 : 1);
}

#ifndef RTLB_TC_MAX_STAGES
#define RTLB_TC_MAX_STAGES 8
#endif

// Largest even stage count that fits (0 = does not fit); even because each
// of the two converter groups owns half of the staging slots.
int fit_stages(int N4, int mode, bool pair, bool gather = false)
{
    for (int st = RTLB_TC_MAX_STAGES & ~1; st >= 2; st -= 2)
        if ((pair ? (gather ? ~(size_t)0 : smem_bytes_pair(N4, st))   // no gather form on CTA pairs
                  : (mode == 4 ? tc_fp8_smem_bytes(N4, st)
                               : (mode == 5 ? tc_tf32_smem_bytes(N4, st)
                                            : (mode == 6 ? tc_fp8x_smem_bytes(N4, st)
                                                         : smem_bytes(N4, mode, st, gather))))) <=
            (size_t)kSmemLimit)
            return st;
    return 0;
}

}  // namespace

bool tc_supported(int n) { return n == 8 || n == 16 || n == 32 || n == 64; }

bool tc_shape_ok(int n, int precision)
{
    if (!tc_supported(n)) return false;
    const int mode = mode_of(precision);
    if (mode == 5 && n > 32) return false;      // the split tf32 table of n = 64 (512 KB) fits no CTA
    return fit_stages(4 * n, mode, false) > 0 || (mode == 2 && fit_stages(4 * n, mode, true) > 0);
}

rtlb_status tc_prepare(rtlb_ctx *c, const double *tables, int n_phase, const uint8_t *dev_cls, cudaStream_t s)
{
    if (c->opt.precision == RTLB_PREC_FP32) return RTLB_OK;
    const int mode = mode_of(c->opt.precision);
    const bool split = mode == 2 || mode == 3;
    const bool tf32 = mode == 5;
    if (!tc_supported(c->n) || (tf32 && c->n > 32)) {
        c->err = tf32 ? "the 3xTF32 form needs n in {8, 16, 32}" : "tensor-core forms need n in {8, 16, 32, 64}";
        return RTLB_E_UNSUPPORTED;
    }
    const int N4 = 4 * c->n, KP = ((N4 + 63) / 64) * 64, C = KP / 64;
    bool pair = false, gather = false;
    int stages = fit_stages(N4, mode, false);
    if (stages == 0 && mode == 2) {
        pair = true;
        stages = fit_stages(N4, mode, true);
    }
    // bilinear streaming is gathered while loading (the bf16 forms) where
    // tiles are row segments and the windows' staging fits
    GatherTaps gtaps{};
    bool taps_ok = c->opt.streaming == RTLB_STREAM_BILINEAR && c->n <= kTcMaxDirs;
    for (int d = 0; taps_ok && d < c->n; ++d) {
        const int *o = &c->tap_o[8 * (size_t)d];
        for (int k = 0; k < 4; ++k)
            if (o[k] != o[0] + (k & 1) || o[4 + k] != o[4] + (k >> 1) || std::abs(o[0]) > 100 || std::abs(o[4]) > 100)
                taps_ok = false;
        const float *w = &c->tap_w[4 * (size_t)d];
        gtaps.w[d] = make_float4(w[0], w[1], w[2], w[3]);
        gtaps.n0x[d] = (int8_t)o[0];
        gtaps.n0z[d] = (int8_t)o[4];
        gtaps.reach_x = std::max(gtaps.reach_x, std::max(std::abs(o[0]), std::abs(o[0] + 1)));
        gtaps.reach_z = std::max(gtaps.reach_z, std::max(std::abs(o[4]), std::abs(o[4] + 1)));
    }
    if (stages > 0 && mode <= 3 && taps_ok && c->nx % kTileM == 0 && c->n % 16 == 0) {
        // at least two staging slots per converter group (four directions
        // each) in flight: with one, each slot's load latency shows in full
        const int gst = fit_stages(N4, mode, pair, true);
        if (gst >= 4) {
            gather = true;
            stages = gst;
        }
    }
    if (stages == 0) {
        c->err = "this precision form does not fit in shared memory for this n";
        return RTLB_E_UNSUPPORTED;
    }
    if (!encode_fn()) {
        c->err = "cuTensorMapEncodeTiled is not available from the driver";
        return RTLB_E_CUDA;
    }
    TcState *t = state_of(c);
    if (!t) {
        t = new TcState();
        c->tc = t;
        cudaDeviceGetAttribute(&t->sm_count, cudaDevAttrMultiProcessorCount, c->dev);
        if (cudaMalloc(&t->d_err, sizeof(int)) != cudaSuccess || cudaMallocHost(&t->h_err, sizeof(int)) != cudaSuccess) {
            c->err = "tensor-core error flag allocation failed";
            return RTLB_E_OOM;
        }
        cudaMemset(t->d_err, 0, sizeof(int));
    }
    // bf16 operand tables, K padded to a multiple of 64.  When a table's
    // forward block Z(i, i) is c_i times the 4x4 identity (true for every
    // table built from Eq. 13-17: no frame rotation and a diagonal phase
    // matrix at zero scattering angle), that block is taken out of the MMA
    // operand and applied exactly in float32 by the converter; it is the
    // largest entry of forward-peaked tables and would otherwise carry the
    // largest bf16 rounding error.  hi = round-to-nearest bf16, lo = the
    // remainder (split form).
    const size_t tsz = (size_t)N4 * N4, psz = (size_t)N4 * KP;
    const int n = c->n;
    std::vector<float> fwd((size_t)n_phase * n, 0.0f);
    std::vector<double> work(tsz);
    const bool fp8 = mode == 4 || mode == 6;
    const int terms = mode == 6 ? 3 : 1;          // e4m3 terms of the table
    const int KP8 = ((N4 + 127) / 128) * 128, ksteps = N4 / 32;
    std::vector<__nv_bfloat16> hi((fp8 || tf32) ? 0 : (size_t)n_phase * psz, __float2bfloat16(0.0f)),
        lo(hi.size(), __float2bfloat16(0.0f));
    std::vector<float> thi(tf32 ? (size_t)n_phase * tsz : 0, 0.0f), tlo(thi.size(), 0.0f);
    std::vector<uint8_t> z8(fp8 ? (size_t)terms * n_phase * N4 * KP8 : 0, 0),
        sfb(fp8 ? (size_t)terms * n_phase * N4 * ksteps : 0, 0);
    if (fp8 && (mode == 6 ? tc_fp8x_tmem_columns(N4, n_phase) : tc_fp8_tmem_columns(N4, n_phase)) > 512) {
        c->err = "the FP8 forms keep every class's table scales in tensor memory: too many phase classes for this n";
        return RTLB_E_UNSUPPORTED;
    }
    for (int ph = 0; ph < n_phase; ++ph) {
        const double *Zp = tables + (size_t)ph * tsz;
        std::copy(Zp, Zp + tsz, work.begin());
        bool diag = true;
        for (int i = 0; i < n && diag; ++i) {
            const double ci = Zp[(size_t)(4 * i) * N4 + 4 * i];
            for (int a = 0; a < 4 && diag; ++a)
                for (int b = 0; b < 4; ++b) {
                    const double want = (a == b) ? ci : 0.0;
                    if (std::fabs(Zp[(size_t)(4 * i + a) * N4 + 4 * i + b] - want) > 1e-14 * std::fabs(ci)) {
                        diag = false;
                        break;
                    }
                }
        }
        if (diag)
            for (int i = 0; i < n; ++i) {
                const double ci = Zp[(size_t)(4 * i) * N4 + 4 * i];
                fwd[(size_t)ph * n + i] = (float)ci;
                // the float32 value is what the kernel applies: keep the
                // remainder of its rounding in the MMA operand
                for (int a = 0; a < 4; ++a)
                    work[(size_t)(4 * i + a) * N4 + 4 * i + a] = ci - (double)(float)ci;
            }
        if (fp8) {
            // e4m3 with one UE8M0 scale per table row and 32-element block; the
            // split form quantizes what the terms before left, each term with
            // the scale of that remainder
            for (int t = 0; t < terms; ++t)
                for (int row = 0; row < N4; ++row)
                    for (int ks = 0; ks < ksteps; ++ks) {
                        double *blk = &work[(size_t)row * N4 + 32 * ks];
                        double amax = 0.0;
                        for (int k = 0; k < 32; ++k) amax = std::max(amax, std::fabs(blk[k]));
                        const int e = table_block_exponent(amax);
                        const size_t tp = (size_t)t * n_phase + ph;
                        sfb[(tp * N4 + row) * ksteps + ks] = (uint8_t)(e + 127);
                        for (int k = 0; k < 32; ++k) {
                            const __nv_fp8_storage_t q = __nv_cvt_double_to_fp8(std::ldexp(blk[k], -e), __NV_SATFINITE, __NV_E4M3);
                            z8[tp * N4 * KP8 + (size_t)row * KP8 + 32 * ks + k] = (uint8_t)q;
                            blk[k] -= std::ldexp((double)__half2float(__half(__nv_cvt_fp8_to_halfraw(q, __NV_E4M3))), e);
                        }
                    }
            continue;
        }
        if (tf32) {
            // tf32 hi = nearest tf32 of the value, lo = nearest tf32 of the
            // remainder (about 22 significand bits together)
            for (size_t k = 0; k < tsz; ++k) {
                const double v = work[k];
                const float h = tf32_round((float)v);
                thi[(size_t)ph * tsz + k] = h;
                tlo[(size_t)ph * tsz + k] = tf32_round((float)(v - (double)h));
            }
            continue;
        }
        for (int row = 0; row < N4; ++row)
            for (int col = 0; col < N4; ++col) {
                const double v = work[(size_t)row * N4 + col];
                const __nv_bfloat16 h = __float2bfloat16((float)v);
                hi[(size_t)ph * psz + (size_t)row * KP + col] = h;
                lo[(size_t)ph * psz + (size_t)row * KP + col] = __float2bfloat16((float)(v - (double)__bfloat162float(h)));
            }
    }
    // per-tile phase class (from the site classes), pure tiles sorted by class
    const size_t ns = c->nsites();
    const int ntiles = (int)((ns + kTileM - 1) / kTileM);
    std::vector<uint8_t> cls(ns, 0);
    if (dev_cls && cudaMemcpy(cls.data(), dev_cls, ns, cudaMemcpyDeviceToHost) != cudaSuccess) {
        c->err = "phase index download failed";
        return RTLB_E_CUDA;
    }
    std::vector<int> pure, mixed;
    for (int tile = 0; tile < ntiles; ++tile) {
        const size_t a = (size_t)tile * kTileM, e = std::min(ns, a + kTileM);
        bool same = true;
        for (size_t k = a + 1; k < e; ++k)
            if (cls[k] != cls[a]) {
                same = false;
                break;
            }
        if (same) pure.push_back(tile | ((int)cls[a] << 24));
        else mixed.push_back(tile);
    }
    if (gather) {
        // by class, then down strips of 512 sites (four tiles): a CTA's tiles
        // go row by row down its strip, so one of the two window rows a tile
        // reads was read four tiles before and is still in L2.  Measured at
        // 2048^2 (ms per step, n = 32 / 16): strips of 1 tile 1.43 / 0.70, 2
        // tiles 1.37 / 0.66, 4 tiles 1.34 / 0.65, 8 tiles 1.34 / 0.66, whole
        // rows 1.31 / 0.68.
        const int nx = c->nx;
        auto key = [nx](int e) {
            const long long site0 = (long long)(e & 0xFFFFFF) * kTileM;
            const long long z = site0 / nx, x0 = site0 - z * nx;
            return std::make_tuple(e >> 24, x0 / (4 * kTileM), z, x0);
        };
        std::stable_sort(pure.begin(), pure.end(), [&](int x, int y) { return key(x) < key(y); });
    } else {
        std::stable_sort(pure.begin(), pure.end(), [](int x, int y) { return (x >> 24) < (y >> 24); });
    }
    if (pair) {
        // consecutive single-class tiles of the same class form a pair; a
        // tile left alone in its class runs on the CUDA-core kernel
        std::vector<int> pairs;
        size_t k = 0;
        while (k < pure.size()) {
            if (k + 1 < pure.size() && (pure[k] >> 24) == (pure[k + 1] >> 24)) {
                pairs.push_back(pure[k]);
                pairs.push_back(pure[k + 1]);
                k += 2;
            } else {
                mixed.push_back(pure[k] & 0xFFFFFF);
                k += 1;
            }
        }
        pure.swap(pairs);
    }

    free_tables(t);
    cudaError_t e = fp8    ? cudaMalloc(&t->d_Z8, z8.size())
                    : tf32 ? cudaMalloc(&t->d_Zt_hi, thi.size() * sizeof(float))
                           : cudaMalloc(&t->d_Zhi, hi.size() * sizeof(__nv_bfloat16));
    if (e == cudaSuccess && tf32) e = cudaMalloc(&t->d_Zt_lo, tlo.size() * sizeof(float));
    if (e == cudaSuccess && tf32) e = cudaMemcpy(t->d_Zt_hi, thi.data(), thi.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && tf32) e = cudaMemcpy(t->d_Zt_lo, tlo.data(), tlo.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && fp8) e = cudaMalloc(&t->d_sfb, sfb.size());
    if (e == cudaSuccess && fp8) e = cudaMemcpy(t->d_Z8, z8.data(), z8.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && fp8) e = cudaMemcpy(t->d_sfb, sfb.data(), sfb.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&t->d_fwd, fwd.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(t->d_fwd, fwd.data(), fwd.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && split) e = cudaMalloc(&t->d_Zlo, lo.size() * sizeof(__nv_bfloat16));
    if (e == cudaSuccess && !pure.empty()) e = cudaMalloc(&t->d_pure, pure.size() * sizeof(int));
    if (e == cudaSuccess && !mixed.empty()) e = cudaMalloc(&t->d_mixed, mixed.size() * sizeof(int));
    if (e == cudaSuccess && !fp8 && !tf32)
        e = cudaMemcpy(t->d_Zhi, hi.data(), hi.size() * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && split)
        e = cudaMemcpy(t->d_Zlo, lo.data(), lo.size() * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !pure.empty())
        e = cudaMemcpy(t->d_pure, pure.data(), pure.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !mixed.empty())
        e = cudaMemcpy(t->d_mixed, mixed.data(), mixed.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_tables(t);
        c->err = std::string("tensor-core table upload: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? RTLB_E_OOM : RTLB_E_CUDA;
    }
    const int box_rows = pair ? N4 / 2 : N4;
    const bool maps_ok =
        fp8 ? encode_z8_map(&t->tmZhi, t->d_Z8, N4, KP8, terms * n_phase)
            : tf32 ? (encode_zt_map(&t->tmZhi, t->d_Zt_hi, N4, n_phase) && encode_zt_map(&t->tmZlo, t->d_Zt_lo, N4, n_phase))
                   : (encode_z_map(&t->tmZhi, t->d_Zhi, N4, KP, n_phase, box_rows) &&
                      (!split || encode_z_map(&t->tmZlo, t->d_Zlo, N4, KP, n_phase, box_rows)));
    if (!maps_ok) {
        free_tables(t);
        c->err = "tensor map encoding for the phase tables failed";
        return RTLB_E_CUDA;
    }
    if (!split && !tf32) t->tmZlo = t->tmZhi;
    t->N4 = N4;
    t->KP = KP;
    t->C = C;
    t->n_phase = n_phase;
    t->mode = mode;
    t->pair = pair;
    t->n_pure = pair ? (int)pure.size() / 2 : (int)pure.size();
    t->n_mixed = (int)mixed.size();
    t->stages = stages;
    t->gather = gather;
    t->gtaps = gtaps;
    t->tmG_ptr[0] = t->tmG_ptr[1] = nullptr;
    t->smem = pair ? smem_bytes_pair(N4, stages)
                   : (mode == 4 ? tc_fp8_smem_bytes(N4, stages)
                                : (mode == 6 ? tc_fp8x_smem_bytes(N4, stages)
                                             : (tf32 ? tc_tf32_smem_bytes(N4, stages)
                                                     : smem_bytes(N4, mode, stages, gather))));
    return RTLB_OK;
}

rtlb_status tc_step(rtlb_ctx *c, const StepParams &p, cudaStream_t s)
{
    TcState *t = state_of(c);
    if (!t || (!t->d_Zhi && !t->d_Z8 && !t->d_Zt_hi)) {
        c->err = "tensor-core tables are not prepared";
        return RTLB_E_STATE;
    }
    const int which = (p.S == c->S[0]) ? 0 : 1;
    const bool gather = p.taps_o != nullptr;
    if (gather) {
        if (!t->gather) {
            c->err = "this tensor-core form has no gather (bilinear) load";
            return RTLB_E_STATE;
        }
        if (t->tmG_ptr[which] != p.S) {
            if (!encode_gather_map(&t->tmG[which], p.S, c->nx, c->nz, c->n)) {
                c->err = "tensor map encoding for the gather windows failed";
                return RTLB_E_CUDA;
            }
            t->tmG_ptr[which] = p.S;
        }
    }
    if (!gather && (!t->tmS_ready[which] || t->tmS_ptr[which] != p.S)) {
        if (!encode_state_map(&t->tmS[which], p.S, c->nsites(), c->n)) {
            c->err = "tensor map encoding for the state failed";
            return RTLB_E_CUDA;
        }
        t->tmS_ready[which] = true;
        t->tmS_ptr[which] = p.S;
    }
    if (t->n_pure > 0) {
        TcParams tp;
        tp.coef = p.coef;
        tp.dir = p.dir;
        tp.inflow = p.inflow;
        tp.S_new = p.S_new;
        tp.tiles = t->d_pure;
        tp.fwd = t->d_fwd;
        tp.n_tiles = t->n_pure;
        tp.nx = p.nx;
        tp.nz = p.nz;
        tp.n = p.n;
        tp.bcbits = pack_bc(p.bc);
        tp.err = t->d_err;
        tp.stall = t->stall_next;
        t->stall_next = 0;
        if (gather) tp.P = p.S;
        cudaError_t e = cudaSuccess;
        if (t->mode == 4) {
            e = launch_step_tc_fp8(t->tmS[which], t->tmZhi, tp, t->d_sfb, t->N4, t->stages, t->n_phase,
                                   std::min(t->sm_count, t->n_pure), s);
        } else if (t->mode == 6) {
            e = launch_step_tc_fp8x(t->tmS[which], t->tmZhi, tp, t->d_sfb, t->N4, t->stages, t->n_phase,
                                    std::min(t->sm_count, t->n_pure), s);
        } else if (t->mode == 5) {
            e = launch_step_tc_tf32(t->tmS[which], t->tmZhi, t->tmZlo, tp, t->N4, t->stages,
                                    std::min(t->sm_count, t->n_pure), s);
        } else if (t->pair) {
            const int grid = 2 * std::min(t->sm_count / 2, t->n_pure);
            e = cudaFuncSetAttribute(k_step_tc_pair, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t->smem);
            if (e == cudaSuccess)
                k_step_tc_pair<<<grid, kThreads, t->smem, s>>>(t->tmS[which], t->tmZhi, t->tmZlo, tp, t->N4, t->stages);
        } else {
            const int grid = std::min(t->sm_count, t->n_pure);
            auto launch = [&](auto kern) {
                e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t->smem);
                if (e == cudaSuccess)
                    kern<<<grid, kThreads, t->smem, s>>>(gather ? t->tmG[which] : t->tmS[which], t->tmZhi, t->tmZlo, tp,
                                                         t->N4, t->stages, t->gtaps);
            };
            if (t->mode == 3) launch(gather ? k_step_tc<3, true> : k_step_tc<3, false>);
            else if (t->mode == 2) launch(gather ? k_step_tc<2, true> : k_step_tc<2, false>);
            else launch(gather ? k_step_tc<1, true> : k_step_tc<1, false>);
        }
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) {
            c->err = std::string("tensor-core launch: ") + cudaGetErrorString(e);
            return RTLB_E_CUDA;
        }
    }
    if (t->n_mixed > 0) {
        StepParams q = p;
        q.tile_list = t->d_mixed;
        q.n_tiles = t->n_mixed;
        q.tile_span = kTileM;
        const cudaError_t e = launch_step_fp32(q, s);
        if (e != cudaSuccess) {
            c->err = std::string("mixed-tile launch: ") + cudaGetErrorString(e);
            return RTLB_E_CUDA;
        }
    }
    return RTLB_OK;
}

rtlb_status tc_arm_stall(rtlb_ctx *c)
{
    TcState *t = state_of(c);
    if (!t || (!t->d_Zhi && !t->d_Z8 && !t->d_Zt_hi)) {
        c->err = "the stall hook needs a tensor-core precision with its medium set";
        return RTLB_E_STATE;
    }
    if (t->mode >= 4) {
        c->err = "the stall hook covers the bf16-class kernels only";
        return RTLB_E_UNSUPPORTED;
    }
    t->stall_next = 1;
    return RTLB_OK;
}

rtlb_status tc_check_error(rtlb_ctx *c, cudaStream_t s)
{
    TcState *t = state_of(c);
    if (!t) return RTLB_OK;
    if (cudaMemcpyAsync(t->h_err, t->d_err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        c->err = "reading the tensor-core error flag failed";
        return RTLB_E_CUDA;
    }
    if (*t->h_err) {
        char buf[128];
        snprintf(buf, sizeof(buf), "tensor-core step gave up waiting (code %d)", *t->h_err);
        c->err = buf;
        cudaMemsetAsync(t->d_err, 0, sizeof(int), s);
        return RTLB_E_TIMEOUT;
    }
    return RTLB_OK;
}

bool tc_encode_state_map(CUtensorMap *m, const float *S, size_t nsites, int n) { return encode_state_map(m, S, nsites, n); }

bool tc_encode_f32_2d(CUtensorMap *m, const float *base, uint64_t inner, uint64_t outer, uint32_t box_inner,
                      uint32_t box_outer)
{
    auto fn = encode_fn();
    if (!fn || inner % 4 != 0) return false;
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    cuuint64_t strides[1] = {(cuuint64_t)inner * 4};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool tc_encode_table_map(CUtensorMap *m, const __nv_bfloat16 *Z, int N4, int KP, int n_phase, int box_rows)
{
    return encode_z_map(m, Z, N4, KP, n_phase, box_rows);
}

bool tc_table_maps(const rtlb_ctx *c, CUtensorMap *zhi, CUtensorMap *zlo, const float **fwd)
{
    const TcState *t = static_cast<const TcState *>(c->tc);
    if (!t || !t->d_Zhi || t->pair || t->mode == 4) return false;
    *zhi = t->tmZhi;
    *zlo = t->tmZlo;
    *fwd = t->d_fwd;
    return true;
}

bool tc_pure_tiles(const rtlb_ctx *c, std::vector<int> &out)
{
    const TcState *t = static_cast<const TcState *>(c->tc);
    if (!t || t->pair) return false;
    out.assign(t->n_pure, 0);
    return t->n_pure == 0 || cudaMemcpy(out.data(), t->d_pure, t->n_pure * sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess;
}

void tc_mixed_list(const rtlb_ctx *c, const int **list, int *count)
{
    const TcState *t = static_cast<const TcState *>(c->tc);
    *list = t ? t->d_mixed : nullptr;
    *count = t ? t->n_mixed : 0;
}

bool tc_gather(const rtlb_ctx *c)
{
    const TcState *t = c ? static_cast<const TcState *>(c->tc) : nullptr;
    return t && t->gather;
}

bool tc_form(const rtlb_ctx *c, int *pair, int *stages)
{
    const TcState *t = c ? static_cast<const TcState *>(c->tc) : nullptr;
    if (!t || (!t->d_Zhi && !t->d_Z8 && !t->d_Zt_hi)) return false;
    *pair = t->pair ? 1 : 0;
    *stages = t->stages;
    return true;
}

int tc_mixed_tiles(const rtlb_ctx *c)
{
    const TcState *t = static_cast<const TcState *>(c->tc);
    return t ? t->n_mixed : 0;
}

void tc_release(rtlb_ctx *c)
{
    TcState *t = state_of(c);
    if (!t) return;
    free_tables(t);
    cudaFree(t->d_err);
    cudaFreeHost(t->h_err);
    delete t;
    c->tc = nullptr;
}

}  // namespace rtlb
