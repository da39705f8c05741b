// FP8 (e4m3, block-scaled) tensor-core form of the fused collide+stream step.
//
// Same contraction as the bf16 forms (Eq. 11/25 per 128-site tile, the
// float32 part alpha * S~ and the forward block written into TMEM first), but
// the scattered part's operands are e4m3 with UE8M0 block scales:
//
//   A[r][k] = e4m3(beta S~[r][k] / 2^ea[r][kb]),  one scale per site and
//             8-direction slot (32 K elements = one MX block: kb = k / 32)
//   B[c][k] = e4m3(Z[c][k] / 2^eb[c][kb]),        one scale per table row and
//             32-element block (prepared on the host)
//   D[r][c] += sum_kb 2^(ea + eb) sum_{k in kb} A[r][k] B[c][k]
//
// issued as tcgen05.mma kind::mxf8f6f4.block_scale (scale_vec::1X, K = 32 per
// instruction), so every block keeps its own scale and the products are
// exact; the tensor core accumulates in float32.
//
// TMEM holds one accumulator (at n = 64 two would fill all 512 columns and
// leave none for the scales) and the scales, each region on an 8-column
// boundary.  The epilogue hands it back one 8-direction
// slot (32 columns) at a time: the next tile's converters write a slot's
// float32 init as soon as the epilogue has read that slot, so conversion of
// tile i + 1 trails the epilogue of tile i instead of waiting for all of it.
// A converter that passed a slot's hand-off also knows the previous tile's
// MMAs completed, so the A operand and its scales need no separate barrier.
//
// Warp roles and the staging pipeline are those of the bf16 kernel: warps 0-7
// epilogue, 8-15 converters (two groups on alternate staging slots), 16 TMA
// producer, 17 MMA issuer.  Every wait is bounded (about 2 s); on timeout the
// CTA records an error code and leaves.
#include <cuda.h>
#include <cuda_fp8.h>

#include <algorithm>

#include "step_common.cuh"
#include "tc.h"
#include "tc_common.cuh"
#include "tc_ptx.cuh"

namespace rtlb {

namespace {

using namespace tcptx;
using namespace tccommon;

// Scale-factor regions in TMEM start on 8-column boundaries (the layout the
// block-scaled MMA was checked with): one 8-column group per K step for A
// (columns + m / 32 used), one per (class, set of four K steps) for B
// (columns + n / 32 used, N4 <= 256).
constexpr int kSfCols = 8;

__global__ void __launch_bounds__(kThreads, 1)
    k_step_tc_fp8(const __grid_constant__ CUtensorMap tmS, const __grid_constant__ CUtensorMap tmZ, TcParams p,
                  const uint8_t *__restrict__ sfb, int N4, int stages, int n_phase, uint32_t tcols, int colA, int colB)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const int C8 = (N4 + 127) / 128;               // 128-byte (128-element) K chunks
    const int ksteps = N4 / 32;                    // MMA K steps = 8-direction slots
    const int n = p.n;
    const int nsites = p.nx * p.nz;
    const int groups = n / kDirsPerStage;          // slots per tile
    const uint32_t z_chunk = (uint32_t)N4 * 128u;
    const uint32_t a_chunk = (uint32_t)kTileM * 128u;
    const int bcols = N4 / 32;                     // TMEM columns of one B scale set used (row n -> column n / 32)
    const int bsets = (ksteps + 3) / 4;            // four K steps per set (one byte each)

    uint8_t *sZ = smem;
    uint8_t *sA = sZ + C8 * z_chunk;
    uint8_t *sStage = sA + C8 * a_chunk;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sStage + (size_t)stages * kStageBytes);
    uint64_t *st_full = bars;
    uint64_t *st_empty = st_full + stages;
    uint64_t *d_free = st_empty + stages;      // [groups] the epilogue has read a slot's columns
    uint64_t *t_ready = d_free + groups;       // converters: A, scales and init of a tile written
    uint64_t *acc_full = t_ready + 1;          // MMAs of a tile completed
    uint64_t *z_full = acc_full + 1;
    uint64_t *drain = z_full + 1;
    uint64_t *z_free = drain + 1;              // the resident table's last MMAs completed
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(z_free + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    int8_t *s_cx = reinterpret_cast<int8_t *>(tmem_slot + 2);   // [n]
    int8_t *s_cz = s_cx + kMaxDirs;                              // [n]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // epilogue warps reading each slot: four (one per quadrant), eight when a
    // slot spans both halves of the directions (n = 8)
    const int dfree_count = (n / 2) % kDirsPerStage == 0 ? 4 : 8;

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(smem_u32(&st_full[s]), 1);
            mbar_init(smem_u32(&st_empty[s]), 4);
        }
        for (int j = 0; j < groups; ++j) mbar_init(smem_u32(&d_free[j]), dfree_count);
        mbar_init(smem_u32(t_ready), kConvWarps);
        mbar_init(smem_u32(acc_full), 1);
        mbar_init(smem_u32(z_full), 1);
        mbar_init(smem_u32(drain), 1);
        mbar_init(smem_u32(z_free), 1);
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

    // B scales of every class, resident for the whole launch: class ph, set
    // st, column cc hold rows n = 32 cc + l at lane l of every quadrant, the
    // byte k of the cell being K step 4 st + k
    if (warp < 4) {
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        for (int ph = 0; ph < n_phase; ++ph)
            for (int st = 0; st < bsets; ++st)
                for (int cc = 0; cc < bcols; ++cc) {
                    const int row = 32 * cc + lane;
                    uint32_t cell = 0;
                    for (int k = 0; k < 4; ++k) {
                        const int ks = 4 * st + k;
                        if (ks < ksteps) cell |= (uint32_t)sfb[((size_t)ph * N4 + row) * ksteps + ks] << (8 * k);
                    }
                    tmem_st1(tmem + lane_base + (uint32_t)(colB + (ph * bsets + st) * kSfCols + cc), cell);
                }
        tmem_wait_st();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    const int t_begin = (int)((long long)p.n_tiles * blockIdx.x / gridDim.x);
    const int t_end = (int)((long long)p.n_tiles * (blockIdx.x + 1) / gridDim.x);
    const int T = t_end - t_begin;

    if (warp == kProdWarp) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            int prev_cls = -1;
            uint32_t gq[2] = {0, 0}, zr = 0;
            bool ok = true;
            for (int i = 0; i < T && ok; ++i) {
                const int e = p.tiles[t_begin + i];
                const int tile = e & 0xFFFFFF, cls = e >> 24;
                if (cls != prev_cls) {
                    if (i > 0) ok = mbar_wait(smem_u32(z_free), (zr++) & 1, abort_flag, p.err, kErrTimeoutProducer);
                    if (!ok) break;
                    const uint32_t zb = smem_u32(z_full);
                    mbar_expect_tx(zb, (uint32_t)C8 * z_chunk);
                    for (int c = 0; c < C8; ++c) tma_load_3d(smem_u32(sZ + c * z_chunk), &tmZ, zb, 128 * c, 0, cls);
                    prev_cls = cls;
                }
                for (int j = 0; j < groups && ok; ++j) {
                    const int gr = j & 1;
                    const uint32_t local = gq[gr]++;
                    const int s = ring_slot(gr, local, stages / 2);
                    ok = mbar_wait(smem_u32(&st_empty[s]), ((local / (uint32_t)(stages / 2)) & 1) ^ 1, abort_flag, p.err,
                                   kErrTimeoutProducer);
                    if (!ok) break;
                    const uint32_t fb = smem_u32(&st_full[s]);
                    mbar_expect_tx(fb, kStageBytes);
                    for (int h = 0; h < kTileM / kHalfSites; ++h)
                        tma_load_2d(smem_u32(sStage + (size_t)s * kStageBytes + h * (kStageBytes / 2)), &tmS, fb,
                                    4 * (tile * kTileM + h * kHalfSites), j * kDirsPerStage);
                }
            }
            // drain: wait (bounded) for the loads this thread issued into each stage
            for (int gr = 0; gr < 2; ++gr)
                for (uint32_t k = 0; k < (uint32_t)(stages / 2) && k < gq[gr]; ++k) {
                    const uint32_t local = gq[gr] - 1 - k;
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
            int prev_cls = -1;
            uint32_t zl = 0;
            bool ok = true, issued = false;
            for (int i = 0; i < T && ok; ++i) {
                const int cls = p.tiles[t_begin + i] >> 24;
                if (cls != prev_cls) {
                    ok = mbar_wait(smem_u32(z_full), zl & 1, abort_flag, p.err, kErrTimeoutMma);
                    ++zl;
                    prev_cls = cls;
                    if (!ok) break;
                }
                ok = mbar_wait(smem_u32(t_ready), i & 1, abort_flag, p.err, kErrTimeoutMma);
                if (!ok) break;
                tc_fence_after();
                for (int ks = 0; ks < ksteps; ++ks) {
                    const uint32_t off = (uint32_t)(ks & 3) * 32u;   // 32-byte K step within the 128-byte row
                    const uint64_t ad = sw128_desc(smem_u32(sA + (ks / 4) * a_chunk + off));
                    const uint64_t bd = sw128_desc(smem_u32(sZ + (ks / 4) * z_chunk + off));
                    const uint32_t sa = tmem + (uint32_t)(colA + kSfCols * ks);
                    const uint32_t sb = tmem + (uint32_t)(colB + (cls * bsets + ks / 4) * kSfCols);
                    mma_mxf8(tmem, ad, bd, idesc_mxf8(kTileM, N4, 0, ks & 3), sa, sb, 1u);
                }
                mma_commit(smem_u32(acc_full));
                if (i + 1 < T && (p.tiles[t_begin + i + 1] >> 24) != cls) mma_commit(smem_u32(z_free));
                issued = true;
            }
            if (issued) {
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
        const int half = r / kHalfSites, hr = r % kHalfSites;
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        const int ring = stages / 2;
        uint32_t gq = 0;
        bool ok = true;
        int e_next = T > 0 ? p.tiles[t_begin] : 0, e_after = T > 1 ? p.tiles[t_begin + 1] : 0;
        float4 cf_next = T > 0 ? load_coef(p.coef, (e_next & 0xFFFFFF) * kTileM + r, nsites) : float4{};
        for (int i = 0; i < T && ok; ++i) {
            const int entry = e_next;
            const float4 cf = cf_next;
            if (i + 1 < T) {
                e_next = e_after;
                cf_next = load_coef(p.coef, (e_next & 0xFFFFFF) * kTileM + r, nsites);
                if (i + 2 < T) e_after = p.tiles[t_begin + i + 2];
            }
            const float *fwd = p.fwd + (size_t)(entry >> 24) * n;
            for (int j = grp; j < groups && ok; j += 2) {
                const int d_beg = 8 * j;
                float fw[8];
#pragma unroll
                for (int k = 0; k < 8; k += 4) {
                    const float4 f = __ldg(reinterpret_cast<const float4 *>(fwd + d_beg + k));
                    fw[k] = f.x;
                    fw[k + 1] = f.y;
                    fw[k + 2] = f.z;
                    fw[k + 3] = f.w;
                }
                const uint32_t local = gq++;
                const int s = ring_slot(grp, local, ring);
                ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&st_full[s]), (local / (uint32_t)ring) & 1, abort_flag,
                                                       p.err, kErrTimeoutConverter));
                if (!ok) break;
                const float4 *stg = reinterpret_cast<const float4 *>(sStage + (size_t)s * kStageBytes) +
                                    half * (kDirsPerStage * kHalfSites) + hr;
                // block scale: largest |beta S~| of the slot's 32 values (rounding
                // to float32 is monotonic, so this is the largest rounded product)
                float amax = 0.f;
#pragma unroll
                for (int dl = 0; dl < kDirsPerStage; ++dl) {
                    float4 v = stg[dl * kHalfSites];
                    v.x += cf.w;
                    amax = fmaxf(amax, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
                }
                const int ea = block_exponent(fabsf(cf.z) * amax);
                const float inv = __uint_as_float((uint32_t)(127 - ea) << 23);   // 2^-ea, exact
                // the previous tile's epilogue has read this slot's columns, so
                // its MMAs (and their reads of A and its scales) completed
                ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&d_free[j]), (i & 1) ^ 1, abort_flag, p.err,
                                                       kErrTimeoutConverter));
                if (!ok) break;
                tc_fence_after();
                uint32_t packed[8];
#pragma unroll
                for (int dl = 0; dl < kDirsPerStage; dl += 2) {
                    const int d = d_beg + dl;
                    float4 v0 = stg[dl * kHalfSites], v1 = stg[(dl + 1) * kHalfSites];
                    v0.x += cf.w;                               // emission (I only)
                    v1.x += cf.w;
                    const float sv[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
                    const float g0 = fmaf(cf.z, fw[dl], cf.y), g1 = fmaf(cf.z, fw[dl + 1], cf.y);
                    float init[8], x[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        init[k] = fmaf(cf.x, sv[k], (k < 4 ? g0 : g1) * sv[k]);   // exact float32 part
                        x[k] = (cf.z * sv[k]) * inv;                              // beta S~ / 2^ea
                    }
                    tmem_st8(tmem + lane_base + (uint32_t)(4 * d), init);
                    packed[dl] = e4m3x2(x[0], x[1]) | (e4m3x2(x[2], x[3]) << 16);
                    packed[dl + 1] = e4m3x2(x[4], x[5]) | (e4m3x2(x[6], x[7]) << 16);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&st_empty[s]));
                // scale of (row r, K step j): lane r, column colA + 8 j + r / 32
                tmem_st1(tmem + lane_base + (uint32_t)(colA + kSfCols * j + q), (uint32_t)(ea + 127));
                // the slot's 32 bytes: chunk j / 4, 16-byte units 2 (j % 4) and 2 (j % 4) + 1
                const uint32_t base = (uint32_t)(j >> 2) * a_chunk + (uint32_t)r * 128u;
                const uint32_t u0 = 2u * (uint32_t)(j & 3);
                *reinterpret_cast<uint4 *>(sA + base + ((u0 ^ (uint32_t)(r & 7)) << 4)) =
                    make_uint4(packed[0], packed[1], packed[2], packed[3]);
                *reinterpret_cast<uint4 *>(sA + base + (((u0 + 1u) ^ (uint32_t)(r & 7)) << 4)) =
                    make_uint4(packed[4], packed[5], packed[6], packed[7]);
            }
            if (!ok) break;
            tmem_wait_st();
            fence_proxy_async();
            tc_fence_before();
            __syncwarp();
            // arrive for tile i only once t_ready's phase for tile i - 1 has
            // completed: a warp with no slot in a tile (group 1 at n = 8) would
            // otherwise run ahead and its arrivals for later tiles would
            // complete tile i's phase before the other group wrote A
            ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(t_ready), (i & 1) ^ 1, abort_flag, p.err,
                                                   kErrTimeoutConverter));
            if (!ok) break;
            if (lane == 0) mbar_arrive(smem_u32(t_ready));
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
            const int site = tile * kTileM + r;
            const int z = site / p.nx, x = site - z * p.nx;
            const bool interior = site < nsites && x > 0 && x < p.nx - 1 && z > 0 && z < p.nz - 1;
            ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(acc_full), i & 1, abort_flag, p.err, kErrTimeoutEpilogue));
            if (!ok) break;
            tc_fence_after();
            for (int d0 = dbeg; d0 < dbeg + dn; d0 += 4) {
                float v[16];
                tmem_ld16(tmem + lane_base + (uint32_t)(4 * d0), v);
                if (interior) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int d = d0 + k;
                        const long long t = (long long)d * nsites + site + s_cx[d] + (long long)s_cz[d] * p.nx;
                        __stcs(&out[t], make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]));
                    }
                } else if (site < nsites) {
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        push_store_xz(p.dir, p.inflow, p.bcbits, p.S_new, p.nx, p.nz, n, site, x, z, d0 + k,
                                   make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]));
                }
                // hand a slot back once this warp has read all of its columns
                const int next = d0 + 4;
                if (next % kDirsPerStage == 0 || next == dbeg + dn) {
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&d_free[(next - 1) / kDirsPerStage]));
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kMmaWarp) tmem_dealloc(tmem, tcols);
}

}  // namespace

int tc_fp8_tmem_columns(int N4, int n_phase)
{
    const int ksteps = N4 / 32, bsets = (ksteps + 3) / 4;
    return N4 + kSfCols * ksteps + n_phase * bsets * kSfCols;
}

size_t tc_fp8_smem_bytes(int N4, int stages)
{
    const int C8 = (N4 + 127) / 128, groups = N4 / 32;
    const size_t b = (size_t)C8 * N4 * 128 + (size_t)C8 * kTileM * 128 + (size_t)stages * kStageBytes +
                     (size_t)(2 * stages + groups + 5) * 8 + 16 + 2 * kMaxDirs;
    return b + 1024;  // alignment slack
}

cudaError_t launch_step_tc_fp8(const CUtensorMap &tmS, const CUtensorMap &tmZ, const TcParams &p, const uint8_t *sfb,
                               int N4, int stages, int n_phase, int grid, cudaStream_t s)
{
    const int cols = tc_fp8_tmem_columns(N4, n_phase);
    if (cols > 512) return cudaErrorInvalidValue;
    uint32_t tcols = 32;
    while (tcols < (uint32_t)cols) tcols <<= 1;
    const int colA = N4, colB = N4 + kSfCols * (N4 / 32);
    if (N4 % 32 != 0 || N4 > 256 || colA % kSfCols != 0 || colB % kSfCols != 0) return cudaErrorInvalidValue;
    const size_t smem = tc_fp8_smem_bytes(N4, stages);
    const cudaError_t e = cudaFuncSetAttribute(k_step_tc_fp8, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_step_tc_fp8<<<grid, kThreads, smem, s>>>(tmS, tmZ, p, sfb, N4, stages, n_phase, tcols, colA, colB);
    return cudaGetLastError();
}

}  // namespace rtlb
