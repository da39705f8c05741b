// 3xTF32 tensor-core form of the fused collide+stream step (precision
// RTLB_PREC_TF32X3, n in {8, 16, 32}): the float32-accuracy contraction of
// Eq. 11/25 on the tensor cores.
//
// Per tile of 128 consecutive sites, with x = beta * S~ (float32):
//
//   E  <- (alpha + beta c_d) S~                          (float32, converters -> TMEM)
//   D  <- A_hi . Zhi^T + A_hi . Zlo^T + A_lo . Zhi^T     (tcgen05.mma kind::tf32, K = 8)
//   S_new(x + c_d, d) = E + D                           (epilogue, float32)
//
// where A_hi = tf32(x) and A_lo = tf32(x - A_hi) (round to nearest), and
// Zhi / Zlo are the tf32 hi and lo parts of the table with its forward
// blocks taken out (prepared on the host from float64).  Each split operand
// carries about 22 significand bits; the dropped A_lo . Zlo product is below
// 2^-22 of each term.
//
// The exact part E is kept out of the MMA accumulator on purpose: the tensor
// core rounds each MMA instruction's float32 sum toward zero (measured on the
// B300: about -0.9 ulp of the accumulator per kind::tf32 instruction), so an
// accumulator that starts from E -- in clear air almost all of the radiance --
// would lose ~0.5-1 ulp of the whole radiance per instruction, 48
// instructions per step at n = 32, and the bias would build up step after
// step.  Started from zero, D holds only the scattered part and its
// truncation is relative to that part; E + D is one round-to-nearest add.
//
// Memory plan at n = 32.  TMEM (512 columns): two accumulators D and two
// regions E, so every role can run a tile ahead of the next (the converters
// of tile i + 2 and its MMAs wait only for the epilogue of tile i).  Shared
// memory: the split table (2 x 64 KB), a ring of split state chunks (a K
// chunk is 32 tf32 values = 8 directions = one staging slot = one 128-byte
// swizzle row; hi and lo, 16 KB each; one ring slot per converter group at
// n = 32, two below) and two staging slots, with the state chunk a few slots
// ahead prefetched into L2.  Because D starts from zero, the MMAs need not
// wait for the whole tile: the MMA thread takes chunk j as soon as its group
// has written it (a_full) and releases the ring slot when those MMAs complete
// (a_empty).  (A layout with the state operand in tensor memory and one E
// region handed back per slot coupled each tile's conversion to the previous
// tile's epilogue and measured 0.59 of HBM at 1024x1024.)
//
// Warp roles as in the bf16 kernel: warps 0-7 epilogue, 8-15 converters (two
// groups of four on alternate staging slots), 16 TMA producer, 17 MMA issuer.
// Every wait is bounded (about 2 s); on timeout the CTA records an error code,
// drains what it issued and leaves.
#include <cuda.h>

#include <algorithm>

#include "step_common.cuh"
#include "tc.h"
#include "tc_common.cuh"
#include "tc_ptx.cuh"

namespace rtlb {

namespace {

using namespace tcptx;
using namespace tccommon;

constexpr int kChunkK = 32;   // tf32 K values per chunk: 8 directions, one 128-byte row

// Instruction descriptor: D f32, A/B tf32 (format 2), both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int m, int n)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// D[tmem] (+)= A[smem] . B[smem]^T, tf32 operands, f32 accumulate, M = 128.
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// tf32 value nearest to x (ties away from zero), as float32 bits.
__device__ __forceinline__ uint32_t to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// A ring slots per converter group (shared memory, 32 KB each: hi and lo)
__host__ __device__ constexpr int tf32_ring(int N4) { return N4 >= 128 ? 1 : 2; }
constexpr uint32_t kRingBytes = (uint32_t)kTileM * 128u;   // one term of one chunk

#ifndef RTLB_TC_TF32_PREFETCH_SLOTS
#define RTLB_TC_TF32_PREFETCH_SLOTS 4
#endif

__global__ void __launch_bounds__(kThreads, 1)
    k_step_tc_tf32(const __grid_constant__ CUtensorMap tmS, const __grid_constant__ CUtensorMap tmZhi,
                   const __grid_constant__ CUtensorMap tmZlo, TcParams p, int N4, int stages)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const int G = N4 / kChunkK;                    // K chunks = staging slots per tile
    const int n = p.n;
    const int nsites = p.nx * p.nz;
    const uint32_t z_chunk = (uint32_t)N4 * 128u;  // bytes per K chunk of one table part
    const int Rg = tf32_ring(N4);                  // A ring slots per converter group
    const int colE = 2 * N4;                       // TMEM: D[b] at b * 4n, E[b] at 2 * 4n + b * 4n
    const uint32_t tcols = N4 * 4 <= 128 ? 128u : (N4 * 4 <= 256 ? 256u : 512u);

    uint8_t *sZ = smem;
    uint8_t *sZlo = sZ + G * z_chunk;
    uint8_t *sRing = sZlo + G * z_chunk;           // [2 Rg][hi, lo][128 rows x 128 B]
    uint8_t *sStage = sRing + (size_t)2 * Rg * 2 * kRingBytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sStage + (size_t)stages * kStageBytes);
    uint64_t *st_full = bars;
    uint64_t *st_empty = st_full + stages;
    uint64_t *a_full = st_empty + stages;      // [2 Rg] a group wrote a ring slot
    uint64_t *a_empty = a_full + 2 * Rg;       // [2 Rg] the MMAs on a ring slot completed
    uint64_t *acc_full = a_empty + 2 * Rg;     // [2]
    uint64_t *acc_empty = acc_full + 2;        // [2] the epilogue has read D[b] and E[b]
    uint64_t *z_full = acc_empty + 2;          // [1]
    uint64_t *drain = z_full + 1;              // [1]
    uint64_t *z_free = drain + 1;              // [1]
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(z_free + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    int8_t *s_cx = reinterpret_cast<int8_t *>(tmem_slot + 2);   // [n]
    int8_t *s_cz = s_cx + kMaxDirs;                              // [n]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(smem_u32(&st_full[s]), 1);
            mbar_init(smem_u32(&st_empty[s]), 4);
        }
        for (int k = 0; k < 2 * Rg; ++k) {
            mbar_init(smem_u32(&a_full[k]), 4);
            mbar_init(smem_u32(&a_empty[k]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&acc_full[b]), 1);
            mbar_init(smem_u32(&acc_empty[b]), kEpiWarps);
        }
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
                    mbar_expect_tx(zb, 2u * G * z_chunk);
                    for (int c = 0; c < G; ++c) {
                        tma_load_3d(smem_u32(sZ + c * z_chunk), &tmZhi, zb, kChunkK * c, 0, cls);
                        tma_load_3d(smem_u32(sZlo + c * z_chunk), &tmZlo, zb, kChunkK * c, 0, cls);
                    }
                    prev_cls = cls;
                }
                for (int j = 0; j < G && ok; ++j) {
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
                    if (RTLB_TC_TF32_PREFETCH_SLOTS > 0) {
                        // few staging slots fit beside the table and the ring: the
                        // chunk a few slots ahead goes to L2 meanwhile
                        const int ahead = i * G + j + RTLB_TC_TF32_PREFETCH_SLOTS;
                        const int ia = ahead / G, ja = ahead - ia * G;
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
            const uint32_t idesc = idesc_tf32(kTileM, N4);
            // descriptors of the table parts and ring slots; a byte offset o (a
            // multiple of 16) moves a descriptor by o >> 4 (its address field)
            const uint64_t bh0 = sw128_desc(smem_u32(sZ)), bl0 = sw128_desc(smem_u32(sZlo));
            const uint64_t ar0 = sw128_desc(smem_u32(sRing));
            int prev_cls = -1;
            uint32_t zl = 0, mc[2] = {0, 0};
            bool ok = true, issued = false;
            for (int i = 0; i < T && ok; ++i) {
                const int cls = p.tiles[t_begin + i] >> 24;
                const int b = i & 1;
                if (cls != prev_cls) {
                    ok = mbar_wait(smem_u32(z_full), zl & 1, abort_flag, p.err, kErrTimeoutMma);
                    ++zl;
                    prev_cls = cls;
                    if (!ok) break;
                }
                // the epilogue of tile i - 2 has read accumulator b
                ok = mbar_wait(smem_u32(&acc_empty[b]), ((i >> 1) & 1) ^ 1, abort_flag, p.err, kErrTimeoutMma);
                if (!ok) break;
                const uint32_t d_tmem = tmem + (uint32_t)(b * N4);
                for (int j = 0; j < G && ok; ++j) {
                    const int g = j & 1;
                    const uint32_t m = mc[g]++;
                    const int k = g * Rg + (int)(m % (uint32_t)Rg);
                    ok = mbar_wait(smem_u32(&a_full[k]), (m / (uint32_t)Rg) & 1, abort_flag, p.err, kErrTimeoutMma);
                    if (!ok) break;
                    tc_fence_after();
                    const uint64_t ah = ar0 + (uint64_t)((2u * k * kRingBytes) >> 4), al = ah + (kRingBytes >> 4);
                    const uint64_t bh = bh0 + (uint64_t)((j * z_chunk) >> 4), bl = bl0 + (uint64_t)((j * z_chunk) >> 4);
#pragma unroll
                    for (int kk = 0; kk < kChunkK / 8; ++kk) {       // K = 8 per instruction (32 bytes)
                        // the tile's first instruction starts D from zero
                        mma_tf32(d_tmem, ah + 2 * kk, bh + 2 * kk, idesc, (j | kk) ? 1u : 0u);
                        mma_tf32(d_tmem, ah + 2 * kk, bl + 2 * kk, idesc, 1u);
                        mma_tf32(d_tmem, al + 2 * kk, bh + 2 * kk, idesc, 1u);
                    }
                    mma_commit(smem_u32(&a_empty[k]));
                    issued = true;
                }
                if (!ok) break;
                mma_commit(smem_u32(&acc_full[b]));
                if (i + 1 < T && (p.tiles[t_begin + i + 1] >> 24) != cls) mma_commit(smem_u32(z_free));
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
        const int half = r / kHalfSites, hr = r % kHalfSites;
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        const int ring = stages / 2;
        uint32_t gq = 0, mc = 0;
        bool ok = true;
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
            // the epilogue of tile i - 2 has read E[b]
            ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&acc_empty[b]), ((i >> 1) & 1) ^ 1, abort_flag, p.err,
                                                   kErrTimeoutConverter));
            if (!ok) break;
            tc_fence_after();
            const uint32_t eb = tmem + lane_base + (uint32_t)(colE + b * N4);
            const float *fwd = p.fwd + (size_t)(entry >> 24) * n;
            for (int j = grp; j < G && ok; j += 2) {
                const int d_beg = kDirsPerStage * j;
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
                const uint32_t m = mc++;
                const int ka = grp * Rg + (int)(m % (uint32_t)Rg);
                ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&st_full[s]), (local / (uint32_t)ring) & 1, abort_flag,
                                                       p.err, kErrTimeoutConverter));
                // the MMAs on this group's ring slot completed
                ok = ok && __all_sync(0xffffffffu, mbar_wait(smem_u32(&a_empty[ka]), ((m / (uint32_t)Rg) & 1) ^ 1,
                                                             abort_flag, p.err, kErrTimeoutConverter));
                if (!ok) break;
                const float4 *stg = reinterpret_cast<const float4 *>(sStage + (size_t)s * kStageBytes) +
                                    half * (kDirsPerStage * kHalfSites) + hr;
                // this row of the ring slot: 128 bytes (32 tf32) per term, 16-byte
                // units at position u ^ (r & 7) (128-byte swizzle)
                uint8_t *rh = sRing + (size_t)2 * ka * kRingBytes + (uint32_t)r * 128u;
                uint8_t *rl = rh + kRingBytes;
#pragma unroll
                for (int dl = 0; dl < kDirsPerStage; dl += 2) {
                    const int d = d_beg + dl;
                    float4 v0 = stg[dl * kHalfSites], v1 = stg[(dl + 1) * kHalfSites];
                    v0.x += cf.w;                               // emission (I only)
                    v1.x += cf.w;
                    const float sv[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
                    const float g0 = fmaf(cf.z, fw[dl], cf.y), g1 = fmaf(cf.z, fw[dl + 1], cf.y);
                    float init[8];
                    uint32_t hi[8], lo[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        init[k] = fmaf(cf.x, sv[k], (k < 4 ? g0 : g1) * sv[k]);   // exact float32 part
                        const float x = cf.z * sv[k];                              // beta S~
                        hi[k] = to_tf32(x);
                        lo[k] = to_tf32(x - __uint_as_float(hi[k]));
                    }
                    tmem_st8(eb + 4 * d, init);
                    const uint32_t u0 = (uint32_t)dl, u1 = (uint32_t)dl + 1u;   // the two 16-byte units of this pair
                    const uint32_t o0 = ((u0 ^ (uint32_t)(r & 7)) << 4), o1 = ((u1 ^ (uint32_t)(r & 7)) << 4);
                    *reinterpret_cast<uint4 *>(rh + o0) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                    *reinterpret_cast<uint4 *>(rh + o1) = make_uint4(hi[4], hi[5], hi[6], hi[7]);
                    *reinterpret_cast<uint4 *>(rl + o0) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
                    *reinterpret_cast<uint4 *>(rl + o1) = make_uint4(lo[4], lo[5], lo[6], lo[7]);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&st_empty[s]));
                tmem_wait_st();
                fence_proxy_async();                        // the ring is read by the tensor core
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&a_full[ka]));
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int q = warp & 3;
        const int dhalf = warp >> 2;
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
            for (int d0 = dbeg; d0 < dbeg + dn; d0 += 4) {
                float v[16], e[16];
                tmem_ld16(tmem + lane_base + (uint32_t)(b * N4 + 4 * d0), v);
                tmem_ld16(tmem + lane_base + (uint32_t)(colE + b * N4 + 4 * d0), e);
#pragma unroll
                for (int k = 0; k < 16; ++k) v[k] += e[k];
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

}  // namespace

size_t tc_tf32_smem_bytes(int N4, int stages)
{
    const int G = N4 / kChunkK;
    const size_t b = (size_t)2 * G * N4 * 128 + (size_t)2 * tf32_ring(N4) * 2 * kRingBytes + (size_t)stages * kStageBytes +
                     (size_t)(2 * stages + 4 * tf32_ring(N4) + 7) * 8 + 16 + 2 * kMaxDirs;
    return b + 1024;  // alignment slack
}

cudaError_t launch_step_tc_tf32(const CUtensorMap &tmS, const CUtensorMap &tmZhi, const CUtensorMap &tmZlo,
                                const TcParams &p, int N4, int stages, int grid, cudaStream_t s)
{
    if (N4 % kChunkK != 0 || N4 > 128 || stages < 2 || stages % 2 != 0) return cudaErrorInvalidValue;
    const size_t smem = tc_tf32_smem_bytes(N4, stages);
    if (smem > (size_t)kSmemLimit) return cudaErrorInvalidValue;
    const cudaError_t e = cudaFuncSetAttribute(k_step_tc_tf32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_step_tc_tf32<<<grid, kThreads, smem, s>>>(tmS, tmZhi, tmZlo, p, N4, stages);
    return cudaGetLastError();
}

}  // namespace rtlb
