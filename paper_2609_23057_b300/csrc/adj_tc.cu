// Tensor-core reverse step of the adjoint (4n in {32, 64, 128}), transposed-stream form.
//
// With nu^t = T^T lambda^{t+1} (the adjoint state already pulled back along
// the streaming), one reverse step of the affine step S^{t+1} = T (C S^t + c0)
// + b is, per site y:
//
//   lambda^t(y) = alpha nu(y) + beta Y(y),   Y = Z_c^T nu(y)   (Eq. 11 / 25 transposed)
//   nu^{t-1}(y - c_d, d) = lambda^t(y, d)    (push along -c_d; entries whose
//                                             source y + c_d left the lattice are 0)
//   dL/dalpha_y += <nu, S~>,  dL/dbeta_y += <Y, S~>,  S~ = S^t + e
//
// and the last step (t = 0) stores lambda^0 unpushed.  Y is one GEMM per tile
// of 128 sites with M = 128, N = K = 4n, on the tensor cores with nu and Z^T
// split into bf16 hi + lo (three MMAs: hi.hi, hi.lo, lo.hi; ~16 significand
// bits per operand, float32 accumulation).
//
// Warp roles as in the forward tensor-core step: warps 0-7 epilogue, 8-15
// converters (two groups on alternate staging slots; at 4n = 32 the tile has
// one slot and group 1 only reports), 16 TMA producer, 17 MMA issuer.  K is
// padded to whole 64-column chunks in shared memory and the tables; the MMAs
// stop at K = 4n.  TMEM holds two buffers of [Y | nu] (4 x 4n columns): the
// converters copy nu into TMEM beside the accumulator so the epilogue has both
// without reading nu again.  The epilogue reads S^t from HBM for the dot
// products; the two halves of a site's directions (warps q and q + 4) add
// into separate float64 accumulators that the chain rule sums in a fixed
// order, so no warp waits on another.  Tiles that mix phase classes go to the
// CUDA-core kernel.  Every
// wait is bounded (about 2 s); on timeout the CTA records an error code and
// leaves.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "rtlb_internal.h"
#include "step_common.cuh"
#include "tc.h"
#include "tc_common.cuh"
#include "tc_ptx.cuh"

namespace rtlb {

namespace {

using namespace tcptx;
using namespace tccommon;

constexpr uint32_t kAChunk = (uint32_t)kTileM * 128u;

// Shape constants of the form at 4n = N4.
template <int N4>
struct AdjTcShape {
    static constexpr int C = (N4 + 63) / 64;                 // 64-wide bf16 K chunks (K padded)
    static constexpr int G = N4 / 4 / kDirsPerStage;         // staging slots per tile
    static constexpr uint32_t ZChunk = (uint32_t)N4 * 128u;  // one K chunk of one table part
    static constexpr uint32_t TCols = 4u * N4;               // two buffers of [Y | nu]
};

struct AdjTcParams {
    const float4 *S;        // S^t, direction-major
    const float4 *coef;     // {alpha_hi, alpha_lo, beta, emission}
    const int *dirT;        // [2n] negated streaming offsets (the push of T^T)
    int bcbitsT;            // boundary kinds with inflow taken as vacuum
    float *nu_out;          // nu^{t-1} (push) or lambda^0 (no push)
    double *g_alpha, *g_beta;   // [2][nsites]: one half per epilogue warp half (summed later, in order)
    const int *tiles;       // tile | class << 24, sorted by class
    int n_tiles;
    int nx, nz, n;
    int push;
    int *err;
};

__device__ int g_adj_tc_err;

template <int kN4>
__global__ void __launch_bounds__(kThreads, 1)
    k_adj_step_tc(const __grid_constant__ CUtensorMap tmNu, const __grid_constant__ CUtensorMap tmZhi,
                  const __grid_constant__ CUtensorMap tmZlo, AdjTcParams p, int stages)
{
    constexpr int kC = AdjTcShape<kN4>::C, kGroups = AdjTcShape<kN4>::G;
    constexpr uint32_t kZChunk = AdjTcShape<kN4>::ZChunk;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const int n = p.n;
    const int nsites = p.nx * p.nz;

    uint8_t *sZ = smem;                                  // Z^T hi  [kC][kN4 rows][128 B]
    uint8_t *sZlo = sZ + kC * kZChunk;                   // Z^T lo
    uint8_t *sA = sZlo + kC * kZChunk;                   // nu hi   [kC][128 rows][128 B]
    uint8_t *sAlo = sA + kC * kAChunk;                   // nu lo
    uint8_t *sStage = sAlo + kC * kAChunk;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sStage + (size_t)stages * kStageBytes);
    uint64_t *st_full = bars;
    uint64_t *st_empty = st_full + stages;
    uint64_t *a_empty = st_empty + stages;     // [kC]
    uint64_t *t_ready = a_empty + kC;          // [2]
    uint64_t *acc_full = t_ready + 2;          // [2]
    uint64_t *acc_empty = acc_full + 2;        // [2]
    uint64_t *z_full = acc_empty + 2;
    uint64_t *drain = z_full + 1;
    uint64_t *z_free = drain + 1;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(z_free + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    int8_t *s_cx = reinterpret_cast<int8_t *>(tmem_slot + 2);   // negated offsets
    int8_t *s_cz = s_cx + kMaxDirs;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t tcols = AdjTcShape<kN4>::TCols;

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(smem_u32(&st_full[s]), 1);
            mbar_init(smem_u32(&st_empty[s]), 4);
        }
        for (int c = 0; c < kC; ++c) mbar_init(smem_u32(&a_empty[c]), 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&t_ready[b]), kConvWarps);
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
        s_cx[d] = (int8_t)p.dirT[d];
        s_cz[d] = (int8_t)p.dirT[n + d];
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
                    mbar_expect_tx(zb, 2u * kC * kZChunk);
                    for (int c = 0; c < kC; ++c) {
                        tma_load_3d(smem_u32(sZ + c * kZChunk), &tmZhi, zb, 64 * c, 0, cls);
                        tma_load_3d(smem_u32(sZlo + c * kZChunk), &tmZlo, zb, 64 * c, 0, cls);
                    }
                    prev_cls = cls;
                }
                for (int j = 0; j < kGroups && ok; ++j) {
                    const int gr = j & 1;
                    const uint32_t local = gq[gr]++;
                    const int s = ring_slot(gr, local, stages / 2);
                    ok = mbar_wait(smem_u32(&st_empty[s]), ((local / (uint32_t)(stages / 2)) & 1) ^ 1, abort_flag, p.err,
                                   kErrTimeoutProducer);
                    if (!ok) break;
                    const uint32_t fb = smem_u32(&st_full[s]);
                    mbar_expect_tx(fb, kStageBytes);
                    for (int h = 0; h < kTileM / kHalfSites; ++h)
                        tma_load_2d(smem_u32(sStage + (size_t)s * kStageBytes + h * (kStageBytes / 2)), &tmNu, fb,
                                    4 * (tile * kTileM + h * kHalfSites), j * kDirsPerStage);
                }
            }
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
            const uint32_t idesc = idesc_bf16(kTileM, kN4);
            int prev_cls = -1;
            uint32_t zl = 0;
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
                ok = mbar_wait(smem_u32(&t_ready[b]), (i >> 1) & 1, abort_flag, p.err, kErrTimeoutMma);
                if (!ok) break;
                tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(b * 2 * kN4);       // Y of buffer b
                for (int c = 0; c < kC; ++c) {
                    for (int kk = 0; kk < 4 && 64 * c + 16 * kk < kN4; ++kk) {   // K stops at 4n
                        const uint32_t ao = c * kAChunk + kk * 32, zo = c * kZChunk + kk * 32;
                        const uint64_t ah = sw128_desc(smem_u32(sA + ao)), al = sw128_desc(smem_u32(sAlo + ao));
                        const uint64_t zh = sw128_desc(smem_u32(sZ + zo)), zlo = sw128_desc(smem_u32(sZlo + zo));
                        mma_bf16(d_tmem, ah, zh, idesc, (c | kk) != 0 ? 1u : 0u);   // Y starts at zero
                        mma_bf16(d_tmem, ah, zlo, idesc, 1u);
                        mma_bf16(d_tmem, al, zh, idesc, 1u);
                    }
                    mma_commit(smem_u32(&a_empty[c]));
                }
                mma_commit(smem_u32(&acc_full[b]));
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
        const int grp = (warp - kConvWarp0) >> 2;
        const int r = q * 32 + lane;
        const int half = r / kHalfSites, hr = r % kHalfSites;
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        const int ring = stages / 2;
        uint32_t gq = 0;
        bool ok = true;
        for (int i = 0; i < T && ok; ++i) {
            const int b = i & 1;
            ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&acc_empty[b]), ((i >> 1) & 1) ^ 1, abort_flag, p.err,
                                                   kErrTimeoutConverter));
            if (!ok) break;
            tc_fence_after();
            const uint32_t nu_t = tmem + lane_base + (uint32_t)(b * 2 * kN4 + kN4);
            for (int c = 0; c < kC && ok; ++c) {
                const int j = 2 * c + grp;                 // this group's staging slot of K chunk c
                if (j >= kGroups) continue;                // 4n = 32: group 1 has no slot
                const int d_beg = kDirsPerStage * j;
                const uint32_t local = gq++;
                const int s = ring_slot(grp, local, ring);
                ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&st_full[s]), (local / (uint32_t)ring) & 1, abort_flag,
                                                       p.err, kErrTimeoutConverter));
                if (!ok) break;
                const float4 *stg = reinterpret_cast<const float4 *>(sStage + (size_t)s * kStageBytes) +
                                    half * (kDirsPerStage * kHalfSites) + hr;
                uint4 hi[4], lo[4];
#pragma unroll
                for (int dl = 0; dl < kDirsPerStage; dl += 2) {
                    const float4 v0 = stg[dl * kHalfSites], v1 = stg[(dl + 1) * kHalfSites];
                    const float x[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
                    tmem_st8(nu_t + (uint32_t)(4 * (d_beg + dl)), x);     // nu for the epilogue
                    uint32_t h[4], l[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        h[k] = pack_bf16(x[2 * k], x[2 * k + 1]);
                        const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&h[k]));
                        l[k] = pack_bf16(x[2 * k] - f.x, x[2 * k + 1] - f.y);
                    }
                    hi[dl >> 1] = make_uint4(h[0], h[1], h[2], h[3]);
                    lo[dl >> 1] = make_uint4(l[0], l[1], l[2], l[3]);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&st_empty[s]));
                // A chunk c is free once the previous tile's MMAs on it completed
                ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&a_empty[c]), (i & 1) ^ 1, abort_flag, p.err,
                                                       kErrTimeoutConverter));
                if (!ok) break;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint32_t gi = 4u * (uint32_t)grp + (uint32_t)k;
                    const uint32_t off = c * kAChunk + r * 128u + ((gi ^ (uint32_t)(r & 7)) << 4);
                    *reinterpret_cast<uint4 *>(sA + off) = hi[k];
                    *reinterpret_cast<uint4 *>(sAlo + off) = lo[k];
                }
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
        const int dhalf = warp >> 2;               // 0: first half of the directions, 1: second
        const int r = q * 32 + lane;
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        const int dn = n / 2, dbeg = dhalf * dn;
        float4 *out = reinterpret_cast<float4 *>(p.nu_out);
        double *ga = p.g_alpha + (size_t)dhalf * nsites, *gb = p.g_beta + (size_t)dhalf * nsites;
        bool ok = true;
        for (int i = 0; i < T && ok; ++i) {
            const int tile = p.tiles[t_begin + i] & 0xFFFFFF;
            const int b = i & 1;
            const int site = tile * kTileM + r;
            const bool valid = site < nsites;
            const int z = site / p.nx, x = site - z * p.nx;
            const bool interior = valid && x > 0 && x < p.nx - 1 && z > 0 && z < p.nz - 1;
            const float4 cf = valid ? __ldg(p.coef + site) : make_float4(0.f, 0.f, 0.f, 0.f);
            const double ga0 = valid ? ga[site] : 0.0, gb0 = valid ? gb[site] : 0.0;
            // the next tile's S (this thread's directions) on its way into L2
            if (i + 1 < T) {
                const int next = (p.tiles[t_begin + i + 1] & 0xFFFFFF) * kTileM + r;
                if (next < nsites)
                    for (int d = dbeg; d < dbeg + dn; ++d)
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(p.S + (size_t)d * nsites + next));
            }
            ok = __all_sync(0xffffffffu,
                            mbar_wait(smem_u32(&acc_full[b]), (i >> 1) & 1, abort_flag, p.err, kErrTimeoutEpilogue));
            if (!ok) break;
            tc_fence_after();
            const uint32_t yb = tmem + lane_base + (uint32_t)(b * 2 * kN4), nb = yb + (uint32_t)kN4;
            float pa = 0.f, pb = 0.f;
            for (int d0 = dbeg; d0 < dbeg + dn; d0 += 4) {
                // S first, so its latency overlaps the tensor-memory loads
                float4 sv4[4];
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    sv4[k] = valid ? __ldg(p.S + (size_t)(d0 + k) * nsites + site) : make_float4(0.f, 0.f, 0.f, 0.f);
                float y[16], nu[16];
                tmem_ld16(yb + (uint32_t)(4 * d0), y);
                tmem_ld16(nb + (uint32_t)(4 * d0), nu);
                if (!valid) continue;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int d = d0 + k;
                    float4 sv = sv4[k];
                    sv.x += cf.w;
                    const float svk[4] = {sv.x, sv.y, sv.z, sv.w};
                    float o[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const float m = nu[4 * k + c], yy = y[4 * k + c];
                        o[c] = fmaf(cf.x, m, fmaf(cf.y, m, cf.z * yy));      // alpha nu + beta Z^T nu
                        pa = fmaf(m, svk[c], pa);
                        pb = fmaf(yy, svk[c], pb);
                    }
                    const float4 val = make_float4(o[0], o[1], o[2], o[3]);
                    if (!p.push) {
                        out[(size_t)d * nsites + site] = val;
                    } else if (interior) {
                        out[(size_t)d * nsites + site + s_cx[d] + (long long)s_cz[d] * p.nx] = val;
                    } else {
                        push_store_xz(p.dirT, nullptr, p.bcbitsT, p.nu_out, p.nx, p.nz, n, site, x, z, d, val);
                    }
                }
            }
            if (valid) {
                ga[site] = ga0 + (double)pa;
                gb[site] = gb0 + (double)pb;
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

template <int N4>
size_t adj_tc_smem(int stages)
{
    constexpr int C = AdjTcShape<N4>::C;
    return (size_t)2 * C * AdjTcShape<N4>::ZChunk + (size_t)2 * C * kAChunk + (size_t)stages * kStageBytes +
           (size_t)(2 * stages + C + 9) * 8 + 16 + 2 * kMaxDirs + 1024;
}

size_t adj_tc_smem_n(int n, int stages)
{
    switch (4 * n) {
    case 32: return adj_tc_smem<32>(stages);
    case 64: return adj_tc_smem<64>(stages);
    case 128: return adj_tc_smem<128>(stages);
    default: return 0;
    }
}

template <int N4>
cudaError_t launch_tc(const CUtensorMap &tmNu, const CUtensorMap &tmZhi, const CUtensorMap &tmZlo, const AdjTcParams &p,
                      int stages, int grid, cudaStream_t s)
{
    const size_t smem = adj_tc_smem<N4>(stages);
    static bool attr = false;
    if (!attr) {
        const cudaError_t e = cudaFuncSetAttribute(k_adj_step_tc<N4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_adj_step_tc<N4><<<grid, kThreads, smem, s>>>(tmNu, tmZhi, tmZlo, p, stages);
    return cudaGetLastError();
}

}  // namespace

int adjoint_tc_stages(int n)
{
    if (n != 8 && n != 16 && n != 32) return 0;
    for (int st = 8; st >= 2; st -= 2)
        if (adj_tc_smem_n(n, st) <= (size_t)kSmemLimit) return st;
    return 0;
}

cudaError_t launch_adjoint_step_tc(const CUtensorMap &tmNu, const CUtensorMap &tmZhi, const CUtensorMap &tmZlo,
                                   const AdjTcLaunch &a, cudaStream_t s)
{
    AdjTcParams p;
    p.S = reinterpret_cast<const float4 *>(a.S);
    p.coef = a.coef;
    p.dirT = a.dirT;
    p.bcbitsT = a.bcbitsT;
    p.nu_out = a.nu_out;
    p.g_alpha = a.g_alpha;
    p.g_beta = a.g_beta;
    p.tiles = a.tiles;
    p.n_tiles = a.n_tiles;
    p.nx = a.nx;
    p.nz = a.nz;
    p.n = a.n;
    p.push = a.push;
    static int *err = nullptr;
    if (!err) {
        const cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void **>(&err), g_adj_tc_err);
        if (e != cudaSuccess) return e;
    }
    p.err = err;
    const int stages = adjoint_tc_stages(a.n);
    if (stages == 0) return cudaErrorInvalidValue;
    const int grid = std::min(a.sm_count, a.n_tiles);
    switch (4 * a.n) {
    case 32: return launch_tc<32>(tmNu, tmZhi, tmZlo, p, stages, grid, s);
    case 64: return launch_tc<64>(tmNu, tmZhi, tmZlo, p, stages, grid, s);
    case 128: return launch_tc<128>(tmNu, tmZhi, tmZlo, p, stages, grid, s);
    default: return cudaErrorInvalidValue;
    }
}

// Nonzero when the reverse-step kernel gave up waiting since the last call
// (the flag is cleared).
int adjoint_step_tc_take_error()
{
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_adj_tc_err, sizeof(int)) != cudaSuccess) return -1;
    if (v) {
        const int z = 0;
        cudaMemcpyToSymbol(g_adj_tc_err, &z, sizeof(int));
    }
    return v;
}

}  // namespace rtlb
