// Many independent lattices (spectral channels, scenes) advanced by one
// persistent tensor-core launch per step.
//
// Every channel is an ordinary context (its own grid, directions, medium,
// phase tables, boundaries and state) created with a tensor-core precision.
// The batch lists the 128-site single-class tiles of all channels as one work
// list, sorted by direction count, channel and class, and keeps a descriptor
// per channel in global memory: TMA maps of both state buffers and of the
// channel's bf16 tables, its coefficients, forward-block factors, streaming
// offsets, inflow and boundary kinds.  The kernel is the single-lattice
// tensor-core kernel with the lattice taken per work item: n (8, 16 or 32)
// and every pointer come from the item's descriptor, the table is reloaded
// when the channel or class changes, and shared memory / TMEM are sized for
// n = 32.  Tiles that mix phase classes run on the CUDA-core kernel (one
// launch per channel that has any).  rtlb_batch_step replays the launches
// from a CUDA graph (two steps per graph, one per ping-pong parity).
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "step_common.cuh"
#include "tc.h"
#include "tc_common.cuh"

namespace rtlb {
namespace {

using namespace tcptx;
using namespace tccommon;

constexpr int kMaxN4 = 128;                 // n <= 32 in a batch

// Fixed cost of a tile in the work balance, in directions' worth.  Measured
// on the 256-channel workload (n in {8, 16, 32}), TB/s of algorithmic
// traffic: 0 -> 3.67, 4 -> 4.40, 8 -> 4.11-4.20, 12 -> 4.05, 16 -> 3.90,
// 24 -> 3.60; equal tile counts per CTA gave 3.05.
// L2 prefetch of the next item's state chunks (0 = none; measured 3.01
// TB/s with it against 3.06 without on the 256-channel workload)
#ifndef RTLB_BATCH_PREFETCH_NEXT
#define RTLB_BATCH_PREFETCH_NEXT 0
#endif

#ifndef RTLB_BATCH_TILE_COST
#define RTLB_BATCH_TILE_COST 4
#endif
constexpr int kMaxC = kMaxN4 / 64;

struct ChanDesc {
    CUtensorMap tmS[2];       // state buffer 0 / 1 (2D view {4 nsites, n}, box {256, 8})
    CUtensorMap tmZhi, tmZlo; // the channel's bf16 tables, 3D {KP, 4n, n_phase}, box {64, 4n, 1}
    float *S[2];
    const float4 *coef;
    const float *fwd;         // [n_phase][n]
    const int *dir;           // [2n]
    const float *inflow;      // [4][n][4]
    int nx, nz, n, bcbits;
};

template <int MODE>
__global__ void __launch_bounds__(kThreads, 1)
    k_step_tc_batch(const ChanDesc *__restrict__ descs, const int2 *__restrict__ items, const int *__restrict__ bounds,
                    int parity,
                    int stages, int *err)
{
    constexpr bool ZLO = MODE >= 2;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const uint32_t zmax_chunk = (uint32_t)kMaxN4 * 128u;
    const uint32_t a_chunk = (uint32_t)kTileM * 128u;
    uint8_t *sZ = smem;
    uint8_t *sZlo = sZ + kMaxC * zmax_chunk;
    uint8_t *sA = sZlo + (ZLO ? kMaxC * zmax_chunk : 0);
    uint8_t *sStage = sA + kMaxC * a_chunk;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sStage + (size_t)stages * kStageBytes);
    uint64_t *st_full = bars;
    uint64_t *st_empty = st_full + stages;
    uint64_t *a_empty = st_empty + stages;     // [kMaxC]
    uint64_t *t_ready = a_empty + kMaxC;       // [2]
    uint64_t *acc_full = t_ready + 2;          // [2]
    uint64_t *acc_empty = acc_full + 2;        // [2]
    uint64_t *z_full = acc_empty + 2;          // [1]
    uint64_t *drain = z_full + 1;              // [1]
    uint64_t *z_free = drain + 1;              // [1]  the resident table's last MMAs completed
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(z_free + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // two accumulators D, then two regions E for the exact float32 part (the
    // MMAs start D from zero and the epilogue adds E, as in the single-lattice
    // kernel at 4n <= 128)
    const uint32_t tcols = 4 * kMaxN4;

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(smem_u32(&st_full[s]), 1);
            mbar_init(smem_u32(&st_empty[s]), 4);
        }
        for (int c = 0; c < kMaxC; ++c) mbar_init(smem_u32(&a_empty[c]), 1);
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
    if (warp == kMmaWarp) tmem_alloc(smem_u32(tmem_slot), tcols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    // this CTA's slice of the item list, balanced by work on the host
    const int t_begin = bounds[blockIdx.x];
    const int t_end = bounds[blockIdx.x + 1];
    const int T = t_end - t_begin;
    // item key of the table that must be resident: channel and class
    auto key_of = [](int2 it) { return (it.x << 8) | (it.y >> 24); };

    if (warp == kProdWarp) {
        if (lane == 0) {
            int prev = -1;
            uint32_t gq[2] = {0, 0}, zr = 0;
            bool ok = true;
            // the next item and its direction count are fetched a tile ahead
            int2 it_next = T > 0 ? items[t_begin] : make_int2(0, 0);
            int n_next = T > 0 ? descs[it_next.x].n : 0;
            for (int i = 0; i < T && ok; ++i) {
                const int2 it = it_next;
                const int n = n_next;
                if (i + 1 < T) {
                    it_next = items[t_begin + i + 1];
                    n_next = descs[it_next.x].n;
                }
                const ChanDesc *d = descs + it.x;
                const int tile = it.y & 0xFFFFFF, cls = it.y >> 24;
                const int N4 = 4 * n, C = (N4 + 63) / 64, groups = n / kDirsPerStage;
                const uint32_t z_chunk = (uint32_t)N4 * 128u;
                const int key = key_of(it);
                if (key != prev) {
                    // one z_free phase per table switch (cannot alias)
                    if (i > 0) ok = mbar_wait(smem_u32(z_free), (zr++) & 1, abort_flag, err, kErrTimeoutProducer);
                    if (!ok) break;
                    const uint32_t zb = smem_u32(z_full);
                    mbar_expect_tx(zb, (ZLO ? 2u : 1u) * C * z_chunk);
                    for (int c = 0; c < C; ++c) {
                        tma_load_3d(smem_u32(sZ + c * z_chunk), &d->tmZhi, zb, 64 * c, 0, cls);
                        if (ZLO) tma_load_3d(smem_u32(sZlo + c * z_chunk), &d->tmZlo, zb, 64 * c, 0, cls);
                    }
                    prev = key;
                }
                if (RTLB_BATCH_PREFETCH_NEXT && i + 1 < T) {
                    // the next item's state chunks on their way into L2
                    const CUtensorMap *tn = &descs[it_next.x].tmS[parity];
                    const int tn_tile = it_next.y & 0xFFFFFF;
                    for (int j = 0; j < n_next / kDirsPerStage; ++j)
                        for (int h = 0; h < kTileM / kHalfSites; ++h)
                            tma_prefetch_2d(tn, 4 * (tn_tile * kTileM + h * kHalfSites), j * kDirsPerStage);
                }
                for (int j = 0; j < groups && ok; ++j) {
                    const int gr = j & 1;
                    const uint32_t local = gq[gr]++;
                    const int s = ring_slot(gr, local, stages / 2);
                    ok = mbar_wait(smem_u32(&st_empty[s]), ((local / (uint32_t)(stages / 2)) & 1) ^ 1, abort_flag, err,
                                   kErrTimeoutProducer);
                    if (!ok) break;
                    const uint32_t fb = smem_u32(&st_full[s]);
                    mbar_expect_tx(fb, kStageBytes);
                    for (int h = 0; h < kTileM / kHalfSites; ++h)
                        tma_load_2d(smem_u32(sStage + (size_t)s * kStageBytes + h * (kStageBytes / 2)), &d->tmS[parity], fb,
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
        if (lane == 0) {
            int prev = -1;
            uint32_t zl = 0;
            bool ok = true, issued = false;
            int2 it_next = T > 0 ? items[t_begin] : make_int2(0, 0);
            int n_next = T > 0 ? descs[it_next.x].n : 0;
            for (int i = 0; i < T && ok; ++i) {
                const int2 it = it_next;
                const int N4 = 4 * n_next, C = (N4 + 63) / 64;
                if (i + 1 < T) {
                    it_next = items[t_begin + i + 1];
                    n_next = descs[it_next.x].n;
                }
                const int b = i & 1;
                const int key = key_of(it);
                if (key != prev) {
                    ok = mbar_wait(smem_u32(z_full), zl & 1, abort_flag, err, kErrTimeoutMma);
                    ++zl;
                    prev = key;
                    if (!ok) break;
                }
                ok = mbar_wait(smem_u32(&t_ready[b]), (i >> 1) & 1, abort_flag, err, kErrTimeoutMma);
                if (!ok) break;
                tc_fence_after();
                const uint32_t idesc = idesc_bf16(kTileM, N4);
                const uint32_t z_chunk = (uint32_t)N4 * 128u;
                const uint32_t d_tmem = tmem + (uint32_t)(b * kMaxN4);
                for (int c = 0; c < kMaxC; ++c) {
                    if (c < C) {
                        const int ksteps = min(4, (N4 - 64 * c) / 16);
                        for (int kk = 0; kk < ksteps; ++kk) {
                            const uint32_t ao = c * a_chunk + kk * 32, zo = c * z_chunk + kk * 32;
                            const uint32_t acc_in = (c == 0 && kk == 0) ? 0u : 1u;   // the item starts D from zero
                            mma_bf16(d_tmem, sw128_desc(smem_u32(sA + ao)), sw128_desc(smem_u32(sZ + zo)), idesc, acc_in);
                            if (ZLO) mma_bf16(d_tmem, sw128_desc(smem_u32(sA + ao)), sw128_desc(smem_u32(sZlo + zo)), idesc, 1u);
                        }
                    }
                    mma_commit(smem_u32(&a_empty[c]));     // one completion per item on every chunk barrier
                }
                mma_commit(smem_u32(&acc_full[b]));
                if (i + 1 < T && key_of(it_next) != key) mma_commit(smem_u32(z_free));
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
        const int q = warp & 3;
        const int grp = (warp - kConvWarp0) >> 2;
        const int r = q * 32 + lane;
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        uint32_t gq = 0;
        bool ok = true;
        // the next item's coefficients are fetched a tile ahead (see load_coef)
        auto coef_of = [&](int k) {
            const int2 it = items[t_begin + k];
            const ChanDesc *d = descs + it.x;
            return load_coef(d->coef, (it.y & 0xFFFFFF) * kTileM + r, d->nx * d->nz);
        };
        float4 cf_next = T > 0 ? coef_of(0) : float4{};
        int2 it_next = T > 0 ? items[t_begin] : make_int2(0, 0);
        int n_next = T > 0 ? descs[it_next.x].n : 0;
        const float *fwd_next = T > 0 ? descs[it_next.x].fwd : nullptr;
        for (int i = 0; i < T && ok; ++i) {
            const int2 it = it_next;
            const int cls = it.y >> 24;
            const int n = n_next;
            const float *fwd = fwd_next;
            const int b = i & 1;
            const float4 cf = cf_next;
            if (i + 1 < T) {
                cf_next = coef_of(i + 1);
                it_next = items[t_begin + i + 1];
                n_next = descs[it_next.x].n;
                fwd_next = descs[it_next.x].fwd;
            }
            ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&acc_empty[b]), ((i >> 1) & 1) ^ 1, abort_flag, err,
                                                   kErrTimeoutConverter));
            if (!ok) break;
            tc_fence_after();
            const uint32_t acc = tmem + lane_base + (uint32_t)(2 * kMaxN4 + b * kMaxN4);   // E of buffer b
            ok = convert_tile<false>(cf, fwd + (size_t)cls * n, r, lane, grp, n, n / kDirsPerStage, stages, gq, i, acc, sA,
                                     sA, sStage, st_full, st_empty, a_empty, a_chunk, abort_flag, err);
            if (!ok) break;
            tmem_wait_st();
            fence_proxy_async();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&t_ready[b]));
        }
    } else {
        const int q = warp & 3;
        const int dhalf = warp >> 2;
        const int r = q * 32 + lane;
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        bool ok = true;
        // the next item's channel fields are fetched a tile ahead
        struct Fields {
            int tile, n, nx, nz, bcbits;
            float *S_new;
            const int *dir;
            const float *inflow;
        };
        auto fields_of = [&](int k) {
            const int2 it = items[t_begin + k];
            const ChanDesc *d = descs + it.x;
            return Fields{it.y & 0xFFFFFF, d->n, d->nx, d->nz, d->bcbits, d->S[parity ^ 1], d->dir, d->inflow};
        };
        Fields f_next = T > 0 ? fields_of(0) : Fields{};
        for (int i = 0; i < T && ok; ++i) {
            const Fields f = f_next;
            if (i + 1 < T) f_next = fields_of(i + 1);
            const int tile = f.tile;
            const int n = f.n, nx = f.nx, nz = f.nz, nsites = nx * nz;
            const int b = i & 1;
            const int site = tile * kTileM + r;
            const int z = site / nx, x = site - z * nx;
            // warp-uniform: a warp with any boundary site pushes all its sites through
            // the general routine (one path instead of two divergent ones).  The
            // channels' lattices are small (a 64-wide row puts a boundary site in
            // every warp): 64 x 64 lattices at n = 32 went from 0.685 to 0.752
            // of HBM.  The single-lattice kernels keep the per-site branch, which
            // measured 1 % faster at 2048 x 2048.
            const bool interior = __all_sync(0xffffffffu, site < nsites && x > 0 && x < nx - 1 && z > 0 && z < nz - 1);
            float *S_new = f.S_new;
            const int *dir = f.dir;
            ok = __all_sync(0xffffffffu,
                            mbar_wait(smem_u32(&acc_full[b]), (i >> 1) & 1, abort_flag, err, kErrTimeoutEpilogue));
            if (!ok) break;
            tc_fence_after();
            const uint32_t acc = tmem + lane_base + (uint32_t)(b * kMaxN4);
            const int dn = n / 2, dbeg = dhalf * dn;
            float4 *out = reinterpret_cast<float4 *>(S_new);
            for (int d0 = dbeg; d0 < dbeg + dn; d0 += 4) {
                float v[16], e[16];
                tmem_ld16(acc + 4 * d0, v);
                tmem_ld16(acc + (uint32_t)(2 * kMaxN4) + 4 * d0, e);
#pragma unroll
                for (int k = 0; k < 16; ++k) v[k] += e[k];
                if (interior) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int dd = d0 + k;
                        const long long t = (long long)dd * nsites + site + __ldg(&dir[dd]) + (long long)__ldg(&dir[n + dd]) * nx;
                        __stcs(&out[t], make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]));
                    }
                } else if (site < nsites) {
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        push_store_xz(dir, f.inflow, f.bcbits, S_new, nx, nz, n, site, x, z, d0 + k,
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

size_t batch_smem(int mode, int stages)
{
    return (size_t)kMaxC * kMaxN4 * 128 * (mode >= 2 ? 2 : 1) + (size_t)kMaxC * kTileM * 128 +
           (size_t)stages * kStageBytes + (size_t)(2 * stages + kMaxC + 9) * 8 + 16 + 1024;
}

}  // namespace
}  // namespace rtlb

using namespace rtlb;

struct rtlb_batch {
    std::vector<rtlb_ctx *> ch;
    int mode = 1;
    int stages = 4;
    ChanDesc *d_desc = nullptr;
    int2 *d_items = nullptr;
    int n_items = 0;
    int *d_bounds = nullptr;           // [grid + 1] item range of each CTA
    int grid = 0;
    std::vector<int> item_n;           // direction count of each work item (for the balance)
    int tile_cost = RTLB_BATCH_TILE_COST;
    std::vector<int> mixed_channels;   // channels with tiles that mix classes
    int *d_err = nullptr, *h_err = nullptr;
    int sm_count = 148;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_parity = -1, graph_stages = -1;
    std::string err;
};

namespace {

rtlb_status batch_fail(rtlb_batch *b, rtlb_status st, const std::string &msg)
{
    if (b) b->err = msg;
    return st;
}

// One contiguous item range per CTA, of equal work: a tile moves 32 n bytes
// per site and carries a fixed cost besides (`cost` directions' worth), so
// equal tile counts would leave the CTAs holding n = 32 tiles with about twice
// the work of those holding n = 8.
std::vector<int> balance_bounds(const std::vector<int> &item_n, int grid, int cost)
{
    const int n_items = (int)item_n.size();
    std::vector<int> bounds(grid + 1, n_items);
    std::vector<double> pre(item_n.size() + 1, 0.0);
    for (size_t i = 0; i < item_n.size(); ++i) pre[i + 1] = pre[i] + item_n[i] + cost;
    size_t i = 0;
    for (int g = 0; g < grid; ++g) {
        const double target = pre.back() * g / grid;
        while (i < item_n.size() && pre[i] < target) ++i;
        bounds[g] = (int)i;
    }
    bounds[grid] = n_items;
    return bounds;
}

void drop_graph(rtlb_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->graph_parity = -1;
}

// One batch step on `s`: the persistent tensor-core launch over every
// single-class tile, then the CUDA-core kernel on the channels' mixed tiles.
cudaError_t batch_launch(rtlb_batch *b, int parity, cudaStream_t s)
{
    const int grid = b->grid;
    const size_t smem = batch_smem(b->mode, b->stages);
    cudaError_t e = cudaSuccess;
    if (grid > 0) {
        if (b->mode == 2) {
            e = cudaFuncSetAttribute(k_step_tc_batch<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess)
                k_step_tc_batch<2><<<grid, kThreads, smem, s>>>(b->d_desc, b->d_items, b->d_bounds, parity, b->stages, b->d_err);
        } else {
            e = cudaFuncSetAttribute(k_step_tc_batch<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess)
                k_step_tc_batch<1><<<grid, kThreads, smem, s>>>(b->d_desc, b->d_items, b->d_bounds, parity, b->stages, b->d_err);
        }
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    for (int k : b->mixed_channels) {
        if (e != cudaSuccess) break;
        rtlb_ctx *c = b->ch[k];
        StepParams p;
        p.S = c->S[parity];
        p.S_new = c->S[parity ^ 1];
        p.coef = c->d_coef;
        p.cls = c->d_cls;
        p.ZT = c->d_ZT;
        p.dir = c->d_dir;
        p.inflow = c->d_inflow;
        p.nx = c->nx;
        p.nz = c->nz;
        p.n = c->n;
        p.n_phase = c->n_phase;
        for (int q = 0; q < 4; ++q) p.bc[q] = c->bc[q];
        tc_mixed_list(c, &p.tile_list, &p.n_tiles);
        p.tile_span = kTileM;
        e = launch_step_fp32(p, s);
    }
    return e;
}

}  // namespace

extern "C" {

rtlb_status rtlb_batch_create(int32_t count, rtlb_ctx *const *channels, rtlb_batch **out)
{
    if (!out || !channels || count < 1) return RTLB_E_ARG;
    *out = nullptr;
    rtlb_batch *b = new rtlb_batch();
    b->ch.assign(channels, channels + count);
    const int prec = channels[0] ? channels[0]->opt.precision : -1;
    if (prec != RTLB_PREC_BF16 && prec != RTLB_PREC_BF16X2) {
        delete b;
        return RTLB_E_UNSUPPORTED;
    }
    b->mode = prec == RTLB_PREC_BF16X2 ? 2 : 1;
    std::vector<ChanDesc> desc(count);
    std::vector<int2> items;
    for (int k = 0; k < count; ++k) {
        rtlb_ctx *c = channels[k];
        if (!c || c->opt.precision != prec || !c->medium_set || c->n > 32 || c->n % 8 != 0 || c->cur != channels[0]->cur ||
            c->dev != channels[0]->dev || c->opt.streaming != RTLB_STREAM_NEAREST8) {
            delete b;
            return c && !c->medium_set ? RTLB_E_STATE : RTLB_E_UNSUPPORTED;
        }
        std::memset(&desc[k], 0, sizeof(ChanDesc));
        if (!tc_encode_state_map(&desc[k].tmS[0], c->S[0], c->nsites(), c->n) ||
            !tc_encode_state_map(&desc[k].tmS[1], c->S[1], c->nsites(), c->n) ||
            !tc_table_maps(c, &desc[k].tmZhi, &desc[k].tmZlo, &desc[k].fwd)) {
            delete b;
            return RTLB_E_CUDA;
        }
        desc[k].S[0] = c->S[0];
        desc[k].S[1] = c->S[1];
        desc[k].coef = c->d_coef;
        desc[k].dir = c->d_dir;
        desc[k].inflow = c->d_inflow;
        desc[k].nx = c->nx;
        desc[k].nz = c->nz;
        desc[k].n = c->n;
        desc[k].bcbits = pack_bc(c->bc);
        std::vector<int> pure;
        if (!tc_pure_tiles(c, pure)) {
            delete b;
            return RTLB_E_CUDA;
        }
        for (int e : pure) items.push_back(make_int2(k, e));
        if (tc_mixed_tiles(c) > 0) b->mixed_channels.push_back(k);
    }
    // group by direction count, then channel, then class (the table reloads)
    std::stable_sort(items.begin(), items.end(), [&](const int2 &a, const int2 &c) {
        const int na = channels[a.x]->n, nc = channels[c.x]->n;
        if (na != nc) return na < nc;
        if (a.x != c.x) return a.x < c.x;
        return (a.y >> 24) < (c.y >> 24);
    });
    cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, channels[0]->dev);
    b->n_items = (int)items.size();
    b->grid = std::min(b->sm_count, b->n_items);
    b->item_n.resize(items.size());
    for (size_t i = 0; i < items.size(); ++i) b->item_n[i] = channels[items[i].x]->n;
    const std::vector<int> bounds = balance_bounds(b->item_n, b->grid, b->tile_cost);
    cudaError_t e = cudaMalloc(&b->d_desc, desc.size() * sizeof(ChanDesc));
    if (e == cudaSuccess && !items.empty()) e = cudaMalloc(&b->d_items, items.size() * sizeof(int2));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_bounds, bounds.size() * sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(b->d_bounds, bounds.data(), bounds.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(b->d_desc, desc.data(), desc.size() * sizeof(ChanDesc), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !items.empty())
        e = cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, sizeof(int));
    if (e != cudaSuccess) {
        rtlb_batch_destroy(b);
        return e == cudaErrorMemoryAllocation ? RTLB_E_OOM : RTLB_E_CUDA;
    }
    b->stages = 4;
    *out = b;
    return RTLB_OK;
}

rtlb_status rtlb_batch_configure(rtlb_batch *b, int32_t stages)
{
    if (!b) return RTLB_E_ARG;
    if (stages < 2 || stages > 8 || stages % 2 != 0 || batch_smem(b->mode, stages) > 232448)
        return batch_fail(b, RTLB_E_RANGE, "stages must be 2, 4, 6 or 8 and fit in shared memory");
    if (stages != b->stages) drop_graph(b);
    b->stages = stages;
    return RTLB_OK;
}

rtlb_status rtlb_batch_balance(rtlb_batch *b, int32_t tile_cost)
{
    if (!b) return RTLB_E_ARG;
    if (tile_cost < 0 || tile_cost > 64) return batch_fail(b, RTLB_E_RANGE, "tile_cost must be in [0, 64]");
    if (b->grid == 0) {
        b->tile_cost = tile_cost;
        return RTLB_OK;
    }
    const std::vector<int> bounds = balance_bounds(b->item_n, b->grid, tile_cost);
    // the ranges are read by launches in flight: wait for them first
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_bounds, bounds.data(), bounds.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return batch_fail(b, RTLB_E_CUDA, std::string("balance: ") + cudaGetErrorString(e));
    b->tile_cost = tile_cost;
    return RTLB_OK;
}

rtlb_status rtlb_batch_step(rtlb_batch *b, int32_t nsteps, void *stream)
{
    if (!b) return RTLB_E_ARG;
    if (nsteps < 0) return batch_fail(b, RTLB_E_ARG, "nsteps must be >= 0");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int cur = b->ch[0]->cur;
    for (rtlb_ctx *c : b->ch)
        if (c->cur != cur) return batch_fail(b, RTLB_E_STATE, "channels were stepped outside the batch");
    int done = 0;
    // two steps per graph replay (parity cur, then cur ^ 1)
    if (nsteps >= 2) {
        if (!b->exec || b->graph_parity != cur || b->graph_stages != b->stages) {
            drop_graph(b);
            cudaStream_t cap;
            if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess)
                return batch_fail(b, RTLB_E_CUDA, "capture stream");
            cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) e = batch_launch(b, cur, cap);
            if (e == cudaSuccess) e = batch_launch(b, cur ^ 1, cap);
            cudaGraph_t g = nullptr;
            const cudaError_t e2 = cudaStreamEndCapture(cap, &g);
            if (e == cudaSuccess) e = e2;
            if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
            cudaStreamDestroy(cap);
            if (e != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return batch_fail(b, RTLB_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
            }
            b->graph = g;
            b->graph_parity = cur;
            b->graph_stages = b->stages;
        }
        for (; done + 2 <= nsteps; done += 2) {
            const cudaError_t e = cudaGraphLaunch(b->exec, s);
            if (e != cudaSuccess) return batch_fail(b, RTLB_E_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
        }
    }
    int parity = cur;
    if (done < nsteps) {
        const cudaError_t e = batch_launch(b, parity, s);
        if (e != cudaSuccess) return batch_fail(b, RTLB_E_CUDA, std::string("batch launch: ") + cudaGetErrorString(e));
        parity ^= 1;
        done += 1;
    }
    for (rtlb_ctx *c : b->ch) {
        c->cur = parity;
        c->steps += nsteps;
        if (nsteps > 0) c->has_prev = true;
    }
    return RTLB_OK;
}

rtlb_status rtlb_batch_check(rtlb_batch *b, void *stream)
{
    if (!b) return RTLB_E_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(b->h_err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return batch_fail(b, RTLB_E_CUDA, "reading the batch error flag failed");
    if (*b->h_err) {
        cudaMemsetAsync(b->d_err, 0, sizeof(int), s);
        return batch_fail(b, RTLB_E_TIMEOUT, "a batch kernel gave up waiting");
    }
    return RTLB_OK;
}

const char *rtlb_batch_last_error(const rtlb_batch *b) { return b ? b->err.c_str() : "null batch"; }

void rtlb_batch_destroy(rtlb_batch *b)
{
    if (!b) return;
    cudaDeviceSynchronize();
    drop_graph(b);
    cudaFree(b->d_desc);
    cudaFree(b->d_items);
    cudaFree(b->d_bounds);
    cudaFree(b->d_err);
    cudaFreeHost(b->h_err);
    delete b;
}

}  // extern "C"
