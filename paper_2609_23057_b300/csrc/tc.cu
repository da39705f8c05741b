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
//   warps 8-11  converter  (FP32 staging -> bf16 A operand in the 128-byte
//                           swizzled K-major layout, alpha * S~ -> TMEM)
//   warp  12    producer   (TMA loads of state chunks and of Z, L2 prefetch
//                           two tiles ahead)
//   warp  13    MMA issuer (one thread; also allocates TMEM)
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
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "step_common.cuh"
#include "tc.h"

namespace rtlb {

namespace {

constexpr int kTileM = 128;
constexpr int kWarps = 14;
constexpr int kEpiWarps = 8;
constexpr int kConvWarp0 = 8;
constexpr int kProdWarp = 12;
constexpr int kMmaWarp = 13;
constexpr int kThreads = kWarps * 32;
constexpr int kDirsPerStage = 8;                    // directions per state chunk
constexpr int kStageBytes = kDirsPerStage * kTileM * 16;
constexpr int kHalfSites = 64;                      // sites per TMA box row (256 floats)
constexpr int kSmemLimit = 232448;                  // max dynamic smem per block
constexpr unsigned long long kTimeoutNs = 2000000000ull;

// Memory-system policy of the streamed state (each byte is read once and
// written once per step): how many tiles ahead the producer prefetches into
// L2, whether the epilogue's stores are marked evict-first, and whether the
// TMA loads of the state are marked evict-first.
#ifndef RTLB_TC_PREFETCH_TILES
#define RTLB_TC_PREFETCH_TILES 0
#endif
#ifndef RTLB_TC_STREAM_STORES
#define RTLB_TC_STREAM_STORES 1
#endif
#ifndef RTLB_TC_LOAD_EVICT_FIRST
#define RTLB_TC_LOAD_EVICT_FIRST 1
#endif

enum ErrCode { kErrTimeoutProducer = 1, kErrTimeoutConverter = 2, kErrTimeoutMma = 4, kErrTimeoutEpilogue = 8 };

struct TcState {
    int N4 = 0, KP = 0, C = 0, n_phase = 0;
    bool split = false;
    __nv_bfloat16 *d_Zhi = nullptr;  // [n_phase][N4][KP]
    __nv_bfloat16 *d_Zlo = nullptr;
    int *d_pure = nullptr;           // tile | class << 24, sorted by class
    int n_pure = 0;
    int *d_mixed = nullptr;          // tile indices
    int n_mixed = 0;
    float *d_fwd = nullptr;          // [n_phase][n] forward-block factors applied in float32
    int *d_err = nullptr;
    int *h_err = nullptr;
    CUtensorMap tmZhi{}, tmZlo{}, tmS[2]{};
    bool tmS_ready[2] = {false, false};
    const float *tmS_ptr[2] = {nullptr, nullptr};
    int sm_count = 0;
    int stages = 0;
    size_t smem = 0;
};

// ------------------------------------------------------------ PTX wrappers

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait on one mbarrier phase.  Returns false (after raising the CTA's
// abort flag and recording `code`) when the wait times out or another role
// has already aborted.
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag, int *err, int code)
{
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned it = 1;; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 63u) == 0u) {
            if (*abort_flag) return false;
            if (global_ns() - t0 > kTimeoutNs) {
                *abort_flag = 1;
                atomicOr(err, code);
                return false;
            }
        }
    }
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int c0, int c1, int c2)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int c0, int c1)
{
#if RTLB_TC_LOAD_EVICT_FIRST
    uint64_t policy;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(policy));
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1, {%3, %4}], [%2], %5;" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1), "l"(policy)
        : "memory");
#else
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1)
        : "memory");
#endif
}

__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap *map, int c0, int c1)
{
    asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global [%0, {%1, %2}];" ::"l"(reinterpret_cast<uint64_t>(map)),
                 "r"(c0), "r"(c1)
                 : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D[tmem] (+)= A[smem] . B[smem]^T, bf16 inputs, f32 accumulate, M = 128.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float v[8])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
                 "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                 "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                 "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO), descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;                 // LBO (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;       // SBO
    d |= (uint64_t)1 << 46;                 // version
    d |= (uint64_t)2 << 61;                 // SWIZZLE_128B
    return d;
}

// Instruction descriptor: D f32, A/B bf16, both K-major, M = 128, N = n4.
__host__ __device__ constexpr uint32_t idesc_bf16(int n4)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n4 >> 3) << 17) | ((uint32_t)(kTileM >> 4) << 24);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
}

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
};

template <bool SPLIT>
__global__ void __launch_bounds__(kThreads, 1)
    k_step_tc(const __grid_constant__ CUtensorMap tmS, const __grid_constant__ CUtensorMap tmZhi,
              const __grid_constant__ CUtensorMap tmZlo, TcParams p, int N4, int stages)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const int C = (N4 + 63) / 64;                  // K chunks of 64
    const int n = p.n;
    const int nsites = p.nx * p.nz;
    const int groups = n / kDirsPerStage;          // state chunks per tile (n % 8 == 0)
    const uint32_t z_chunk = (uint32_t)N4 * 128u;  // bytes per K chunk of Z
    const uint32_t a_chunk = (uint32_t)kTileM * 128u;

    uint8_t *sZ = smem;
    uint8_t *sZlo = sZ + C * z_chunk;
    uint8_t *sA = sZlo + (SPLIT ? C * z_chunk : 0);
    uint8_t *sAlo = sA + C * a_chunk;
    uint8_t *sStage = sAlo + (SPLIT ? C * a_chunk : 0);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sStage + (size_t)stages * kStageBytes);
    uint64_t *st_full = bars;
    uint64_t *st_empty = st_full + stages;
    uint64_t *a_empty = st_empty + stages;     // [C]
    uint64_t *t_ready = a_empty + C;           // [2]
    uint64_t *acc_full = t_ready + 2;          // [2]
    uint64_t *acc_empty = acc_full + 2;        // [2]
    uint64_t *z_full = acc_empty + 2;          // [1]
    uint64_t *drain = z_full + 1;              // [1]
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    int8_t *s_cx = reinterpret_cast<int8_t *>(tmem_slot + 2);   // [n]
    int8_t *s_cz = s_cx + kMaxDirs;                              // [n]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t tcols = N4 * 2 <= 32 ? 32u : (N4 * 2 <= 64 ? 64u : (N4 * 2 <= 128 ? 128u : (N4 * 2 <= 256 ? 256u : 512u)));

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(smem_u32(&st_full[s]), 1);
            mbar_init(smem_u32(&st_empty[s]), 4);
        }
        for (int c = 0; c < C; ++c) mbar_init(smem_u32(&a_empty[c]), 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&t_ready[b]), 4);
            mbar_init(smem_u32(&acc_full[b]), 1);
            mbar_init(smem_u32(&acc_empty[b]), kEpiWarps);
        }
        mbar_init(smem_u32(z_full), 1);
        mbar_init(smem_u32(drain), 1);
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
            int prev_cls = -1;
            uint32_t g = 0;
            bool ok = true;
            for (int i = 0; i < T && ok; ++i) {
                const int e = p.tiles[t_begin + i];
                const int tile = e & 0xFFFFFF, cls = e >> 24;
                if (cls != prev_cls) {
                    if (i > 0)
                        ok = mbar_wait(smem_u32(&acc_full[(i - 1) & 1]), ((i - 1) >> 1) & 1, abort_flag, p.err, kErrTimeoutProducer);
                    if (!ok) break;
                    const uint32_t zb = smem_u32(z_full);
                    mbar_expect_tx(zb, (SPLIT ? 2u : 1u) * C * z_chunk);
                    for (int c = 0; c < C; ++c) {
                        tma_load_3d(smem_u32(sZ + c * z_chunk), &tmZhi, zb, 64 * c, 0, cls);
                        if (SPLIT) tma_load_3d(smem_u32(sZlo + c * z_chunk), &tmZlo, zb, 64 * c, 0, cls);
                    }
                    prev_cls = cls;
                }
                // keep the next tiles' state on its way into L2
                for (int ahead = (i == 0 ? 1 : RTLB_TC_PREFETCH_TILES); ahead <= RTLB_TC_PREFETCH_TILES; ++ahead) {
                    if (i + ahead >= T) break;
                    const int nt = p.tiles[t_begin + i + ahead] & 0xFFFFFF;
                    for (int j = 0; j < groups; ++j)
                        for (int h = 0; h < kTileM / kHalfSites; ++h)
                            tma_prefetch_2d(&tmS, 4 * (nt * kTileM + h * kHalfSites), j * kDirsPerStage);
                }
                for (int j = 0; j < groups && ok; ++j, ++g) {
                    const int s = g % stages;
                    ok = mbar_wait(smem_u32(&st_empty[s]), ((g / stages) & 1) ^ 1, abort_flag, p.err, kErrTimeoutProducer);
                    if (!ok) break;
                    const uint32_t fb = smem_u32(&st_full[s]);
                    mbar_expect_tx(fb, kStageBytes);
                    for (int h = 0; h < kTileM / kHalfSites; ++h)
                        tma_load_2d(smem_u32(sStage + (size_t)s * kStageBytes + h * (kStageBytes / 2)), &tmS, fb,
                                    4 * (tile * kTileM + h * kHalfSites), j * kDirsPerStage);
                }
            }
            // drain: wait (bounded) for the loads this thread issued into each stage
            for (uint32_t k = 0; k < (uint32_t)stages && k < g; ++k) {
                const uint32_t gg = g - 1 - k;
                const int s = gg % stages;
                unsigned long long t0 = global_ns();
                while (!mbar_try(smem_u32(&st_full[s]), (gg / stages) & 1) && global_ns() - t0 < kTimeoutNs) {
                }
            }
        }
    } else if (warp == kMmaWarp) {
        // ---------------------------------------------------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(N4);
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
                        mma_bf16(d_tmem, sw128_desc(smem_u32(sA + ao)), sw128_desc(smem_u32(sZ + zo)), idesc, 1u);
                        if (SPLIT) {
                            mma_bf16(d_tmem, sw128_desc(smem_u32(sAlo + ao)), sw128_desc(smem_u32(sZ + zo)), idesc, 1u);
                            mma_bf16(d_tmem, sw128_desc(smem_u32(sA + ao)), sw128_desc(smem_u32(sZlo + zo)), idesc, 1u);
                        }
                    }
                    mma_commit(smem_u32(&a_empty[c]));
                }
                mma_commit(smem_u32(&acc_full[b]));
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
        const int r = q * 32 + lane;               // site row = TMEM lane
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        const int half = r / kHalfSites, hr = r % kHalfSites;
        uint32_t g = 0;
        bool ok = true;
        for (int i = 0; i < T && ok; ++i) {
            const int entry = p.tiles[t_begin + i];
            const int tile = entry & 0xFFFFFF;
            const float *fwd = p.fwd + (size_t)(entry >> 24) * n;
            const int b = i & 1;
            const int site = tile * kTileM + r;
            float4 cf = make_float4(0.f, 0.f, 0.f, 0.f);
            if (site < nsites) cf = p.coef[site];
            ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&acc_empty[b]), ((i >> 1) & 1) ^ 1, abort_flag, p.err,
                                                   kErrTimeoutConverter));
            if (!ok) break;
            tc_fence_after();
            const uint32_t acc = tmem + lane_base + (uint32_t)(b * N4);
            for (int j = 0; j < groups && ok; ++j, ++g) {
                const int s = g % stages;
                ok = __all_sync(0xffffffffu,
                                mbar_wait(smem_u32(&st_full[s]), (g / stages) & 1, abort_flag, p.err, kErrTimeoutConverter));
                if (!ok) break;
                // stage layout: [half][direction][64 sites][4]
                const float4 *stg = reinterpret_cast<const float4 *>(sStage + (size_t)s * kStageBytes) +
                                    half * (kDirsPerStage * kHalfSites) + hr;
#pragma unroll
                for (int dl = 0; dl < kDirsPerStage; dl += 2) {
                    const int d = j * kDirsPerStage + dl;
                    const int c = d >> 4;                       // K chunk of this direction pair
                    if ((d & 15) == 0) {
                        ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&a_empty[c]), (i & 1) ^ 1, abort_flag, p.err,
                                                               kErrTimeoutConverter));
                        if (!ok) break;
                    }
                    float4 v0 = stg[dl * kHalfSites], v1 = stg[(dl + 1) * kHalfSites];
                    v0.x += cf.w;                               // emission (I only)
                    v1.x += cf.w;
                    const float sv[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
                    // alpha (hi + lo) * S~ plus the forward block beta * c_d * S~
                    const float g0 = fmaf(cf.z, __ldg(&fwd[d]), cf.y), g1 = fmaf(cf.z, __ldg(&fwd[d + 1]), cf.y);
                    float init[8], bs[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        init[k] = fmaf(cf.x, sv[k], (k < 4 ? g0 : g1) * sv[k]);
                        bs[k] = cf.z * sv[k];                       // beta * S~ (MMA operand)
                    }
                    tmem_st8(acc + 4 * d, init);
                    uint4 hi;
                    hi.x = pack_bf16(bs[0], bs[1]);
                    hi.y = pack_bf16(bs[2], bs[3]);
                    hi.z = pack_bf16(bs[4], bs[5]);
                    hi.w = pack_bf16(bs[6], bs[7]);
                    const uint32_t gran = (uint32_t)((d & 15) >> 1);          // 16-byte granule in the row
                    const uint32_t off = c * a_chunk + r * 128u + ((gran ^ (uint32_t)(r & 7)) << 4);
                    *reinterpret_cast<uint4 *>(sA + off) = hi;
                    if (SPLIT) {
                        const __nv_bfloat162 *h2 = reinterpret_cast<const __nv_bfloat162 *>(&hi);
                        uint4 lo;
                        uint32_t *lw = reinterpret_cast<uint32_t *>(&lo);
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const float2 f = __bfloat1622float2(h2[k]);
                            lw[k] = pack_bf16(bs[2 * k] - f.x, bs[2 * k + 1] - f.y);
                        }
                        *reinterpret_cast<uint4 *>(sAlo + off) = lo;
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&st_empty[s]));
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
                        push_store(p.dir, p.inflow, p.bcbits, p.S_new, p.nx, p.nz, n, site, d0 + k,
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

bool encode_z_map(CUtensorMap *m, const __nv_bfloat16 *Z, int N4, int KP, int n_phase)
{
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)KP, (cuuint64_t)N4, (cuuint64_t)n_phase};
    cuuint64_t strides[2] = {(cuuint64_t)KP * 2, (cuuint64_t)N4 * KP * 2};
    cuuint32_t box[3] = {64, (cuuint32_t)N4, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16 *>(Z), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

TcState *state_of(rtlb_ctx *c) { return static_cast<TcState *>(c->tc); }

void free_tables(TcState *t)
{
    cudaFree(t->d_Zhi);
    cudaFree(t->d_Zlo);
    cudaFree(t->d_fwd);
    cudaFree(t->d_pure);
    cudaFree(t->d_mixed);
    t->d_fwd = nullptr;
    t->d_Zhi = t->d_Zlo = nullptr;
    t->d_pure = t->d_mixed = nullptr;
    t->n_pure = t->n_mixed = 0;
}

size_t smem_bytes(int N4, bool split, int stages)
{
    const int C = (N4 + 63) / 64;
    size_t b = (size_t)C * N4 * 128 * (split ? 2 : 1) + (size_t)C * kTileM * 128 * (split ? 2 : 1) +
               (size_t)stages * kStageBytes + (size_t)(2 * stages + C + 8) * 8 + 16 + 2 * kMaxDirs;
    return b + 1024;  // alignment slack
}

}  // namespace

bool tc_supported(int n) { return n == 8 || n == 16 || n == 32 || n == 64; }

bool tc_shape_ok(int n, bool split)
{
    if (!tc_supported(n)) return false;
    for (int st = 8; st >= 2; --st)
        if (smem_bytes(4 * n, split, st) <= (size_t)kSmemLimit) return true;
    return false;
}

rtlb_status tc_prepare(rtlb_ctx *c, const double *tables, int n_phase, const uint8_t *dev_cls, cudaStream_t s)
{
    if (c->opt.precision == RTLB_PREC_FP32) return RTLB_OK;
    const bool split = c->opt.precision == RTLB_PREC_BF16X3;
    if (!tc_supported(c->n)) {
        c->err = "tensor-core forms need n in {8, 16, 32, 64}";
        return RTLB_E_UNSUPPORTED;
    }
    const int N4 = 4 * c->n, KP = ((N4 + 63) / 64) * 64, C = KP / 64;
    int stages = 0;
    for (int st = 8; st >= 2; --st)
        if (smem_bytes(N4, split, st) <= (size_t)kSmemLimit) {
            stages = st;
            break;
        }
    if (stages == 0) {
        c->err = "the split bf16 form does not fit in shared memory for n = 64";
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
    std::vector<__nv_bfloat16> hi((size_t)n_phase * psz, __float2bfloat16(0.0f)), lo(hi.size(), __float2bfloat16(0.0f));
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
    std::stable_sort(pure.begin(), pure.end(), [](int x, int y) { return (x >> 24) < (y >> 24); });

    free_tables(t);
    cudaError_t e = cudaMalloc(&t->d_Zhi, hi.size() * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMalloc(&t->d_fwd, fwd.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(t->d_fwd, fwd.data(), fwd.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && split) e = cudaMalloc(&t->d_Zlo, lo.size() * sizeof(__nv_bfloat16));
    if (e == cudaSuccess && !pure.empty()) e = cudaMalloc(&t->d_pure, pure.size() * sizeof(int));
    if (e == cudaSuccess && !mixed.empty()) e = cudaMalloc(&t->d_mixed, mixed.size() * sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(t->d_Zhi, hi.data(), hi.size() * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice);
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
    if (!encode_z_map(&t->tmZhi, t->d_Zhi, N4, KP, n_phase) ||
        (split && !encode_z_map(&t->tmZlo, t->d_Zlo, N4, KP, n_phase))) {
        free_tables(t);
        c->err = "tensor map encoding for the phase tables failed";
        return RTLB_E_CUDA;
    }
    if (!split) t->tmZlo = t->tmZhi;
    t->N4 = N4;
    t->KP = KP;
    t->C = C;
    t->n_phase = n_phase;
    t->split = split;
    t->n_pure = (int)pure.size();
    t->n_mixed = (int)mixed.size();
    t->stages = stages;
    t->smem = smem_bytes(N4, split, stages);
    return RTLB_OK;
}

rtlb_status tc_step(rtlb_ctx *c, const StepParams &p, cudaStream_t s)
{
    TcState *t = state_of(c);
    if (!t || !t->d_Zhi) {
        c->err = "tensor-core tables are not prepared";
        return RTLB_E_STATE;
    }
    const int which = (p.S == c->S[0]) ? 0 : 1;
    if (!t->tmS_ready[which] || t->tmS_ptr[which] != p.S) {
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
        const int grid = std::min(t->sm_count, t->n_pure);
        cudaError_t e;
        if (t->split) {
            e = cudaFuncSetAttribute(k_step_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t->smem);
            if (e == cudaSuccess)
                k_step_tc<true><<<grid, kThreads, t->smem, s>>>(t->tmS[which], t->tmZhi, t->tmZlo, tp, t->N4, t->stages);
        } else {
            e = cudaFuncSetAttribute(k_step_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t->smem);
            if (e == cudaSuccess)
                k_step_tc<false><<<grid, kThreads, t->smem, s>>>(t->tmS[which], t->tmZhi, t->tmZlo, tp, t->N4, t->stages);
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
