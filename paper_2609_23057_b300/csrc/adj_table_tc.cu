// Tensor-core form of the adjoint's phase-table gradient:
//
//   dL/dZ_c[r][k] += sum over the sites of class c of (beta mu)[site][r] S~[site][k]
//
// (the reverse-mode counterpart of the scattering contraction of Eq. 11 / 25;
// beta mu and S~ = S^t + e come from the reverse step).  One GEMM per class
// with M = N = 4n and the sites as the reduction dimension K.
//
// Persistent kernel, one CTA per SM, each reducing a contiguous slice of
// 64-site chunks.  The threads copy beta mu and S (coalesced, cp.async) into
// a staging slot two chunks ahead, so the loads of chunks ch + 1 and ch + 2
// are in flight while chunk ch is converted.  Conversion splits each value into bf16 hi + lo and writes
// four K-major, 128-byte-swizzled operand tiles (rows = table index r or k,
// K = the chunk's 64 sites); one thread then issues three tcgen05 MMAs per
// 16-site step (hi.hi, hi.lo, lo.hi: float32-class products) into the
// class's TMEM accumulator.  A chunk whose
// sites mix classes is reduced once per class present with the other
// classes' sites zeroed in A.  At the end each CTA adds its accumulators into
// its own float64 slot (no atomics); the slots are summed after the sweep.
//
// Needs 4n <= 128 and n_phase * 4n <= 512 TMEM columns; other shapes use the
// CUDA-core kernel.  Every wait is bounded (about 2 s): on timeout the CTA
// records an error code and skips the rest of its work.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "rtlb_internal.h"
#include "tc_ptx.cuh"

namespace rtlb {
namespace {

using namespace tcptx;

constexpr int kChunk = 64;                       // sites per K chunk: one 128-byte bf16 row
constexpr int kRows = 128;                       // operand rows (table index; zero beyond 4n)
constexpr int kTT = 256;                         // threads
constexpr uint32_t kTile = kRows * 128;          // one operand tile, 16 KB
constexpr uint32_t kBuf = 4 * kTile;             // A hi, A lo, B hi, B lo
constexpr int kErrTableTimeout = 16;

// hi + lo bf16 split of eight values: two 16-byte rows of packed pairs
__device__ __forceinline__ void split8(const float v[8], uint4 &hi, uint4 &lo)
{
    uint32_t h[4], l[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        h[k] = pack_bf16(v[2 * k], v[2 * k + 1]);
        const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&h[k]));
        l[k] = pack_bf16(v[2 * k] - f.x, v[2 * k + 1] - f.y);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// Stores the 16-byte group `sg` (sites 8 sg .. 8 sg + 7) of row r of a
// K-major SW128 tile.
__device__ __forceinline__ void put_row(uint8_t *tile, int r, int sg, uint4 v)
{
    *reinterpret_cast<uint4 *>(tile + r * 128 + (((uint32_t)sg ^ (uint32_t)(r & 7)) << 4)) = v;
}

// Per-thread asynchronous copies (cp.async) into shared memory; `bytes` = 0
// writes zeros (sites past the lattice).
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async4(uint32_t dst, const void *src, uint32_t bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async8(uint32_t dst, const void *src, uint32_t bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Staging slot of one chunk: beta mu (or mu, scaled here by beta) and S as
// [direction][site] rows of 64 float4 (1 KB per direction), then the chunk's
// emission e[64], beta[64] and classes.
// Within each 128-byte group of eight sites the 16-byte entries are permuted
// (entry i of group g sits at position i ^ g), so that both the coalesced
// copies (one group of eight sites per eight threads) and the conversion
// reads (one group per thread) spread over all banks.
constexpr uint32_t kRowBytes = kChunk * 16;
constexpr uint32_t kStageS = (kTT / 8) * kRowBytes;            // S rows follow the 32 beta mu rows
constexpr uint32_t kStageData = 2 * kStageS;
constexpr uint32_t kStageE = kStageData;                         // e[64] floats
constexpr uint32_t kStageBeta = kStageE + kChunk * 4;             // beta[64] floats
constexpr uint32_t kStageCls = kStageBeta + kChunk * 4;           // cls[64] bytes
constexpr uint32_t kStage = kStageCls + kChunk;
constexpr uint32_t kStageAligned = (kStage + 127) / 128 * 128;

__device__ __forceinline__ uint32_t stage_pos(int site) { return (uint32_t)((site & ~7) | ((site ^ (site >> 3)) & 7)) * 16u; }

// Writes rows 4d .. 4d + 3 (hi and lo tiles) from the staged row of direction
// d, sites 8 sg .. 8 sg + 7; `e` (or null) is added to I, `scale` (or null)
// multiplies every component; sites of classes other than `only` are zeroed
// when only >= 0.
__device__ __forceinline__ void put_rows(const uint8_t *row, const float *e, const float *scale, const uint8_t *cl,
                                         int only, int d, int sg, uint8_t *hi_tile, uint8_t *lo_tile)
{
    float v[4][8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        float4 x = *reinterpret_cast<const float4 *>(row + stage_pos(8 * sg + i));
        if (e) x.x += e[8 * sg + i];
        const float keep = ((only < 0 || cl[8 * sg + i] == only) ? 1.f : 0.f) * (scale ? scale[8 * sg + i] : 1.f);
        v[0][i] = x.x * keep;
        v[1][i] = x.y * keep;
        v[2][i] = x.z * keep;
        v[3][i] = x.w * keep;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        uint4 h, l;
        split8(v[c], h, l);
        put_row(hi_tile, 4 * d + c, sg, h);
        put_row(lo_tile, 4 * d + c, sg, l);
    }
}

__device__ int g_table_tc_err;

__global__ void __launch_bounds__(kTT, 1)
    k_adj_table_tc(const float4 *__restrict__ beta_mu, const float4 *__restrict__ S, const float4 *__restrict__ coef,
                   const uint8_t *__restrict__ cls, double *__restrict__ slots, int nsites, int n, int n_phase,
                   uint32_t tcols, int beta_scale)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023u)) & 1023u);
    uint8_t *Ahi = smem, *Alo = smem + kTile, *Bhi = smem + 2 * kTile, *Blo = smem + 3 * kTile;   // one operand buffer
    uint8_t *stage = smem + kBuf;                                                              // [2] staging slots
    uint64_t *done = reinterpret_cast<uint64_t *>(stage + 2 * kStageAligned);                  // MMAs completed
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int N4 = 4 * n;

    // operand tiles start at zero: rows 4n .. 127 of A are never written
    for (uint32_t o = (uint32_t)tid * 16u; o < kBuf; o += kTT * 16u)
        *reinterpret_cast<uint4 *>(smem + o) = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) {
        mbar_init(smem_u32(done), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(smem_u32(tmem_slot), tcols);
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int nchunks = (nsites + kChunk - 1) / kChunk;
    const int c_begin = (int)((long long)nchunks * blockIdx.x / gridDim.x);
    const int c_end = (int)((long long)nchunks * (blockIdx.x + 1) / gridDim.x);
    const int d = tid >> 3, sg = tid & 7;          // conversion item: direction d, sites 8 sg .. 8 sg + 7
    const bool loader = d < n;
    const uint32_t idesc = idesc_bf16(kRows, N4);

    // copies of chunk ch into staging slot `slot` (one commit group per call)
    auto issue = [&](int ch, int slot) {
        if (ch < c_end) {
            const uint32_t base = smem_u32(stage + slot * kStageAligned);
            if (loader) {   // group j of direction d: site 8 j + sg by thread (d, sg), 4 full lines per warp
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int site = ch * kChunk + 8 * j + sg;
                    const bool in = site < nsites;
                    const size_t off = in ? (size_t)d * nsites + site : 0;
                    const uint32_t dst = base + d * kRowBytes + stage_pos(8 * j + sg);
                    cp_async16(dst, beta_mu + off, in ? 16u : 0u);
                    cp_async16(dst + kStageS, S + off, in ? 16u : 0u);
                }
            }
            const int site0 = ch * kChunk + 8 * sg;
            if (d == 0) {   // emission (coef.w) and classes of sites 8 sg .. 8 sg + 7
                const float *ew = reinterpret_cast<const float *>(coef) + 3;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int site = site0 + i;
                    const bool in = site < nsites;
                    cp_async4(base + kStageE + (8 * sg + i) * 4, ew + 4 * (size_t)(in ? site : 0), in ? 4u : 0u);
                    if (beta_scale)
                        cp_async4(base + kStageBeta + (8 * sg + i) * 4, ew - 1 + 4 * (size_t)(in ? site : 0), in ? 4u : 0u);
                }
                const int left = nsites - site0;   // class bytes present in this group (rest zero-filled)
                const uint32_t nb = left <= 0 ? 0u : (left >= 8 ? 8u : (uint32_t)left);
                cp_async8(base + kStageCls + 8 * sg, cls + (nb ? site0 : 0), nb);
            }
        }
        cp_async_commit();
    };

    issue(c_begin, 0);
    issue(c_begin + 1, 1);
    uint32_t cnt = 0;                              // commits issued (same in every thread)
    unsigned seen = 0u;                            // classes with an accumulator (same in every thread)
    bool ok = true;
    auto ops_free = [&]() -> bool {                // the last pass's MMAs completed; vote = barrier
        const bool w = cnt == 0u || mbar_wait(smem_u32(done), (cnt - 1u) & 1u, abort_flag, &g_table_tc_err,
                                              kErrTableTimeout);
        return __syncthreads_and(w) != 0;
    };

    for (int ch = c_begin, it = 0; ch < c_end && ok; ++ch, ++it) {
        const int slot = it & 1;
        uint8_t *st = stage + slot * kStageAligned;
        const uint8_t *mine = st + d * kRowBytes;
        const float *e = reinterpret_cast<const float *>(st + kStageE);
        const float *bt = beta_scale ? reinterpret_cast<const float *>(st + kStageBeta) : nullptr;
        const uint8_t *cl = st + kStageCls;
        const int site0 = ch * kChunk;
        cp_async_wait1();                          // own copies of this chunk (the next chunk's may be pending)
        unsigned mask = 0u;
        for (int c = 0; c < n_phase; ++c)          // the votes also publish every thread's copies to the block
            if (__syncthreads_or(tid < kChunk && site0 + tid < nsites && cl[tid] == c)) mask |= 1u << c;
        const bool single = (mask & (mask - 1u)) == 0u;
        bool first = true;
        for (int c = 0; c < n_phase; ++c) {
            if (!(mask & (1u << c))) continue;
            if (!(ok = ops_free())) break;
            if (loader) {
                if (first) put_rows(mine + kStageS, e, nullptr, cl, -1, d, sg, Bhi, Blo);   // S~ = S + e
                put_rows(mine, nullptr, bt, cl, single ? -1 : c, d, sg, Ahi, Alo);        // beta mu (this class)
            }
            fence_proxy_async();
            tc_fence_before();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
                const uint32_t acc = tmem + (uint32_t)(c * N4);
                uint32_t accum = (seen >> c) & 1u;
#pragma unroll
                for (int kk = 0; kk < kChunk / 16; ++kk) {
                    const uint64_t ah = sw128_desc(smem_u32(Ahi + kk * 32)), al = sw128_desc(smem_u32(Alo + kk * 32));
                    const uint64_t bh = sw128_desc(smem_u32(Bhi + kk * 32)), bl = sw128_desc(smem_u32(Blo + kk * 32));
                    mma_bf16(acc, ah, bh, idesc, accum);
                    mma_bf16(acc, ah, bl, idesc, 1u);
                    mma_bf16(acc, al, bh, idesc, 1u);
                    accum = 1u;
                }
                mma_commit(smem_u32(done));
            }
            ++cnt;
            seen |= 1u << c;
            first = false;
        }
        // every thread has read its staged values and e[] / cl[] of this slot
        __syncthreads();
        issue(ch + 2, slot);
    }
    cp_async_wait0();
    // every MMA issued has completed (bounded) before TMEM is read and freed
    bool drained = true;
    if (cnt > 0u) {
        const unsigned long long t0 = global_ns();
        while (!mbar_try(smem_u32(done), (cnt - 1u) & 1u) && global_ns() - t0 < kTimeoutNs) {
        }
        drained = mbar_try(smem_u32(done), (cnt - 1u) & 1u);
    }
    ok = __syncthreads_and(ok && drained) != 0;
    tc_fence_after();
    if (ok) {
        // warps 0-3 and 4-7 read the same lanes (rows r), each half of the columns
        const int q = warp & 3, half = warp >> 2;
        const int r = q * 32 + lane;
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        for (int c = 0; c < n_phase; ++c) {
            if (!(seen & (1u << c))) continue;
            double *slot = slots + ((size_t)blockIdx.x * n_phase + c) * (size_t)N4 * N4;
            for (int col = half * (N4 / 2); col < (half + 1) * (N4 / 2); col += 16) {
                float v[16];
                tmem_ld16(tmem + lane_base + (uint32_t)(c * N4 + col), v);
                if (r < N4) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) slot[(size_t)r * N4 + col + j] += (double)v[j];
                }
            }
        }
    } else if (tid == 0) {
        atomicOr(&g_table_tc_err, kErrTableTimeout);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, tcols);
}

}  // namespace

bool adjoint_table_tc_supported(int n, int n_phase)
{
    const int N4 = 4 * n;
    return (N4 == 32 || N4 == 64 || N4 == 128) && n_phase * N4 <= 512;
}

cudaError_t launch_adjoint_table_tc(const AdjointParams &p, double *slots, int nslots, cudaStream_t s)
{
    const int N4 = 4 * p.n, nsites = p.nx * p.nz;
    uint32_t tcols = 32;
    while (tcols < (uint32_t)(p.n_phase * N4)) tcols <<= 1;
    const size_t smem = (size_t)kBuf + 2 * (size_t)kStageAligned + 64 + 1024;
    static bool attr = false;
    if (!attr) {
        const cudaError_t e = cudaFuncSetAttribute(k_adj_table_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int grid = std::min(nslots, (nsites + kChunk - 1) / kChunk);
    k_adj_table_tc<<<grid, kTT, smem, s>>>(reinterpret_cast<const float4 *>(p.beta_mu),
                                          reinterpret_cast<const float4 *>(p.S), p.coef, p.cls, slots, nsites, p.n,
                                          p.n_phase, tcols, p.beta_scale);
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
