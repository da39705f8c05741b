// Split FP8 tensor-core form of the fused collide+stream step (precision
// RTLB_PREC_FP8X): e4m3 operands with UE8M0 block scales, both operands
// split into several e4m3 terms so that the form reaches the accuracy of the
// bf16 split-table form.
//
// Per tile of 128 sites, with x = beta * S~ (float32) and the table Z with its
// forward blocks taken out (as in every tensor-core form):
//
//   state:  x = s0 + s1 (+ remainder below 2^-8 |x|): per site and 8-direction
//           slot (one 32-value MX block), s0 = e4m3(x 2^-e0) 2^e0 with e0 from
//           the block's largest |x|, s1 = e4m3(r 2^-d) 2^(e0 + d) for the exact
//           remainder r = x 2^-e0 - e4m3(x 2^-e0), d from the block's largest |r|
//   table:  Z = t0 + t1 + t2 (+ remainder below 2^-12 |Z|): per row and 32-column
//           block, each term the e4m3 of what the terms before it left, with
//           its own scale (prepared on the host from float64)
//   D  <- (alpha + beta c_d) S~                             (float32, converters)
//   D  += s0.t0 + s0.t1 + s0.t2 + s1.t0 + s1.t1             (block-scaled MMAs)
//
// issued as tcgen05.mma kind::mxf8f6f4.block_scale.scale_vec::1X (K = 32 per
// instruction: one slot).  The dropped s1.t2 product is below 2^-12 of a
// product.  On the paper's cloud workload this form's error matches the
// bf16 split-table form's (a CPU emulation with exact accumulation: 3.3e-4 on
// the top radiance of a 128x128 crop after 200 steps; single-term e4m3:
// 5.9e-2).
//
// Memory plan at n = 64: the three table terms take 192 KB of shared memory,
// so the two state terms live in tensor memory and the MMA reads A from
// there (TS form; each TMEM column holds one direction's four Stokes bytes).
// TMEM (512 columns at n = 64 with two phase classes): the accumulator D
// (4n), A terms s0 and s1 (n each), the A scales packed four K steps per
// 32-bit cell (a converter group owns slots j = g, g + 2, ..., so its four
// scale bytes of a tile go into one cell per term: 4 regions of 8 columns),
// and the B scales of every (term, class), resident for the launch.  The
// accumulator is single and handed back per slot as in the single-term FP8
// kernel (d_free[j]); a converter past slot j's hand-off also knows the
// previous tile's MMAs completed, so A, its scales and the init may be
// overwritten.  Two 16 KB staging slots fit beside the table; the producer
// also prefetches the state chunk a few slots ahead into L2.
//
// Warp roles: warps 0-7 epilogue, 8-15 converters (two groups on alternate
// slots), 16 TMA producer, 17 MMA issuer.  Every wait is bounded (about 2 s);
// on timeout the CTA records an error code, drains what it issued and leaves.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <algorithm>

#include "step_common.cuh"
#include "tc.h"
#include "tc_common.cuh"
#include "tc_ptx.cuh"

#ifndef RTLB_TC_FP8X_PREFETCH_SLOTS
#define RTLB_TC_FP8X_PREFETCH_SLOTS 4
#endif

namespace rtlb {

namespace {

using namespace tcptx;
using namespace tccommon;

constexpr int kSfCols = 8;     // scale regions start on 8-column boundaries
constexpr int kTerms = 3;      // table terms
// products issued per K step: (state term, table term) = (0,0), (0,1), (0,2),
// (1,0), (1,1)

// D[tmem] (+)= A[tmem] . B[smem]^T, e4m3 operands, block scales (see mma_mxf8).
__device__ __forceinline__ void mma_mxf8_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                            uint32_t sfa, uint32_t sfb, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %6, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::mxf8f6f4.block_scale.scale_vec::1X [%0], [%1], %2, %3, [%4], [%5], p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(sfa), "r"(sfb), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tmem_st8w(uint32_t taddr, const uint32_t v[8])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
                 "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}

// The four e4m3 values of a packed word as floats (exact).
__device__ __forceinline__ void e4m3x4_to_float(uint32_t w, float f[4])
{
    const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w & 0xFFFFu), __NV_E4M3);
    const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w >> 16), __NV_E4M3);
    const float2 a = __half22float2(__half2(lo)), b = __half22float2(__half2(hi));
    f[0] = a.x;
    f[1] = a.y;
    f[2] = b.x;
    f[3] = b.y;
}

// TMEM columns of the form (regions on 32-column boundaries): the
// accumulator D [0, 4n), the state terms s0 and s1 (n columns each: one per
// direction, its four Stokes bytes), the A scales (4 regions of 8: term x
// converter group) and the B scales of every (term, class, set of 4 K steps).
struct FxCols {
    int a0, a1, sa, sb;
};
__host__ __device__ constexpr int round32(int v) { return (v + 31) / 32 * 32; }
__host__ __device__ inline FxCols fx_cols(int N4)
{
    FxCols c{};
    c.a0 = round32(N4);
    c.a1 = c.a0 + round32(N4 / 4);
    c.sa = c.a1 + round32(N4 / 4);
    c.sb = c.sa + 4 * kSfCols;
    return c;
}

// Order in which a tile's staging slots are loaded and converted.  The two
// halves of the epilogue warps hand the accumulator back slot by slot from
// the start of each half of the directions; at n = 64 (8 slots) the order
// 0, 1, 4, 5, 2, 3, 6, 7 gives each converter group its slots in the order
// they are handed back (group 0: 0, 4, 2, 6; group 1: 1, 5, 3, 7).
__device__ __forceinline__ int slot_of(int k, int groups)
{
    return groups == 8 ? ((k & 1) | ((k >> 1) & 1) << 2 | (k >> 2) << 1) : k;
}

__global__ void __launch_bounds__(kThreads, 1)
    k_step_tc_fp8x(const __grid_constant__ CUtensorMap tmS, const __grid_constant__ CUtensorMap tmZ, TcParams p,
                   const uint8_t *__restrict__ sfb, int N4, int stages, int n_phase, uint32_t tcols)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const int C8 = (N4 + 127) / 128;               // 128-byte (128-element) K chunks
    const int ksteps = N4 / 32;                    // MMA K steps = 8-direction slots
    const int n = p.n;
    const int nsites = p.nx * p.nz;
    const int groups = n / kDirsPerStage;          // slots per tile
    const uint32_t z_chunk = (uint32_t)N4 * 128u;
    const int bcols = N4 / 32;                     // TMEM columns of one B scale set used
    const int bsets = (ksteps + 3) / 4;            // four K steps per set (one byte each)
    const FxCols L = fx_cols(N4);                  // TMEM layout: D at 0, the two state terms, scales
    const int colA0 = L.a0, colA1 = L.a1, colSA = L.sa, colSB = L.sb;

    uint8_t *sZ = smem;                            // [term][chunk] of z_chunk bytes
    uint8_t *sStage = sZ + kTerms * C8 * z_chunk;
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

    // B scales of every (term, class), resident for the whole launch: set st,
    // column cc hold rows n = 32 cc + l at lane l of every quadrant, the byte k
    // of the cell being K step 4 st + k
    if (warp < 4) {
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        for (int tc = 0; tc < kTerms * n_phase; ++tc)
            for (int st = 0; st < bsets; ++st)
                for (int cc = 0; cc < bcols; ++cc) {
                    const int row = 32 * cc + lane;
                    uint32_t cell = 0;
                    for (int k = 0; k < 4; ++k) {
                        const int ks = 4 * st + k;
                        if (ks < ksteps) cell |= (uint32_t)sfb[((size_t)tc * N4 + row) * ksteps + ks] << (8 * k);
                    }
                    tmem_st1(tmem + lane_base + (uint32_t)(colSB + (tc * bsets + st) * kSfCols + cc), cell);
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
                    mbar_expect_tx(zb, (uint32_t)(kTerms * C8) * z_chunk);
                    for (int t = 0; t < kTerms; ++t)
                        for (int c = 0; c < C8; ++c)
                            tma_load_3d(smem_u32(sZ + (t * C8 + c) * z_chunk), &tmZ, zb, 128 * c, 0, t * n_phase + cls);
                    prev_cls = cls;
                }
                for (int kq = 0; kq < groups && ok; ++kq) {
                    const int j = slot_of(kq, groups);
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
                    if (RTLB_TC_FP8X_PREFETCH_SLOTS > 0) {
                        // two staging slots hold ~32 KB in flight: the chunk a
                        // few slots ahead goes to L2 meanwhile
                        const int ahead = i * groups + kq + RTLB_TC_FP8X_PREFETCH_SLOTS;
                        const int ia = ahead / groups, ja = slot_of(ahead - ia * groups, groups);
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
            // descriptors of the three table terms; a byte offset o (a multiple
            // of 16) moves a descriptor by o >> 4 (its start-address field)
            uint64_t bz[kTerms];
#pragma unroll
            for (int b = 0; b < kTerms; ++b) bz[b] = sw128_desc(smem_u32(sZ + (uint32_t)(b * C8) * z_chunk));
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
                uint32_t sbb[kTerms];                  // B scale columns of this class, per term
#pragma unroll
                for (int b = 0; b < kTerms; ++b) sbb[b] = tmem + (uint32_t)(colSB + (b * n_phase + cls) * bsets * kSfCols);
                for (int ks = 0; ks < ksteps; ++ks) {
                    const uint64_t doff = (uint64_t)(((uint32_t)(ks & 3) * 32u + (uint32_t)(ks / 4) * z_chunk) >> 4);
                    const uint32_t idesc = idesc_mxf8(kTileM, N4, ks >> 1, ks & 3);
                    const uint32_t sa0 = tmem + (uint32_t)(colSA + kSfCols * (ks & 1));   // term 0; term 1 two regions on
                    const uint32_t sbo = (uint32_t)((ks / 4) * kSfCols);
                    const uint32_t a0 = tmem + (uint32_t)(colA0 + 8 * ks), a1 = tmem + (uint32_t)(colA1 + 8 * ks);
                    mma_mxf8_ts(tmem, a0, bz[0] + doff, idesc, sa0, sbb[0] + sbo, 1u);
                    mma_mxf8_ts(tmem, a0, bz[1] + doff, idesc, sa0, sbb[1] + sbo, 1u);
                    mma_mxf8_ts(tmem, a0, bz[2] + doff, idesc, sa0, sbb[2] + sbo, 1u);
                    mma_mxf8_ts(tmem, a1, bz[0] + doff, idesc, sa0 + 2 * kSfCols, sbb[0] + sbo, 1u);
                    mma_mxf8_ts(tmem, a1, bz[1] + doff, idesc, sa0 + 2 * kSfCols, sbb[1] + sbo, 1u);
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
            uint32_t sc0 = 0, sc1 = 0;                 // this group's packed scale bytes (four slots)
            for (int kq = grp; kq < groups && ok; kq += 2) {
                const int j = slot_of(kq, groups);     // same group: slot_of keeps the parity
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
                // the slot's 32 values S~ = S + e (emission on I) into registers;
                // the staging slot goes back to the producer at once, and all
                // the quantization happens before the wait for this slot's
                // accumulator columns
                float sv[32];
#pragma unroll
                for (int dl = 0; dl < kDirsPerStage; ++dl) {
                    const float4 v = stg[dl * kHalfSites];
                    sv[4 * dl] = v.x + cf.w;
                    sv[4 * dl + 1] = v.y;
                    sv[4 * dl + 2] = v.z;
                    sv[4 * dl + 3] = v.w;
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&st_empty[s]));
                // hi scale: largest |beta S~| of the slot's 32 values
                float amax = 0.f;
#pragma unroll
                for (int k = 0; k < 32; ++k) amax = fmaxf(amax, fabsf(sv[k]));
                const int e0 = block_exponent(fabsf(cf.z) * amax);
                const float inv0 = __uint_as_float((uint32_t)(127 - e0) << 23);   // 2^-e0, exact
                uint32_t w0[8];
                float rmax = 0.f;
#pragma unroll
                for (int dl = 0; dl < kDirsPerStage; ++dl) {
                    float x[4], h[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) x[k] = (cf.z * sv[4 * dl + k]) * inv0;   // beta S~ / 2^e0
                    w0[dl] = e4m3x2(x[0], x[1]) | (e4m3x2(x[2], x[3]) << 16);
                    e4m3x4_to_float(w0[dl], h);
#pragma unroll
                    for (int k = 0; k < 4; ++k) rmax = fmaxf(rmax, fabsf(x[k] - h[k]));   // exact remainders
                }
                // lo scale from the remainders' own maximum; a lo term below the
                // smallest scale (e0 + d < -127) is left out
                const int dlo = block_exponent(rmax);
                const bool lo_on = e0 + dlo >= -127;
                const float invd = __uint_as_float((uint32_t)(127 - dlo) << 23);   // 2^-d, exact (d <= 127)
                uint32_t w1[8];
#pragma unroll
                for (int dl = 0; dl < kDirsPerStage; ++dl) {
                    float h[4], y[4];
                    e4m3x4_to_float(w0[dl], h);
#pragma unroll
                    for (int k = 0; k < 4; ++k) y[k] = lo_on ? ((cf.z * sv[4 * dl + k]) * inv0 - h[k]) * invd : 0.f;
                    w1[dl] = e4m3x2(y[0], y[1]) | (e4m3x2(y[2], y[3]) << 16);
                }
                // the previous tile's epilogue has read this slot's columns, so
                // its MMAs (and their reads of A and its scales) completed
                ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&d_free[j]), (i & 1) ^ 1, abort_flag, p.err,
                                                       kErrTimeoutConverter));
                if (!ok) break;
                tc_fence_after();
#pragma unroll
                for (int dl = 0; dl < kDirsPerStage; dl += 2) {
                    const float g0 = fmaf(cf.z, fw[dl], cf.y), g1 = fmaf(cf.z, fw[dl + 1], cf.y);
                    float init[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        init[k] = fmaf(cf.x, sv[4 * dl + k], (k < 4 ? g0 : g1) * sv[4 * dl + k]);   // exact float32 part
                    tmem_st8(tmem + lane_base + (uint32_t)(4 * (d_beg + dl)), init);
                }
                tmem_st8w(tmem + lane_base + (uint32_t)(colA0 + 8 * j), w0);
                tmem_st8w(tmem + lane_base + (uint32_t)(colA1 + 8 * j), w1);
                const int e1 = lo_on ? e0 + dlo : -127;
                sc0 |= (uint32_t)(e0 + 127) << (8 * (j >> 1));
                sc1 |= (uint32_t)(e1 + 127) << (8 * (j >> 1));
            }
            if (!ok) break;
            // scale cells of this group (every slot of the tile passed its hand-off)
            if (grp < groups) {
                tmem_st1(tmem + lane_base + (uint32_t)(colSA + kSfCols * (0 + grp) + q), sc0);
                tmem_st1(tmem + lane_base + (uint32_t)(colSA + kSfCols * (2 + grp) + q), sc1);
            }
            tmem_wait_st();
            tc_fence_before();
            __syncwarp();
            // arrive for tile i only once t_ready's phase for tile i - 1 has
            // completed (a warp without a slot, group 1 at n = 8, would run ahead)
            ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(t_ready), (i & 1) ^ 1, abort_flag, p.err,
                                                   kErrTimeoutConverter));
            if (!ok) break;
            if (lane == 0) mbar_arrive(smem_u32(t_ready));
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
            const int site = tile * kTileM + r;
            const int z = site / p.nx, x = site - z * p.nx;
            const bool interior = site < nsites && x > 0 && x < p.nx - 1 && z > 0 && z < p.nz - 1;
            ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(acc_full), i & 1, abort_flag, p.err, kErrTimeoutEpilogue));
            if (!ok) break;
            tc_fence_after();
            // two slots (16 directions, 64 columns) per load where the half
            // holds them, fewer at small n; the slots go back to the converters
            // as soon as their columns are in registers, before the stores
            // (which proceed at the SM's share of the write bandwidth)
            const int step = dn >= 16 ? 16 : (dn >= kDirsPerStage ? kDirsPerStage : 4);
            for (int d0 = dbeg; d0 < dbeg + dn; d0 += step) {
                float v[64];
                if (step == 16) tmem_ld64(tmem + lane_base + (uint32_t)(4 * d0), v);
                else if (step == kDirsPerStage) tmem_ld32(tmem + lane_base + (uint32_t)(4 * d0), v);
                else tmem_ld16(tmem + lane_base + (uint32_t)(4 * d0), v);
                tc_fence_before();
                __syncwarp();
                if (lane == 0)
                    for (int sl = d0 / kDirsPerStage; sl * kDirsPerStage < d0 + step; ++sl)
                        mbar_arrive(smem_u32(&d_free[sl]));
                if (interior) {
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        if (k < step) {
                            const int d = d0 + k;
                            const long long t = (long long)d * nsites + site + s_cx[d] + (long long)s_cz[d] * p.nx;
                            __stcs(&out[t], make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]));
                        }
                    }
                } else if (site < nsites) {
#pragma unroll
                    for (int k = 0; k < 16; ++k)
                        if (k < step)
                            push_store_xz(p.dir, p.inflow, p.bcbits, p.S_new, p.nx, p.nz, n, site, x, z, d0 + k,
                                       make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]));
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

int tc_fp8x_tmem_columns(int N4, int n_phase)
{
    const int ksteps = N4 / 32, bsets = (ksteps + 3) / 4;
    return fx_cols(N4).sb + kTerms * n_phase * bsets * kSfCols;
}

size_t tc_fp8x_smem_bytes(int N4, int stages)
{
    const int C8 = (N4 + 127) / 128, groups = N4 / 32;
    const size_t b = (size_t)kTerms * C8 * N4 * 128 + (size_t)stages * kStageBytes + (size_t)(2 * stages + groups + 5) * 8 +
                     16 + 2 * kMaxDirs;
    return b + 1024;  // alignment slack
}

cudaError_t launch_step_tc_fp8x(const CUtensorMap &tmS, const CUtensorMap &tmZ, const TcParams &p, const uint8_t *sfb,
                                int N4, int stages, int n_phase, int grid, cudaStream_t s)
{
    const int cols = tc_fp8x_tmem_columns(N4, n_phase);
    if (cols > 512 || N4 % 32 != 0 || N4 > 256 || stages < 2 || stages % 2 != 0) return cudaErrorInvalidValue;
    uint32_t tcols = 32;
    while (tcols < (uint32_t)cols) tcols <<= 1;
    const size_t smem = tc_fp8x_smem_bytes(N4, stages);
    if (smem > (size_t)kSmemLimit) return cudaErrorInvalidValue;
    const cudaError_t e = cudaFuncSetAttribute(k_step_tc_fp8x, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_step_tc_fp8x<<<grid, kThreads, smem, s>>>(tmS, tmZ, p, sfb, N4, stages, n_phase, tcols);
    return cudaGetLastError();
}

}  // namespace rtlb
