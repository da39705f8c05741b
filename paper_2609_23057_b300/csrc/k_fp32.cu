// Fused collide+stream step, float32 on the CUDA cores.
//
// One step (Eq. 2 with the operator order of Sec. 2.1: emission, absorption,
// scattering, streaming) for a tile of consecutive lattice sites:
//   S~ = S + e (I of every direction)                         (Eq. 6/8)
//   P  = alpha S~ + beta Z_c S~                                (absorption, Eq. 11)
//   S_new(x + c_d, d) = P(x, d)                                (streaming)
// The 4n x 4n contraction Z_c S~ is a small GEMM per tile (M = sites,
// N = K = 4n), register-tiled 8 sites x 8 outputs per thread.  Streaming is a
// push: every thread stores its post-collision Stokes vectors at the neighbour
// site, and also writes the ghost value (zero or inflow) into its own entries
// whose upstream cell lies outside a non-periodic side -- those entries have
// no other writer.  The state is direction-major [d][site][4], so a warp's
// loads of one direction are contiguous 16-byte vectors.  With bilinear
// streaming in the gather form the kernel stores P at the site itself and the
// next step's load forms S~ from four taps of it (step_common.cuh).
#include "rtlb_internal.h"
#include "step_common.cuh"

namespace rtlb {

namespace {

template <int N4>
struct Cfg {
    static constexpr int TS = 8;                         // sites per thread
    static constexpr int CG = N4 / 8;                    // column groups (8 outputs each)
    static constexpr int SG = 256 / CG;                  // site groups
    static constexpr int SITES = SG * TS;                // sites per CTA
    static constexpr int KC = 16;                        // k rows per B chunk
    // S~ tile, two Z^T chunks (the next one is copied in while the current one
    // is used), four per-site words; the gather form adds the bilinear taps
    // (n = N4 / 4 directions x 12 words)
    static constexpr size_t SMEM = (size_t)N4 * SITES * 4 + (size_t)2 * KC * N4 * 4 + (size_t)SITES * 16;
    static constexpr size_t SMEM_GATHER = SMEM + (size_t)(N4 / 4) * 48;
};

__device__ __forceinline__ void cp_async16(float *dst, const float *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void store_out(const StepParams &p, int site, int x, int z, int d, float4 v)
{
    push_store_xz(p.dir, p.inflow, pack_bc(p.bc), p.S_new, p.nx, p.nz, p.n, site, x, z, d, v);
}

// GATHER: S holds the previous step's P and the tile load gathers S~ from
// the taps (the mixed tiles of a tensor-core gather form); a template
// parameter so that the plain step's load loop stays as it is.
template <int N4, bool GATHER>
__global__ void __launch_bounds__(256, 2) k_step_fp32_tiled(StepParams p)
{
    using C = Cfg<N4>;
    constexpr int TS = C::TS, SG = C::SG, SITES = C::SITES, KC = C::KC;
    extern __shared__ __align__(16) float smem[];
    float *As = smem;                        // [N4][SITES]   S~ (k-major)
    float *Bs = As + N4 * SITES;             // [2][KC][N4]   Z^T chunks
    float *s_alpha = Bs + 2 * KC * N4;       // [SITES]  alpha hi
    float *s_alo = s_alpha + SITES;          // [SITES]  alpha lo
    float *s_beta = s_alo + SITES;           // [SITES]
    int *s_cls = reinterpret_cast<int *>(s_beta + SITES);
    int *s_to = s_cls + SITES;                                   // [n][8] tap offsets (gather form)
    float *s_tw = reinterpret_cast<float *>(s_to + 8 * (N4 / 4)); // [n][4] tap weights
    __shared__ unsigned s_mask;

    const int n = p.n;
    int site0, nsites;
    if (p.tile_list) {
        // one CTA per slice of a listed tile of p.tile_span sites
        const int per = p.tile_span > SITES ? p.tile_span / SITES : 1;
        const int tile = p.tile_list[blockIdx.x / per];
        site0 = tile * p.tile_span + (blockIdx.x % per) * SITES;
        nsites = min(p.nx * p.nz, tile * p.tile_span + p.tile_span);
    } else {
        site0 = blockIdx.x * SITES;
        nsites = p.nx * p.nz;
    }
    const int nsites_all = p.nx * p.nz;
    const int tid = threadIdx.x;
    if (tid == 0) s_mask = 0u;
    if (GATHER)
        for (int k = tid; k < 12 * n; k += 256) {
            if (k < 8 * n) s_to[k] = p.taps_o[k];
            else s_tw[k - 8 * n] = p.taps_w[k - 8 * n];
        }
    __syncthreads();

    // coefficients and classes of the tile
    unsigned my_mask = 0u;
    for (int s = tid; s < SITES; s += 256) {
        const int site = site0 + s;
        float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
        int cl = 0;
        if (site < nsites) {
            c = p.coef[site];
            cl = p.cls[site];
        }
        s_alpha[s] = c.x;
        s_alo[s] = c.y;
        s_beta[s] = c.z;
        s_cls[s] = cl;
        if (site < nsites) my_mask |= 1u << cl;
    }
    if (my_mask) atomicOr(&s_mask, my_mask);

    // S~ tile, transposed to k-major; emission added to I (Eq. 6/8).  In the
    // gather form S~ is the bilinear sum of the previous step's P.
    const float4 *S4 = reinterpret_cast<const float4 *>(p.S);
    const int bcbits = pack_bc(p.bc);
    for (int idx = tid; idx < n * SITES; idx += 256) {
        const int d = idx / SITES, s = idx - d * SITES;
        const int site = site0 + s;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (site < nsites) {
            if (GATHER) {
                const int z = site / p.nx;
                v = gather_bilinear(load_taps<true>(s_to, s_tw, d), S4 + (size_t)d * nsites_all,
                                    reinterpret_cast<const float4 *>(p.inflow), bcbits, p.nx, p.nz, n, d, site,
                                    site - z * p.nx, z);
            } else {
                v = S4[(size_t)d * nsites_all + site];
            }
            v.x += p.coef[site].w;
        }
        As[(4 * d + 0) * SITES + s] = v.x;
        As[(4 * d + 1) * SITES + s] = v.y;
        As[(4 * d + 2) * SITES + s] = v.z;
        As[(4 * d + 3) * SITES + s] = v.w;
    }
    __syncthreads();

    // this thread's eight sites: four at sg * 4 and four half a tile further,
    // so that a warp's site groups read consecutive 16-byte chunks of a row
    // of As (one wavefront per 128 bytes, no bank conflicts)
    const int sg = tid % SG, cg = tid / SG;
    const int sl0 = sg * 4, sl1 = SITES / 2 + sg * 4;
    auto site_of = [&](int i) { return i < 4 ? sl0 + i : sl1 + i - 4; };
    const int c0 = cg * 8;        // first output column of this thread
    const unsigned mask = s_mask;
    const bool mixed = (mask & (mask - 1u)) != 0u;

    float acc[TS][8];
#pragma unroll
    for (int i = 0; i < TS; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    // the (class, chunk) sequence: every KC-row chunk of Z_c^T for each class
    // present, the next chunk's copies in flight while the current one is used
    constexpr int NCH = N4 / KC;
    auto next_class = [&](int cl) {
        const unsigned rest = cl < 31 ? mask & ~((2u << cl) - 1u) : 0u;
        return rest ? __ffs(rest) - 1 : -1;
    };
    auto load_chunk = [&](int cl, int ch, int buf) {
        const float *src = p.ZT + (size_t)cl * N4 * N4 + (size_t)ch * KC * N4;
        float *dst = Bs + buf * KC * N4;
        for (int idx = tid; idx < KC * N4 / 4; idx += 256) cp_async16(dst + 4 * idx, src + 4 * idx);
        cp_async_commit();
    };
    int cl = mask ? __ffs(mask) - 1 : -1;
    if (cl >= 0) load_chunk(cl, 0, 0);
    int buf = 0;
    while (cl >= 0) {
        const int ncl = next_class(cl);
        float m[TS];
#pragma unroll
        for (int i = 0; i < TS; ++i) m[i] = (!mixed || s_cls[site_of(i)] == cl) ? 1.f : 0.f;
        for (int ch = 0; ch < NCH; ++ch) {
            const int k0 = ch * KC;
            if (ch + 1 < NCH) load_chunk(cl, ch + 1, buf ^ 1);
            else if (ncl >= 0) load_chunk(ncl, 0, buf ^ 1);
            else cp_async_commit();              // empty group: the wait below counts the same way
            cp_async_wait1();                    // this thread's copies of the current chunk
            __syncthreads();                     // everyone's
            const float *Bc = Bs + buf * KC * N4;
#pragma unroll 4
            for (int k = 0; k < KC; ++k) {
                const float4 a0 = *reinterpret_cast<const float4 *>(&As[(k0 + k) * SITES + sl0]);
                const float4 a1 = *reinterpret_cast<const float4 *>(&As[(k0 + k) * SITES + sl1]);
                const float4 b0 = *reinterpret_cast<const float4 *>(&Bc[k * N4 + c0]);
                const float4 b1 = *reinterpret_cast<const float4 *>(&Bc[k * N4 + c0 + 4]);
                float a[TS] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
                if (mixed) {
#pragma unroll
                    for (int i = 0; i < TS; ++i) a[i] *= m[i];
                }
#pragma unroll
                for (int i = 0; i < TS; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
            }
            __syncthreads();                     // the buffer is free for the chunk after next
            buf ^= 1;
        }
        cl = ncl;
    }
    cp_async_wait0();

    // epilogue: P = alpha S~ + beta Y, pushed to the neighbour
#pragma unroll
    for (int i = 0; i < TS; ++i) {
        const int s = site_of(i), site = site0 + s;
        if (site >= nsites) continue;
        const int z = site / p.nx, x = site - z * p.nx;
        const float al = s_alpha[s], alo = s_alo[s], be = s_beta[s];
#pragma unroll
        for (int jd = 0; jd < 2; ++jd) {
            const int d = (c0 >> 2) + jd;
            const int col = 4 * d;
            float o[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float sv = As[(col + k) * SITES + s];
                o[k] = fmaf(al, sv, fmaf(alo, sv, be * acc[i][4 * jd + k]));
            }
            store_out(p, site, x, z, d, make_float4(o[0], o[1], o[2], o[3]));
        }
    }
}

// Any n: one thread per (site, outgoing direction); Z^T read through the
// read-only cache (the whole warp shares one direction and usually one class).
template <bool GATHER>
__global__ void __launch_bounds__(128) k_step_fp32_generic(StepParams p)
{
    const int nsites = p.nx * p.nz;
    const int site = blockIdx.x * blockDim.x + threadIdx.x;
    const int o = blockIdx.y;
    if (site >= nsites) return;
    const int N4 = 4 * p.n;
    const float4 cf = p.coef[site];
    const float *Zc = p.ZT + (size_t)p.cls[site] * N4 * N4;
    const float4 *S4 = reinterpret_cast<const float4 *>(p.S);
    float y[4] = {0.f, 0.f, 0.f, 0.f};
    float4 own = make_float4(0.f, 0.f, 0.f, 0.f);
    const int zs = site / p.nx;
    for (int d = 0; d < p.n; ++d) {
        float4 v = GATHER ? gather_bilinear(load_taps(p.taps_o, p.taps_w, d), S4 + (size_t)d * nsites,
                                              reinterpret_cast<const float4 *>(p.inflow), pack_bc(p.bc), p.nx, p.nz,
                                              p.n, d, site, site - zs * p.nx, zs)
                            : S4[(size_t)d * nsites + site];
        v.x += cf.w;
        if (d == o) own = v;
        const float sv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int r = 0; r < 4; ++r) y[r] = fmaf(__ldg(&Zc[(size_t)(4 * d + k) * N4 + 4 * o + r]), sv[k], y[r]);
    }
    float4 v;
    v.x = fmaf(cf.x, own.x, fmaf(cf.y, own.x, cf.z * y[0]));
    v.y = fmaf(cf.x, own.y, fmaf(cf.y, own.y, cf.z * y[1]));
    v.z = fmaf(cf.x, own.z, fmaf(cf.y, own.z, cf.z * y[2]));
    v.w = fmaf(cf.x, own.w, fmaf(cf.y, own.w, cf.z * y[3]));
    store_out(p, site, site - zs * p.nx, zs, o, v);
}

template <int N4, bool GATHER>
cudaError_t launch_tiled(const StepParams &p, cudaStream_t s)
{
    using C = Cfg<N4>;
    constexpr size_t smem = GATHER ? C::SMEM_GATHER : C::SMEM;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_step_fp32_tiled<N4, GATHER>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    int grid;
    if (p.tile_list) {
        const int per = p.tile_span > C::SITES ? p.tile_span / C::SITES : 1;
        grid = p.n_tiles * per;
    } else {
        grid = (p.nx * p.nz + C::SITES - 1) / C::SITES;
    }
    if (grid == 0) return cudaSuccess;
    k_step_fp32_tiled<N4, GATHER><<<grid, 256, smem, s>>>(p);
    return cudaGetLastError();
}

template <bool GATHER>
cudaError_t launch_fp32(const StepParams &p, cudaStream_t s)
{
    switch (4 * p.n) {
    case 32: return launch_tiled<32, GATHER>(p, s);
    case 64: return launch_tiled<64, GATHER>(p, s);
    case 128: return launch_tiled<128, GATHER>(p, s);
    case 256: return launch_tiled<256, GATHER>(p, s);
    default: {
        const int nsites = p.nx * p.nz;
        dim3 grid((nsites + 127) / 128, p.n);
        k_step_fp32_generic<GATHER><<<grid, 128, 0, s>>>(p);
        return cudaGetLastError();
    }
    }
}

}  // namespace

cudaError_t launch_step_fp32(const StepParams &p, cudaStream_t s)
{
    return p.taps_o ? launch_fp32<true>(p, s) : launch_fp32<false>(p, s);
}

}  // namespace rtlb
