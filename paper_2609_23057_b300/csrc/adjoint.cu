// Reverse-mode adjoint of the fused step (float32 on the CUDA cores).
//
// The step is affine in the state: S^{t+1} = T (C S^t + c0) + b with
// C = blockdiag(alpha I + beta Z_c) per site (Eq. 11 with the emission of
// Eq. 6 folded into c0) and T the push streaming with its ghost values b.
// For a loss L(S^N) with seed lambda^N = dL/dS^N the adjoint recursion is
//   mu^{t+1} = T^T lambda^{t+1}   (pull from each entry's streaming target;
//                                  zero when the vector left the lattice)
//   lambda^t = alpha mu + beta Z_c^T mu
// and the parameter gradients of step t are
//   dL/dalpha_site += <mu, S~>,  dL/dbeta_site += <Z_c^T mu, S~>,
//   dL/dZ_c        += sum over the class's sites of beta mu (x) S~,
// with S~ = S^t + e.  k_adj_step computes the first three (the Z^T mu
// contraction is the forward kernel's GEMM with the table untransposed);
// k_adj_table accumulates the last one as a GEMM over sites.
#include <algorithm>
#include <cmath>

#include "rtlb_internal.h"
#include "step_common.cuh"

namespace rtlb {

namespace {

template <int N4>
struct AdjCfg {
    static constexpr int TS = 8;
    static constexpr int CG = N4 / 8;
    static constexpr int SG = 256 / CG;
    static constexpr int SITES = SG * TS;
    static constexpr int KC = 16;
    // mu tile, table chunk, five per-site words and the per-site dot-product
    // partials of each column group (summed in a fixed order, so the
    // gradients are deterministic); S~ is read from global memory where it is
    // used, which keeps two CTAs resident per SM
    static constexpr size_t SMEM =
        (size_t)N4 * SITES * 4 + (size_t)KC * N4 * 4 + (size_t)SITES * 20 + (size_t)2 * CG * SITES * 4;
};

// NU = false: lambda form (mu = T^T lambda^{t+1} pulled here, lambda^t stored
// in place, beta mu written for the table gradient); one block per SITES
// consecutive sites.  NU = true (4n = 128, SITES = 128): transposed-stream
// form for the tiles of p.tiles -- the input is nu^t = mu itself, lambda^t is
// pushed along the negated offsets (or stored in place when !p.push), and the
// table gradient reads nu^t directly.
template <int N4, bool NU>
__global__ void __launch_bounds__(256, 2) k_adj_step(AdjointParams p)
{
    using Cf = AdjCfg<N4>;
    constexpr int TS = Cf::TS, SG = Cf::SG, SITES = Cf::SITES, KC = Cf::KC;
    extern __shared__ __align__(16) float smem[];
    float *Ms = smem;                          // [N4][SITES]  mu (k-major)
    float *Bs = Ms + N4 * SITES;               // [KC][N4]     table chunk
    float *s_ahi = Bs + KC * N4;
    float *s_alo = s_ahi + SITES;
    float *s_beta = s_alo + SITES;
    float *s_e = s_beta + SITES;
    int *s_cls = reinterpret_cast<int *>(s_e + SITES);
    float *s_pa = reinterpret_cast<float *>(s_cls + SITES);   // [CG][TS][SG] partials of <mu, S~>
    float *s_pb = s_pa + Cf::CG * SITES;                      // [CG][TS][SG] partials of <Y, S~>
    __shared__ unsigned s_mask;

    const int n = p.n;
    const int nsites = p.nx * p.nz;
    const int site0 = NU ? (p.tiles[blockIdx.x] & 0xFFFFFF) * SITES : blockIdx.x * SITES;
    const int tid = threadIdx.x;
    if (tid == 0) s_mask = 0u;
    __syncthreads();
    unsigned my_mask = 0u;
    for (int s = tid; s < SITES; s += 256) {
        const int site = site0 + s;
        float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
        int cl = 0;
        if (site < nsites) {
            c = p.coef[site];
            cl = p.cls[site];
            my_mask |= 1u << cl;
        }
        s_ahi[s] = c.x;
        s_alo[s] = c.y;
        s_beta[s] = c.z;
        s_e[s] = c.w;
        s_cls[s] = cl;
    }
    if (my_mask) atomicOr(&s_mask, my_mask);

    // mu = T^T lambda (pull from the push target)
    const float4 *L4 = reinterpret_cast<const float4 *>(p.lam_next);
    const float4 *S4 = reinterpret_cast<const float4 *>(p.S);
    const bool per_x = p.bc[RTLB_SIDE_LEFT] == RTLB_BC_PERIODIC, per_z = p.bc[RTLB_SIDE_TOP] == RTLB_BC_PERIODIC;
    for (int idx = tid; idx < n * SITES; idx += 256) {
        const int d = idx / SITES, s = idx - d * SITES;
        const int site = site0 + s;
        float4 m = make_float4(0.f, 0.f, 0.f, 0.f);
        if (site < nsites) {
            if (NU) {
                m = L4[(size_t)d * nsites + site];
            } else {
                const int z = site / p.nx, x = site - z * p.nx;
                int xt = x + p.dir[d], zt = z + p.dir[n + d];
                if (per_x) xt = wrap_coord(xt, p.nx);
                if (per_z) zt = wrap_coord(zt, p.nz);
                if (xt >= 0 && xt < p.nx && zt >= 0 && zt < p.nz) m = L4[(size_t)d * nsites + (size_t)zt * p.nx + xt];
            }
        }
        Ms[(4 * d + 0) * SITES + s] = m.x;
        Ms[(4 * d + 1) * SITES + s] = m.y;
        Ms[(4 * d + 2) * SITES + s] = m.z;
        Ms[(4 * d + 3) * SITES + s] = m.w;
    }
    __syncthreads();

    // this thread's eight sites: four at sg * 4 and four half a tile further,
    // so that a warp's site groups read consecutive 16-byte chunks of a row of
    // Ms (no shared-memory bank conflicts)
    const int sg = tid % SG, cg = tid / SG;
    const int sl0 = sg * 4, sl1 = SITES / 2 + sg * 4, c0 = cg * 8;
    auto site_of = [&](int i) { return i < 4 ? sl0 + i : sl1 + i - 4; };
    const unsigned mask = s_mask;
    const bool mixed = (mask & (mask - 1u)) != 0u;
    float acc[TS][8];
#pragma unroll
    for (int i = 0; i < TS; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
    // Y = mu . Z  (Y[site][col] = sum_k mu[site][k] Z[k][col] = (Z^T mu)[col])
    for (int cl = 0; cl < p.n_phase; ++cl) {
        if (!(mask & (1u << cl))) continue;
        const float *Zc = p.Z + (size_t)cl * N4 * N4;
        float msk[TS];
#pragma unroll
        for (int i = 0; i < TS; ++i) msk[i] = (!mixed || s_cls[site_of(i)] == cl) ? 1.f : 0.f;
        for (int k0 = 0; k0 < N4; k0 += KC) {
            __syncthreads();
            for (int idx = tid; idx < KC * N4 / 4; idx += 256)
                reinterpret_cast<float4 *>(Bs)[idx] = reinterpret_cast<const float4 *>(Zc + (size_t)k0 * N4)[idx];
            __syncthreads();
#pragma unroll 4
            for (int k = 0; k < KC; ++k) {
                const float4 a0 = *reinterpret_cast<const float4 *>(&Ms[(k0 + k) * SITES + sl0]);
                const float4 a1 = *reinterpret_cast<const float4 *>(&Ms[(k0 + k) * SITES + sl1]);
                const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[k * N4 + c0]);
                const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[k * N4 + c0 + 4]);
                float a[TS] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
                if (mixed) {
#pragma unroll
                    for (int i = 0; i < TS; ++i) a[i] *= msk[i];
                }
#pragma unroll
                for (int i = 0; i < TS; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
            }
        }
    }

    // lambda^t = alpha mu + beta Y at the site itself; beta mu for the table
    // gradient; per-site <mu, S~> and <Y, S~>
    float4 *Lo = reinterpret_cast<float4 *>(p.lam_out);
    float4 *Mo = reinterpret_cast<float4 *>(p.beta_mu);
#pragma unroll
    for (int i = 0; i < TS; ++i) {
        const int s = site_of(i), site = site0 + s;
        if (site >= nsites) {
            s_pa[(cg * TS + i) * SG + sg] = 0.f;
            s_pb[(cg * TS + i) * SG + sg] = 0.f;
            continue;
        }
        const float ah = s_ahi[s], al = s_alo[s], be = s_beta[s];
        float pa = 0.f, pb = 0.f;
#pragma unroll
        for (int jd = 0; jd < 2; ++jd) {
            const int d = (c0 >> 2) + jd;
            float o[4], bm[4];
            float4 sv4 = __ldg(S4 + (size_t)d * nsites + site);
            sv4.x += s_e[s];
            const float svk[4] = {sv4.x, sv4.y, sv4.z, sv4.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float m = Ms[(4 * d + k) * SITES + s], sv = svk[k];
                const float y = acc[i][4 * jd + k];
                o[k] = fmaf(ah, m, fmaf(al, m, be * y));
                bm[k] = be * m;
                pa = fmaf(m, sv, pa);
                pb = fmaf(y, sv, pb);
            }
            const float4 lv = make_float4(o[0], o[1], o[2], o[3]);
            if (!NU) {
                Lo[(size_t)d * nsites + site] = lv;
                Mo[(size_t)d * nsites + site] = make_float4(bm[0], bm[1], bm[2], bm[3]);
            } else if (p.push) {
                push_store(p.dirT, nullptr, p.bcbitsT, p.lam_out, p.nx, p.nz, n, site, d, lv);
            } else {
                Lo[(size_t)d * nsites + site] = lv;
            }
        }
        s_pa[(cg * TS + i) * SG + sg] = pa;
        s_pb[(cg * TS + i) * SG + sg] = pb;
    }
    __syncthreads();
    for (int s = tid; s < SITES; s += 256) {
        const int site = site0 + s;
        if (site < nsites) {
            // the (i, sg) that site_of maps to s
            const int h = s >= SITES / 2, r = s - h * (SITES / 2);
            const int i = 4 * h + (r & 3), g = r >> 2;
            float a = 0.f, b = 0.f;
            for (int c = 0; c < Cf::CG; ++c) {
                a += s_pa[(c * TS + i) * SG + g];
                b += s_pb[(c * TS + i) * SG + g];
            }
            p.g_alpha[site] += (double)a;
            p.g_beta[site] += (double)b;
        }
    }
}

// dL/dZ_c += sum over the sites of class c of (beta mu)[site][r] S~[site][k]:
// a GEMM with the sites as the reduction dimension.  blockIdx.y picks a
// 128 x 128 (or N4 x N4) tile of the table, blockIdx.z the class; each CTA
// reduces a strided set of 32-site chunks in registers and adds its sum into
// its own slot of `slots` (no atomics).
template <int N4>
__global__ void __launch_bounds__(256, 2) k_adj_table(AdjointParams p, double *__restrict__ slots)
{
    constexpr int TT = N4 < 128 ? N4 : 128;    // tile edge
    constexpr int TPR = TT / 8;                // threads per tile row (8 outputs each)
    constexpr int NT = TPR * TPR;              // threads that own outputs
    constexpr int CH = 32;                     // sites per chunk
    __shared__ __align__(16) float Mt[CH][TT + 4];   // +4: conflict-free transposed stores
    __shared__ __align__(16) float St[CH][TT + 4];
    const int n = p.n, nsites = p.nx * p.nz;
    const int tiles_per_edge = N4 / TT;
    const int ty = blockIdx.y / tiles_per_edge, tx = blockIdx.y % tiles_per_edge;
    const int r0 = ty * TT, k0 = tx * TT;
    const int cl = blockIdx.z;
    const int tid = threadIdx.x;
    const int tr = tid / TPR, tc = tid % TPR;
    const bool owner = tid < NT;
    float acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
    const float4 *M4 = reinterpret_cast<const float4 *>(p.beta_mu);
    const float4 *S4 = reinterpret_cast<const float4 *>(p.S);
    for (int base = blockIdx.x * CH; base < nsites; base += gridDim.x * CH) {
        // skip chunks without a site of this class (single-class layers); the
        // vote is also the barrier before the tiles are overwritten
        if (!__syncthreads_or(tid < CH && base + tid < nsites && p.cls[base + tid] == cl)) continue;
        for (int idx = tid; idx < CH * (TT / 4); idx += 256) {
            const int s = idx % CH, dd = idx / CH;      // dd: direction within the tile edge
            const int site = base + s;
            float4 m = make_float4(0.f, 0.f, 0.f, 0.f), v = m;
            if (site < nsites && p.cls[site] == cl) {
                m = M4[(size_t)(r0 / 4 + dd) * nsites + site];
                if (p.beta_scale) {
                    const float be = p.coef[site].z;
                    m.x *= be;
                    m.y *= be;
                    m.z *= be;
                    m.w *= be;
                }
                v = S4[(size_t)(k0 / 4 + dd) * nsites + site];
                if ((k0 / 4 + dd) < n) v.x += p.coef[site].w;
            }
            *reinterpret_cast<float4 *>(&Mt[s][4 * dd]) = m;
            *reinterpret_cast<float4 *>(&St[s][4 * dd]) = v;
        }
        __syncthreads();
        if (owner) {
#pragma unroll 4
            for (int s = 0; s < CH; ++s) {
                const float4 a0 = *reinterpret_cast<const float4 *>(&Mt[s][8 * tr]);
                const float4 a1 = *reinterpret_cast<const float4 *>(&Mt[s][8 * tr + 4]);
                const float4 b0 = *reinterpret_cast<const float4 *>(&St[s][8 * tc]);
                const float4 b1 = *reinterpret_cast<const float4 *>(&St[s][8 * tc + 4]);
                const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
            }
        }
    }
    if (owner) {
        double *slot = slots + ((size_t)blockIdx.x * p.n_phase + cl) * (size_t)N4 * N4;   // [slot][class][r][k]
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) slot[(size_t)(r0 + 8 * tr + i) * N4 + k0 + 8 * tc + j] += (double)acc[i][j];
    }
}

// lambda^N: the loss gradient on the top row's outgoing directions.
__global__ void k_adj_seed(float *__restrict__ lam, const float4 *__restrict__ dL_dout, const int *__restrict__ dir,
                           int nx, int nz, int n)
{
    const size_t nsites = (size_t)nx * nz;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nx * n; j += gridDim.x * blockDim.x) {
        const int x = j / n, d = j % n;
        if (dir[n + d] == 1)
            reinterpret_cast<float4 *>(lam)[(size_t)d * nsites + (size_t)(nz - 1) * nx + x] = dL_dout[j];
    }
}

// Chain rule from (alpha, beta) to (tau, albedo):  alpha = A s, beta = A (1 - s),
// A = exp(-(1-w) tau) or 1 - (1-w) tau,  s = 1 - w tau or exp(-w tau).
__global__ void k_adj_chain(const double *__restrict__ ga, const double *__restrict__ gb, const float *__restrict__ tau,
                            const float *__restrict__ alb, int nsites, int surv_mode, int abs_mode,
                            float *__restrict__ g_tau, float *__restrict__ g_alb)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nsites; j += gridDim.x * blockDim.x) {
        const double t = tau[j], w = alb[j];
        const double kabs = (1.0 - w) * t, ksca = w * t;
        const double A = abs_mode == RTLB_ABS_TAYLOR ? 1.0 - kabs : exp(-kabs);
        const double dA = abs_mode == RTLB_ABS_TAYLOR ? -1.0 : -A;            // dA / dkabs
        const double s = surv_mode == RTLB_SURV_LINEAR ? 1.0 - ksca : exp(-ksca);
        const double ds = surv_mode == RTLB_SURV_LINEAR ? -1.0 : -s;          // ds / dksca
        // d/dtau: dkabs = (1 - w), dksca = w;   d/dw: dkabs = -t, dksca = t
        const double dAt = dA * (1.0 - w), dAw = -dA * t, dst = ds * w, dsw = ds * t;
        const double da_t = dAt * s + A * dst, da_w = dAw * s + A * dsw;
        const double db_t = dAt * (1.0 - s) - A * dst, db_w = dAw * (1.0 - s) - A * dsw;
        const double a = ga[j] + ga[nsites + j], b = gb[j] + gb[nsites + j];   // the two halves, in order
        g_tau[j] = (float)(a * da_t + b * db_t);
        g_alb[j] = (float)(a * da_w + b * db_w);
    }
}

__global__ void k_adj_fold_slots(const double *__restrict__ slots, int nslots, size_t len, double *__restrict__ out)
{
    for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < len; j += (size_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int s = 0; s < nslots; ++s) acc += slots[(size_t)s * len + j];
        out[j] = acc;
    }
}

template <int N4, bool NU>
cudaError_t launch_adj(const AdjointParams &p, int blocks, cudaStream_t s)
{
    using Cf = AdjCfg<N4>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_adj_step<N4, NU>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cf::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_adj_step<N4, NU><<<blocks, 256, Cf::SMEM, s>>>(p);
    return cudaGetLastError();
}

template <int N4>
cudaError_t launch_adj(const AdjointParams &p, cudaStream_t s)
{
    return launch_adj<N4, false>(p, (p.nx * p.nz + AdjCfg<N4>::SITES - 1) / AdjCfg<N4>::SITES, s);
}

// nu^{N-1} = T^T lambda^N: the loss gradient on the top row's outgoing
// directions, pushed along the negated offsets (the rest of nu is zero).
__global__ void k_adj_seed_nu(float *__restrict__ nu, const float4 *__restrict__ dL_dout, const int *__restrict__ dir,
                              int nx, int nz, int n, int bcbits)
{
    const size_t nsites = (size_t)nx * nz;
    const bool per_x = bc_of(bcbits, RTLB_SIDE_LEFT) == RTLB_BC_PERIODIC;
    const bool per_z = bc_of(bcbits, RTLB_SIDE_TOP) == RTLB_BC_PERIODIC;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nx * n; j += gridDim.x * blockDim.x) {
        const int x = j / n, d = j % n;
        if (dir[n + d] != 1) continue;
        int xt = x - dir[d], zt = nz - 1 - dir[n + d];
        if (per_x) xt = wrap_coord(xt, nx);
        if (per_z) zt = wrap_coord(zt, nz);
        if (xt >= 0 && xt < nx && zt >= 0 && zt < nz)
            reinterpret_cast<float4 *>(nu)[(size_t)d * nsites + (size_t)zt * nx + xt] = dL_dout[j];
    }
}

template <int N4>
cudaError_t launch_table(const AdjointParams &p, double *slots, int nslots, cudaStream_t s)
{
    constexpr int TT = N4 < 128 ? N4 : 128;
    dim3 grid(nslots, (N4 / TT) * (N4 / TT), p.n_phase);
    k_adj_table<N4><<<grid, 256, 0, s>>>(p, slots);
    return cudaGetLastError();
}

}  // namespace

bool adjoint_supported(int n) { return n == 8 || n == 16 || n == 32 || n == 64; }

int adjoint_table_slots() { return 148; }

cudaError_t launch_adjoint_step(const AdjointParams &p, double *slots, cudaStream_t s)
{
    // the table gradient runs on the tensor cores where its accumulators fit
    // in TMEM, on the CUDA cores otherwise
    const bool tc = adjoint_table_tc_supported(p.n, p.n_phase);
    const int ns = adjoint_table_slots();
    cudaError_t e;
    switch (4 * p.n) {
    case 32: e = launch_adj<32>(p, s); if (e == cudaSuccess) e = tc ? launch_adjoint_table_tc(p, slots, ns, s) : launch_table<32>(p, slots, ns, s); break;
    case 64: e = launch_adj<64>(p, s); if (e == cudaSuccess) e = tc ? launch_adjoint_table_tc(p, slots, ns, s) : launch_table<64>(p, slots, ns, s); break;
    case 128: e = launch_adj<128>(p, s); if (e == cudaSuccess) e = tc ? launch_adjoint_table_tc(p, slots, ns, s) : launch_table<128>(p, slots, ns, s); break;
    case 256: e = launch_adj<256>(p, s); if (e == cudaSuccess) e = launch_table<256>(p, slots, ns, s); break;
    default: e = cudaErrorInvalidValue;
    }
    return e;
}

cudaError_t launch_adjoint_step_nu_mixed(const AdjointParams &p, int n_tiles, cudaStream_t s)
{
    if (n_tiles == 0) return cudaSuccess;
    if (p.n != 32) return cudaErrorInvalidValue;   // the variant exists for 4n = 128 only
    return launch_adj<128, true>(p, n_tiles, s);
}

cudaError_t launch_adjoint_table(const AdjointParams &p, double *slots, cudaStream_t s)
{
    const int ns = adjoint_table_slots();
    if (adjoint_table_tc_supported(p.n, p.n_phase)) return launch_adjoint_table_tc(p, slots, ns, s);
    switch (4 * p.n) {
    case 32: return launch_table<32>(p, slots, ns, s);
    case 64: return launch_table<64>(p, slots, ns, s);
    case 128: return launch_table<128>(p, slots, ns, s);
    case 256: return launch_table<256>(p, slots, ns, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_adjoint_seed_nu(float *nu, const float *dL_dout, const int *dir, int nx, int nz, int n, int bcbits,
                                   cudaStream_t s)
{
    k_adj_seed_nu<<<(nx * n + 255) / 256, 256, 0, s>>>(nu, reinterpret_cast<const float4 *>(dL_dout), dir, nx, nz, n,
                                                       bcbits);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_seed(float *lam, const float *dL_dout, const int *dir, int nx, int nz, int n, cudaStream_t s)
{
    k_adj_seed<<<(nx * n + 255) / 256, 256, 0, s>>>(lam, reinterpret_cast<const float4 *>(dL_dout), dir, nx, nz, n);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_chain(const double *ga, const double *gb, const float *tau, const float *alb, int nsites,
                                 int surv_mode, int abs_mode, float *g_tau, float *g_alb, cudaStream_t s)
{
    const int grid = std::min((nsites + 255) / 256, 148 * 32);
    k_adj_chain<<<grid, 256, 0, s>>>(ga, gb, tau, alb, nsites, surv_mode, abs_mode, g_tau, g_alb);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_fold(const double *slots, int nslots, size_t len, double *out, cudaStream_t s)
{
    const int grid = (int)std::min<size_t>((len + 255) / 256, 148 * 8);
    k_adj_fold_slots<<<grid, 256, 0, s>>>(slots, nslots, len, out);
    return cudaGetLastError();
}

}  // namespace rtlb
