// Semi-Lagrangian bilinear streaming (Eq. 33-38): the field arriving at a
// site is a weighted sum of four integer translations of the post-collision
// field, with weights (1 - f_x, f_x) x (1 - f_z, f_z) fixed per direction.
//
// Layout: direction-major [d][site][4] float32, site = z * nx + x.  One block
// row (blockIdx.y) per direction, so the taps are uniform across the block;
// consecutive threads take consecutive sites, so the four taps of a warp are
// four contiguous 512-byte runs (two of them one row apart): the x-neighbour
// tap hits L1 and the row above or below hits L2 while the neighbouring row's
// blocks are still running.  HBM traffic per site and direction is one 16-byte
// read and one 16-byte write.
#include "rtlb_internal.h"
#include "step_common.cuh"

namespace rtlb {
namespace {

constexpr int kStreamThreads = 256;

__device__ __forceinline__ int wrap_mod(int v, int n) { return ((v % n) + n) % n; }

// Value of (xs, zs) after periodic wrapping: the site itself, or the ghost of
// the side it lies beyond (ghost corners belong to the top / bottom side).
// Taps reach up to two cells away, so lattices of one or two cells wrap more
// than once.
__device__ __forceinline__ float4 source_or_ghost(const float4 *__restrict__ Pd, const float4 *__restrict__ inflow,
                                                  int bcbits, int nx, int nz, int n, int d, int xs, int zs)
{
    if (bc_of(bcbits, RTLB_SIDE_LEFT) == RTLB_BC_PERIODIC) xs = wrap_mod(xs, nx);
    if (bc_of(bcbits, RTLB_SIDE_TOP) == RTLB_BC_PERIODIC) zs = wrap_mod(zs, nz);
    int side = -1;
    if (zs >= nz) side = RTLB_SIDE_TOP;
    else if (zs < 0) side = RTLB_SIDE_BOTTOM;
    else if (xs < 0) side = RTLB_SIDE_LEFT;
    else if (xs >= nx) side = RTLB_SIDE_RIGHT;
    if (side < 0) return __ldg(Pd + (size_t)zs * nx + xs);
    if (bc_of(bcbits, side) == RTLB_BC_INFLOW) return __ldg(inflow + side * n + d);
    return make_float4(0.f, 0.f, 0.f, 0.f);
}

__device__ __forceinline__ void axpy4(float4 &acc, float w, float4 v)
{
    acc.x = fmaf(w, v.x, acc.x);
    acc.y = fmaf(w, v.y, acc.y);
    acc.z = fmaf(w, v.z, acc.z);
    acc.w = fmaf(w, v.w, acc.w);
}

__global__ void __launch_bounds__(kStreamThreads)
    k_stream_bilinear(const float4 *__restrict__ P, float4 *__restrict__ S, const int *__restrict__ taps_o,
                      const float *__restrict__ taps_w, const float4 *__restrict__ inflow, int nx, int nz, int n,
                      int bcbits)
{
    const int d = blockIdx.y;
    int ox[4], oz[4];
    float w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        ox[k] = taps_o[8 * d + k];
        oz[k] = taps_o[8 * d + 4 + k];
        w[k] = taps_w[4 * d + k];
    }
    // the taps span [x - xmax, x - xmin] x [z - zmax, z - zmin]
    int xmin = ox[0], xmax = ox[0], zmin = oz[0], zmax = oz[0];
#pragma unroll
    for (int k = 1; k < 4; ++k) {
        xmin = min(xmin, ox[k]);
        xmax = max(xmax, ox[k]);
        zmin = min(zmin, oz[k]);
        zmax = max(zmax, oz[k]);
    }
    const size_t nsites = (size_t)nx * nz;
    const float4 *Pd = P + (size_t)d * nsites;
    float4 *Sd = S + (size_t)d * nsites;
    for (size_t site = (size_t)blockIdx.x * kStreamThreads + threadIdx.x; site < nsites;
         site += (size_t)gridDim.x * kStreamThreads) {
        const int z = (int)(site / nx), x = (int)(site - (size_t)z * nx);
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        if (x - xmax >= 0 && x - xmin < nx && z - zmax >= 0 && z - zmin < nz) {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (w[k] != 0.f) axpy4(acc, w[k], __ldg(Pd + (ptrdiff_t)site - ox[k] - (ptrdiff_t)oz[k] * nx));
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (w[k] != 0.f)
                    axpy4(acc, w[k], source_or_ghost(Pd, inflow, bcbits, nx, nz, n, d, x - ox[k], z - oz[k]));
        }
        __stcs(Sd + site, acc);
    }
}

}  // namespace

cudaError_t launch_stream_bilinear(const float *P, float *S, const int *taps_o, const float *taps_w,
                                   const float *inflow, int nx, int nz, int n, int bcbits, cudaStream_t s)
{
    const size_t nsites = (size_t)nx * nz;
    const size_t blocks = (nsites + kStreamThreads - 1) / kStreamThreads;
    const dim3 grid((unsigned)std::min<size_t>(blocks, 1u << 20), (unsigned)n);
    k_stream_bilinear<<<grid, kStreamThreads, 0, s>>>(reinterpret_cast<const float4 *>(P),
                                                      reinterpret_cast<float4 *>(S), taps_o, taps_w,
                                                      reinterpret_cast<const float4 *>(inflow), nx, nz, n, bcbits);
    return cudaGetLastError();
}

}  // namespace rtlb
