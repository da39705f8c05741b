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
// read and one 16-byte write.  Used after a collision pass by the forms that
// do not gather while loading, by the adjoint (negated taps), and to form the
// state from a deferred P (readouts, residual).
#include "rtlb_internal.h"
#include "step_common.cuh"

namespace rtlb {
namespace {

constexpr int kStreamThreads = 256;

__global__ void __launch_bounds__(kStreamThreads)
    k_stream_bilinear(const float4 *__restrict__ P, float4 *__restrict__ S, const int *__restrict__ taps_o,
                      const float *__restrict__ taps_w, const float4 *__restrict__ inflow, int nx, int nz, int n,
                      int bcbits)
{
    const int d = blockIdx.y;
    const BilinearTaps t = load_taps(taps_o, taps_w, d);
    const size_t nsites = (size_t)nx * nz;
    const float4 *Pd = P + (size_t)d * nsites;
    float4 *Sd = S + (size_t)d * nsites;
    for (size_t site = (size_t)blockIdx.x * kStreamThreads + threadIdx.x; site < nsites;
         site += (size_t)gridDim.x * kStreamThreads) {
        const int z = (int)(site / nx), x = (int)(site - (size_t)z * nx);
        const float4 acc = gather_bilinear(t, Pd, inflow, bcbits, nx, nz, n, d, site, x, z);
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
