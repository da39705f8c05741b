// Streaming part of the fused step, shared by the CUDA-core and tensor-core
// kernels: where a post-collision Stokes vector goes (push along the
// direction's D2Q9 offset, periodic wrap) and which entries take a ghost value
// (upstream cell outside a non-periodic side: zero for vacuum, the side's
// inflow vector for inflow; ghost corners belong to the top/bottom side).
#pragma once
#include "rtlb_internal.h"

namespace rtlb {

__device__ __forceinline__ int wrap_coord(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Stores the post-collision vector v of (site, d) at its streaming target and,
// when (site, d) itself is fed from a ghost cell, writes that ghost value.
// Boundary kinds packed two bits per side (top, bottom, left, right).
__host__ __device__ __forceinline__ int pack_bc(const int bc[4])
{
    return bc[0] | (bc[1] << 2) | (bc[2] << 4) | (bc[3] << 6);
}
__device__ __forceinline__ int bc_of(int bcbits, int side) { return (bcbits >> (2 * side)) & 3; }

// The push of one post-collision Stokes vector of site (x, z) along
// direction d (with the site's coordinates already known).
__device__ __forceinline__ void push_store_xz(const int *__restrict__ dir, const float *__restrict__ inflow,
                                              int bcbits, float *__restrict__ S_new, int nx, int nz,
                                              int n, int site, int x, int z, int d, float4 v)
{
    const size_t nsites = (size_t)nx * nz;
    const int cx = dir[d], cz = dir[n + d];
    const bool per_x = bc_of(bcbits, RTLB_SIDE_LEFT) == RTLB_BC_PERIODIC;
    const bool per_z = bc_of(bcbits, RTLB_SIDE_TOP) == RTLB_BC_PERIODIC;
    float4 *out = reinterpret_cast<float4 *>(S_new) + (size_t)d * nsites;
    int xt = x + cx, zt = z + cz;
    if (per_x) xt = wrap_coord(xt, nx);
    if (per_z) zt = wrap_coord(zt, nz);
    if (xt >= 0 && xt < nx && zt >= 0 && zt < nz) out[(size_t)zt * nx + xt] = v;
    int xs = x - cx, zs = z - cz;
    if (per_x) xs = wrap_coord(xs, nx);
    if (per_z) zs = wrap_coord(zs, nz);
    int side = -1;
    if (zs >= nz) side = RTLB_SIDE_TOP;
    else if (zs < 0) side = RTLB_SIDE_BOTTOM;
    else if (xs < 0) side = RTLB_SIDE_LEFT;
    else if (xs >= nx) side = RTLB_SIDE_RIGHT;
    if (side >= 0) {
        float4 gv = make_float4(0.f, 0.f, 0.f, 0.f);
        if (bc_of(bcbits, side) == RTLB_BC_INFLOW) gv = reinterpret_cast<const float4 *>(inflow)[side * n + d];
        out[site] = gv;
    }
}

__device__ __forceinline__ void push_store(const int *__restrict__ dir, const float *__restrict__ inflow,
                                           int bcbits, float *__restrict__ S_new, int nx, int nz,
                                           int n, int site, int d, float4 v)
{
    const int z = site / nx, x = site - z * nx;
    push_store_xz(dir, inflow, bcbits, S_new, nx, nz, n, site, x, z, d, v);
}

}  // namespace rtlb
