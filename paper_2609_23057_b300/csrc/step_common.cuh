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

// ---- semi-Lagrangian bilinear streaming (Eq. 33-38), the gather form ----
//
// The field arriving at (x, z) along direction d is the weighted sum of the
// post-collision field P at four sources (x - ox_k, z - oz_k); the taps of
// direction d are ox[8d..8d+3], oz[8d+4..8d+7] (int) and w[4d..4d+3] (float).
// The adjoint passes the negated taps.  The two-pass step (a
// collision pass, then k_stream_bilinear) and the kernels that gather while
// loading their operand evaluate the same sum in the same order (k = 0..3,
// zero weights skipped), so both forms give identical bits.

struct BilinearTaps {
    int ox[4], oz[4];
    float w[4];
    int xmin, xmax, zmin, zmax;   // the sources span [x - xmax, x - xmin] x [z - zmax, z - zmin]
};

// Taps of direction d from global memory (LDG) or from a copy in shared
// memory (SMEM = true).
template <bool SMEM = false>
__device__ __forceinline__ BilinearTaps load_taps(const int *__restrict__ taps_o, const float *__restrict__ taps_w,
                                                  int d)
{
    BilinearTaps t;
    const int4 *o4 = reinterpret_cast<const int4 *>(taps_o + 8 * d);
    const float4 *w4 = reinterpret_cast<const float4 *>(taps_w + 4 * d);
    const int4 a = SMEM ? o4[0] : __ldg(o4);
    const int4 b = SMEM ? o4[1] : __ldg(o4 + 1);
    const float4 w = SMEM ? *w4 : __ldg(w4);
    t.ox[0] = a.x, t.ox[1] = a.y, t.ox[2] = a.z, t.ox[3] = a.w;
    t.oz[0] = b.x, t.oz[1] = b.y, t.oz[2] = b.z, t.oz[3] = b.w;
    t.w[0] = w.x, t.w[1] = w.y, t.w[2] = w.z, t.w[3] = w.w;
    t.xmin = t.xmax = t.ox[0];
    t.zmin = t.zmax = t.oz[0];
#pragma unroll
    for (int k = 1; k < 4; ++k) {
        t.xmin = min(t.xmin, t.ox[k]);
        t.xmax = max(t.xmax, t.ox[k]);
        t.zmin = min(t.zmin, t.oz[k]);
        t.zmax = max(t.zmax, t.oz[k]);
    }
    return t;
}

__device__ __forceinline__ int wrap_mod(int v, int n) { return ((v % n) + n) % n; }

__device__ __forceinline__ void axpy4(float4 &acc, float w, float4 v)
{
    acc.x = fmaf(w, v.x, acc.x);
    acc.y = fmaf(w, v.y, acc.y);
    acc.z = fmaf(w, v.z, acc.z);
    acc.w = fmaf(w, v.w, acc.w);
}

// Value of source (xs, zs) of direction d after periodic wrapping: the site
// itself, or the ghost of the side it lies beyond (ghost corners belong to the
// top / bottom side).  Taps reach up to two cells away, so lattices of one or
// two cells wrap more than once.
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

// Whether every tap of (x, z) lies inside the lattice.
__device__ __forceinline__ bool taps_inside(const BilinearTaps &t, int nx, int nz, int x, int z)
{
    return x - t.xmax >= 0 && x - t.xmin < nx && z - t.zmax >= 0 && z - t.zmin < nz;
}

// The gathered field of (site, d) read from P's direction plane Pd.
__device__ __forceinline__ float4 gather_bilinear(const BilinearTaps &t, const float4 *__restrict__ Pd,
                                                  const float4 *__restrict__ inflow, int bcbits, int nx, int nz, int n,
                                                  int d, size_t site, int x, int z)
{
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    if (taps_inside(t, nx, nz, x, z)) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (t.w[k] != 0.f) axpy4(acc, t.w[k], __ldg(Pd + (ptrdiff_t)site - t.ox[k] - (ptrdiff_t)t.oz[k] * nx));
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (t.w[k] != 0.f) axpy4(acc, t.w[k], source_or_ghost(Pd, inflow, bcbits, nx, nz, n, d, x - t.ox[k], z - t.oz[k]));
    }
    return acc;
}

}  // namespace rtlb
