// Memory-bound helper kernels: layout conversion, per-site medium
// coefficients, float64 reductions (steady-state residual, total intensity)
// and boundary readout.  All loads and stores are 16-byte Stokes vectors.
#include <cfloat>
#include <cmath>

#include "rtlb_internal.h"

namespace rtlb {

namespace {

constexpr int kThreads = 256;

inline int grid_for(size_t work, int per_block = kThreads)
{
    size_t g = (work + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > 148u * 64u) g = 148u * 64u;
    return (int)g;
}

// user [site][d][4]  ->  direction-major [d][site][4]
// Layout conversion between the user's [site][d] and the direction-major
// [d][site] state (float4 entries): a transpose through shared memory in
// tiles of kXS sites x kXD directions, so that both the reads and the writes
// of global memory are contiguous runs.  The tile rows are padded by one
// float4 so that neither shared-memory phase has bank conflicts.
constexpr int kXS = 32, kXD = 64;

__global__ void __launch_bounds__(256) k_user_to_dm(const float4 *__restrict__ user, float4 *__restrict__ dm,
                                                    int nsites, int n)
{
    __shared__ float4 t[kXD][kXS + 1];
    const int s0 = blockIdx.x * kXS, d0 = blockIdx.y * kXD;
    const int ns = min(kXS, nsites - s0), nd = min(kXD, n - d0);
    // read: for each site, its nd directions are contiguous in the user layout
    for (int k = threadIdx.x; k < kXS * kXD; k += blockDim.x) {
        const int s = k / kXD, dd = k - s * kXD;
        if (s < ns && dd < nd) t[dd][s] = user[(size_t)(s0 + s) * n + d0 + dd];
    }
    __syncthreads();
    // write: for each direction, the tile's sites are contiguous
    for (int k = threadIdx.x; k < kXS * kXD; k += blockDim.x) {
        const int dd = k / kXS, s = k - dd * kXS;
        if (s < ns && dd < nd) dm[(size_t)(d0 + dd) * nsites + s0 + s] = t[dd][s];
    }
}

__global__ void __launch_bounds__(256) k_dm_to_user(const float4 *__restrict__ dm, float4 *__restrict__ user,
                                                    int nsites, int n)
{
    __shared__ float4 t[kXD][kXS + 1];
    const int s0 = blockIdx.x * kXS, d0 = blockIdx.y * kXD;
    const int ns = min(kXS, nsites - s0), nd = min(kXD, n - d0);
    for (int k = threadIdx.x; k < kXS * kXD; k += blockDim.x) {
        const int dd = k / kXS, s = k - dd * kXS;
        if (s < ns && dd < nd) t[dd][s] = dm[(size_t)(d0 + dd) * nsites + s0 + s];
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kXS * kXD; k += blockDim.x) {
        const int s = k / kXD, dd = k - s * kXD;
        if (s < ns && dd < nd) user[(size_t)(s0 + s) * n + d0 + dd] = t[dd][s];
    }
}

// Per-site step coefficients (emission e, absorption A, survival s):
//   P = alpha * (S + e) + beta * Z (S + e),  alpha = A s,  beta = A (1 - s)
// with A = exp(-(1-w) tau) or 1 - (1-w) tau and s = 1 - w tau or exp(-w tau).
// Evaluated once per medium in float64 and stored as float32; alpha, which
// multiplies the whole state every step, is kept as a hi + lo pair so that a
// uniform layer does not turn its rounding into a per-step bias.
__global__ void k_prep_medium(const float *__restrict__ tau, const float *__restrict__ albedo,
                              const float *__restrict__ emis, const uint8_t *__restrict__ cls_in,
                              float4 *__restrict__ coef, uint8_t *__restrict__ cls_out, int nsites,
                              int n_phase, int surv_mode, int abs_mode, int *__restrict__ flags)
{
    int bad = 0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nsites; j += gridDim.x * blockDim.x) {
        const float t = tau[j], w = albedo[j];
        const float e = emis ? emis[j] : 0.0f;
        const int c = cls_in ? (int)cls_in[j] : 0;
        if (!isfinite(t) || !isfinite(w) || !isfinite(e)) bad |= 1;
        if (!(t >= 0.0f) || !(w >= 0.0f) || !(w <= 1.0f) || !(e >= 0.0f)) bad |= 2;
        if (c >= n_phase) bad |= 4;
        const double kabs = (1.0 - (double)w) * (double)t, ksca = (double)w * (double)t;
        if (surv_mode == RTLB_SURV_LINEAR && ksca > 1.0) bad |= 2;
        if (abs_mode == RTLB_ABS_TAYLOR && kabs > 1.0) bad |= 2;
        const double A = (abs_mode == RTLB_ABS_TAYLOR) ? 1.0 - kabs : exp(-kabs);
        double s, one_minus_s;
        if (surv_mode == RTLB_SURV_LINEAR) {
            s = 1.0 - ksca;
            one_minus_s = ksca;
        } else {
            s = exp(-ksca);
            one_minus_s = -expm1(-ksca);
        }
        const double alpha = A * s;
        const float a_hi = (float)alpha;
        coef[j] = make_float4(a_hi, (float)(alpha - (double)a_hi), (float)(A * one_minus_s), e);
        cls_out[j] = (uint8_t)(c < n_phase ? c : 0);
    }
    if (bad) atomicOr(flags, bad);
}

__device__ __forceinline__ double warp_max(double v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Pass 1: per block max|b - a|, max|b| and a count of non-finite entries,
// accumulated in float64 (the difference of two floats is exact in double).
__global__ void k_residual_partial(const float4 *__restrict__ a, const float4 *__restrict__ b,
                                   size_t nvec, double *__restrict__ partials)
{
    double dmax = 0.0, vmax = 0.0, bad = 0.0;
    for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < nvec;
         j += (size_t)gridDim.x * blockDim.x) {
        const float4 x = a[j], y = b[j];
        const float yy[4] = {y.x, y.y, y.z, y.w}, xx[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (!isfinite(yy[k])) bad += 1.0;
            dmax = fmax(dmax, fabs((double)yy[k] - (double)xx[k]));
            vmax = fmax(vmax, fabs((double)yy[k]));
        }
    }
    __shared__ double sd[32], sv[32], sb[32];
    dmax = warp_max(dmax);
    vmax = warp_max(vmax);
    bad = warp_sum(bad);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sd[wid] = dmax;
        sv[wid] = vmax;
        sb[wid] = bad;
    }
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        dmax = lane < nw ? sd[lane] : 0.0;
        vmax = lane < nw ? sv[lane] : 0.0;
        bad = lane < nw ? sb[lane] : 0.0;
        dmax = warp_max(dmax);
        vmax = warp_max(vmax);
        bad = warp_sum(bad);
        if (lane == 0) {
            partials[3 * blockIdx.x + 0] = dmax;
            partials[3 * blockIdx.x + 1] = vmax;
            partials[3 * blockIdx.x + 2] = bad;
        }
    }
}

// Pass 2: one block folds the partials; out = {max|b-a|, max|b|, nonfinite}.
__global__ void k_residual_final(const double *__restrict__ partials, int nblocks,
                                 double *__restrict__ out)
{
    double dmax = 0.0, vmax = 0.0, bad = 0.0;
    for (int j = threadIdx.x; j < nblocks; j += blockDim.x) {
        dmax = fmax(dmax, partials[3 * j]);
        vmax = fmax(vmax, partials[3 * j + 1]);
        bad += partials[3 * j + 2];
    }
    __shared__ double sd[32], sv[32], sb[32];
    dmax = warp_max(dmax);
    vmax = warp_max(vmax);
    bad = warp_sum(bad);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sd[wid] = dmax;
        sv[wid] = vmax;
        sb[wid] = bad;
    }
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        dmax = lane < nw ? sd[lane] : 0.0;
        vmax = lane < nw ? sv[lane] : 0.0;
        bad = lane < nw ? sb[lane] : 0.0;
        dmax = warp_max(dmax);
        vmax = warp_max(vmax);
        bad = warp_sum(bad);
        if (lane == 0) {
            out[0] = dmax;
            out[1] = vmax;
            out[2] = bad;
        }
    }
}

// Sum of the I components in float64: per block partial sums, then one block
// adds them in a fixed order (deterministic).
__global__ void k_total_partial(const float4 *__restrict__ v, size_t nvec, double *__restrict__ partials)
{
    double acc = 0.0;
    for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < nvec;
         j += (size_t)gridDim.x * blockDim.x)
        acc += (double)v[j].x;
    __shared__ double sa[32];
    acc = warp_sum(acc);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sa[wid] = acc;
    __syncthreads();
    if (wid == 0) {
        acc = lane < (int)(blockDim.x >> 5) ? sa[lane] : 0.0;
        acc = warp_sum(acc);
        if (lane == 0) partials[blockIdx.x] = acc;
    }
}

__global__ void k_total_final(const double *__restrict__ partials, int nblocks, double *__restrict__ out)
{
    double acc = 0.0;
    for (int j = threadIdx.x; j < nblocks; j += blockDim.x) acc += partials[j];
    __shared__ double sa[32];
    acc = warp_sum(acc);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sa[wid] = acc;
    __syncthreads();
    if (wid == 0) {
        acc = lane < (int)(blockDim.x >> 5) ? sa[lane] : 0.0;
        acc = warp_sum(acc);
        if (lane == 0) out[0] = acc;
    }
}

// out[p][d] = state at the boundary row/column for directions leaving through
// `side`, zero otherwise.
__global__ void k_radiance_out(const float4 *__restrict__ dm, float4 *__restrict__ out, int nx,
                               int nz, int n, const int *__restrict__ dir, int side)
{
    const int len = (side == RTLB_SIDE_TOP || side == RTLB_SIDE_BOTTOM) ? nx : nz;
    const size_t nsites = (size_t)nx * nz;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < len * n; j += gridDim.x * blockDim.x) {
        const int p = j / n, d = j % n;
        const int cx = dir[d], cz = dir[n + d];
        int x, z;
        bool leaves;
        switch (side) {
        case RTLB_SIDE_TOP: x = p; z = nz - 1; leaves = cz == 1; break;
        case RTLB_SIDE_BOTTOM: x = p; z = 0; leaves = cz == -1; break;
        case RTLB_SIDE_LEFT: x = 0; z = p; leaves = cx == -1; break;
        default: x = nx - 1; z = p; leaves = cx == 1; break;
        }
        out[j] = leaves ? dm[(size_t)d * nsites + (size_t)z * nx + x] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// Degree of polarization (Sec. 3.2.1, Eq. 36: sqrt(Q^2 + U^2 + V^2) / I) of
// the radiance leaving through `side`, out[p][d]; zero for directions that
// do not leave through it and where I <= 0.  Evaluated in float64 from the
// float32 Stokes vector, rounded once.
__global__ void k_dop_out(const float4 *__restrict__ dm, float *__restrict__ out, int nx, int nz, int n,
                          const int *__restrict__ dir, int side)
{
    const int len = (side == RTLB_SIDE_TOP || side == RTLB_SIDE_BOTTOM) ? nx : nz;
    const size_t nsites = (size_t)nx * nz;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < len * n; j += gridDim.x * blockDim.x) {
        const int p = j / n, d = j % n;
        const int cx = dir[d], cz = dir[n + d];
        int x, z;
        bool leaves;
        switch (side) {
        case RTLB_SIDE_TOP: x = p; z = nz - 1; leaves = cz == 1; break;
        case RTLB_SIDE_BOTTOM: x = p; z = 0; leaves = cz == -1; break;
        case RTLB_SIDE_LEFT: x = 0; z = p; leaves = cx == -1; break;
        default: x = nx - 1; z = p; leaves = cx == 1; break;
        }
        float v = 0.f;
        if (leaves) {
            const float4 st = dm[(size_t)d * nsites + (size_t)z * nx + x];
            if (st.x > 0.f) {
                const double q = st.y, u = st.z, w = st.w;
                v = (float)(sqrt(q * q + u * u + w * w) / (double)st.x);
            }
        }
        out[j] = v;
    }
}

__global__ void k_fill(float *p, size_t count, float v)
{
    for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < count;
         j += (size_t)gridDim.x * blockDim.x)
        p[j] = v;
}

}  // namespace

cudaError_t launch_user_to_dm(const float *user, float *dm, int nsites, int n, cudaStream_t s)
{
    const dim3 grid((nsites + kXS - 1) / kXS, (n + kXD - 1) / kXD);
    k_user_to_dm<<<grid, 256, 0, s>>>(reinterpret_cast<const float4 *>(user), reinterpret_cast<float4 *>(dm), nsites, n);
    return cudaGetLastError();
}

cudaError_t launch_dm_to_user(const float *dm, float *user, int nsites, int n, cudaStream_t s)
{
    const dim3 grid((nsites + kXS - 1) / kXS, (n + kXD - 1) / kXD);
    k_dm_to_user<<<grid, 256, 0, s>>>(reinterpret_cast<const float4 *>(dm), reinterpret_cast<float4 *>(user), nsites, n);
    return cudaGetLastError();
}

cudaError_t launch_prep_medium(const float *tau, const float *albedo, const float *emis,
                               const uint8_t *cls_in, float4 *coef, uint8_t *cls_out, int nsites,
                               int n_phase, int surv_mode, int abs_mode, int *flags, cudaStream_t s)
{
    k_prep_medium<<<grid_for(nsites), kThreads, 0, s>>>(tau, albedo, emis, cls_in, coef, cls_out, nsites,
                                                        n_phase, surv_mode, abs_mode, flags);
    return cudaGetLastError();
}

int residual_blocks(size_t count)
{
    const size_t nvec = count / 4;
    int g = grid_for(nvec);
    return g > 148 * 8 ? 148 * 8 : g;
}

cudaError_t launch_residual(const float *a, const float *b, size_t count, double *partials,
                            int nblocks, double *out3, cudaStream_t s)
{
    k_residual_partial<<<nblocks, kThreads, 0, s>>>(reinterpret_cast<const float4 *>(a),
                                                    reinterpret_cast<const float4 *>(b), count / 4,
                                                    partials);
    k_residual_final<<<1, kThreads, 0, s>>>(partials, nblocks, out3);
    return cudaGetLastError();
}

cudaError_t launch_total_I(const float *dm, size_t nvec, double *partials, int nblocks,
                           double *out, cudaStream_t s)
{
    k_total_partial<<<nblocks, kThreads, 0, s>>>(reinterpret_cast<const float4 *>(dm), nvec, partials);
    k_total_final<<<1, kThreads, 0, s>>>(partials, nblocks, out);
    return cudaGetLastError();
}

cudaError_t launch_radiance_out(const float *dm, float *out, int nx, int nz, int n,
                                const int *dir, int side, cudaStream_t s)
{
    const int len = (side == RTLB_SIDE_TOP || side == RTLB_SIDE_BOTTOM) ? nx : nz;
    k_radiance_out<<<grid_for((size_t)len * n), kThreads, 0, s>>>(
        reinterpret_cast<const float4 *>(dm), reinterpret_cast<float4 *>(out), nx, nz, n, dir, side);
    return cudaGetLastError();
}

cudaError_t launch_dop_out(const float *dm, float *out, int nx, int nz, int n, const int *dir, int side,
                           cudaStream_t s)
{
    const int len = (side == RTLB_SIDE_TOP || side == RTLB_SIDE_BOTTOM) ? nx : nz;
    k_dop_out<<<grid_for((size_t)len * n), kThreads, 0, s>>>(reinterpret_cast<const float4 *>(dm), out, nx, nz, n,
                                                             dir, side);
    return cudaGetLastError();
}

cudaError_t launch_fill(float *p, size_t count, float v, cudaStream_t s)
{
    k_fill<<<grid_for(count), kThreads, 0, s>>>(p, count, v);
    return cudaGetLastError();
}

}  // namespace rtlb
