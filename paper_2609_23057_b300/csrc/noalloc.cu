// Steady-state residual over two caller buffers, with no allocation at all.
//
// Who needs this: code that runs where cudaMalloc is off limits -- inside a
// host callback or a custom allocator hook, in a process whose memory pool is
// owned and capped by another framework, or in a real-time loop that must not
// touch the driver's allocator -- but still wants the float64 residual
// max|S_new - S_old| / max|S_new| that rtlb_run_to_steady uses.  The regular
// path keeps its per-block partial results in a buffer the context allocates;
// this variant keeps them in a fixed array compiled into the library instead.
//
// Scratch: g_noalloc_partials, 3 doubles per block for at most kMaxBlocks
// blocks (1.5 MiB).  Every GPU that loads the library holds it until the
// process exits.  Each block covers a fixed chunk of kChunkVec Stokes vectors,
// so at most kMaxBlocks * kChunkVec * 4 = 2^30 floats fit in one call.
//
// Host code cannot use the array's name as a device address (it is a
// host-side stand-in); the first call in each CUDA context (one per device in
// the usual runtime use), with that device current, looks the address up
// with cudaGetSymbolAddress and caches it under the context.  A device reset
// creates a new context, so the next call looks the address up again instead
// of reusing one from the freed context.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <mutex>

#include "rtlb_internal.h"

namespace {

constexpr size_t kChunkVec = 4096;  // float4 vectors per block
constexpr int kMaxBlocks = 65536;
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_partials[3 * kMaxBlocks];

std::mutex g_mutex;
struct CachedAddress {
    CUcontext ctx = nullptr;
    double *addr = nullptr;
};
CachedAddress g_partials_addr[kMaxDevices];

__device__ __forceinline__ double wmax(double v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double wsum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block j reduces vectors [j * kChunkVec, (j + 1) * kChunkVec) and overwrites
// its own three partial slots (nothing is accumulated across calls).
__global__ void k_residual_chunks(const float4 *__restrict__ a, const float4 *__restrict__ b,
                                  size_t nvec, double *__restrict__ partials)
{
    const size_t lo = (size_t)blockIdx.x * kChunkVec;
    const size_t hi = lo + kChunkVec < nvec ? lo + kChunkVec : nvec;
    double dmax = 0.0, vmax = 0.0, bad = 0.0;
    for (size_t j = lo + threadIdx.x; j < hi; j += blockDim.x) {
        const float4 x = a[j], y = b[j];
        const float xs[4] = {x.x, x.y, x.z, x.w}, ys[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (!isfinite(ys[k])) bad += 1.0;
            dmax = fmax(dmax, fabs((double)ys[k] - (double)xs[k]));
            vmax = fmax(vmax, fabs((double)ys[k]));
        }
    }
    __shared__ double s[3][kThreads / 32];
    dmax = wmax(dmax);
    vmax = wmax(vmax);
    bad = wsum(bad);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        s[0][w] = dmax;
        s[1][w] = vmax;
        s[2][w] = bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < kThreads / 32; ++k) {
            dmax = fmax(dmax, s[0][k]);
            vmax = fmax(vmax, s[1][k]);
            bad += s[2][k];
        }
        partials[3 * blockIdx.x + 0] = dmax;
        partials[3 * blockIdx.x + 1] = vmax;
        partials[3 * blockIdx.x + 2] = bad;
    }
}

__global__ void k_residual_fold(const double *__restrict__ partials, int nblocks, double *__restrict__ out)
{
    double dmax = 0.0, vmax = 0.0, bad = 0.0;
    for (int j = threadIdx.x; j < nblocks; j += blockDim.x) {
        dmax = fmax(dmax, partials[3 * j]);
        vmax = fmax(vmax, partials[3 * j + 1]);
        bad += partials[3 * j + 2];
    }
    __shared__ double s[3][kThreads / 32];
    dmax = wmax(dmax);
    vmax = wmax(vmax);
    bad = wsum(bad);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        s[0][w] = dmax;
        s[1][w] = vmax;
        s[2][w] = bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < kThreads / 32; ++k) {
            dmax = fmax(dmax, s[0][k]);
            vmax = fmax(vmax, s[1][k]);
            bad += s[2][k];
        }
        out[0] = dmax;
        out[1] = vmax;
        out[2] = bad;
    }
}

// The driver's cuCtxGetCurrent, through the runtime's entry-point query (the
// library links only the runtime).
PFN_cuCtxGetCurrent_v4000 ctx_get_current()
{
    static PFN_cuCtxGetCurrent_v4000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void *ptr = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &ptr, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(ptr);
    }
    return fn;
}

// Device address of the fixed scratch array in the current device's current
// context, looked up once per context.
rtlb_status partials_address(double **addr)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return RTLB_E_CUDA;
    }
    auto get_ctx = ctx_get_current();
    CUcontext ctx = nullptr;
    if (!get_ctx || get_ctx(&ctx) != CUDA_SUCCESS || !ctx) return RTLB_E_CUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    CachedAddress &c = g_partials_addr[dev];
    if (c.ctx != ctx || !c.addr) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || !p) {
            cudaGetLastError();
            return RTLB_E_CUDA;
        }
        c.ctx = ctx;
        c.addr = static_cast<double *>(p);
    }
    *addr = c.addr;
    return RTLB_OK;
}

// True when p is device (or managed) memory of the current device: a host
// pointer handed to the kernels would be read as a device address.
bool on_current_device(const void *p)
{
    int dev = 0;
    cudaPointerAttributes a;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace

extern "C" rtlb_status rtlb_residual_noalloc(const float *S_old, const float *S_new, size_t count,
                                             double *out, void *stream)
{
    if (!S_old || !S_new || !out) return RTLB_E_ARG;
    if (count % 4 != 0 || (reinterpret_cast<uintptr_t>(S_old) & 15u) || (reinterpret_cast<uintptr_t>(S_new) & 15u) ||
        (reinterpret_cast<uintptr_t>(out) & 7u))
        return RTLB_E_ARG;
    if (count > RTLB_NOALLOC_MAX_COUNT) return RTLB_E_SHAPE;
    if (!on_current_device(S_old) || !on_current_device(S_new) || !on_current_device(out)) return RTLB_E_ARG;
    double *partials = nullptr;
    const rtlb_status st = partials_address(&partials);
    if (st != RTLB_OK) return st;
    const size_t nvec = count / 4;
    const int nblocks = (int)((nvec + kChunkVec - 1) / kChunkVec);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (nblocks > 0)
        k_residual_chunks<<<nblocks, kThreads, 0, s>>>(reinterpret_cast<const float4 *>(S_old),
                                                       reinterpret_cast<const float4 *>(S_new), nvec, partials);
    k_residual_fold<<<1, kThreads, 0, s>>>(partials, nblocks, out);
    return cudaGetLastError() == cudaSuccess ? RTLB_OK : RTLB_E_CUDA;
}
