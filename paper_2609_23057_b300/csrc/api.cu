// C-ABI entry points of librtlb (declared in include/rtlb.h).
//
// A context owns: the direction set and streaming offsets, the boundary
// description, the per-site step coefficients and phase tables of the current
// medium, and two direction-major state buffers [d][site][4] that alternate
// every step (the new state is written by push streaming from the old one).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <new>

#include "rtlb_internal.h"
#include "step_common.cuh"
#include "tc.h"

using namespace rtlb;

// Order of the two reverse-sweep kernels of a step in the transposed-stream
// form: 1 = table gradient first (it reads the reverse step's inputs only).
// Measured with the table kernel's loads at normal L2 priority, 300 steps of
// the 1024 x 256, n = 32 adjoint with every state kept: 73.4 ms first, 74.0 ms
// after (74.5 ms after with evict-first loads).
#ifndef RTLB_ADJ_TABLE_FIRST
#define RTLB_ADJ_TABLE_FIRST 1
#endif

namespace rtlb {

cudaError_t DevBuf::ensure(size_t bytes)
{
    if (bytes <= cap) return cudaSuccess;
    release();
    const cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        p = nullptr;
        return e;
    }
    cap = bytes;
    return cudaSuccess;
}

void DevBuf::release()
{
    cudaFree(p);
    p = nullptr;
    cap = 0;
}

}  // namespace rtlb

namespace {

rtlb_status fail(rtlb_ctx *ctx, rtlb_status st, const char *fmt, ...)
{
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return st;
}

rtlb_status cuda_fail(rtlb_ctx *ctx, cudaError_t e, const char *what)
{
    return fail(ctx, e == cudaErrorMemoryAllocation ? RTLB_E_OOM : RTLB_E_CUDA, "%s: %s (%s)", what,
                cudaGetErrorName(e), cudaGetErrorString(e));
}

#define CK(ctx, call, what)                                        \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, (what)); \
    } while (0)

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

inline cudaStream_t S(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// Direction set, and per direction its streaming description: for NEAREST8
// the D2Q9 offset (cx, cz) and a single unit tap; for BILINEAR the four taps of
// Eq. 34 and, in (cx, cz), the sign of each displacement component (the sense
// of motion, used by the boundary readout and the adjoint seed).
rtlb_status build_dirs(const rtlb_directions *dirs, int streaming, int plane, std::vector<double> &mu,
                       std::vector<double> &phi, std::vector<int> &cx, std::vector<int> &cz,
                       std::vector<int> &tap_o, std::vector<double> &tap_w, rtlb_ctx *ctx)
{
    if (!dirs) return fail(ctx, RTLB_E_ARG, "directions is NULL");
    if (streaming != RTLB_STREAM_NEAREST8 && streaming != RTLB_STREAM_BILINEAR)
        return fail(ctx, RTLB_E_ARG, "unknown streaming scheme %d", streaming);
    if (plane != RTLB_PLANE_XZ && plane != RTLB_PLANE_XY) return fail(ctx, RTLB_E_ARG, "unknown lattice plane %d", plane);
    if (dirs->n_zen < 1 || dirs->n_az < 1 || (int64_t)dirs->n_zen * dirs->n_az > kMaxDirs)
        return fail(ctx, RTLB_E_SHAPE, "need 1 <= n_zen*n_az <= %d (got %d x %d)", kMaxDirs, dirs->n_zen,
                    dirs->n_az);
    const int n = dirs->n_zen * dirs->n_az;
    if ((dirs->mu == nullptr) != (dirs->phi == nullptr))
        return fail(ctx, RTLB_E_ARG, "mu and phi must both be given or both be NULL");
    if (dirs->mu) {
        mu.assign(dirs->mu, dirs->mu + n);
        phi.assign(dirs->phi, dirs->phi + n);
        for (int d = 0; d < n; ++d)
            if (!std::isfinite(mu[d]) || !std::isfinite(phi[d]) || mu[d] < -1.0 || mu[d] > 1.0)
                return fail(ctx, RTLB_E_RANGE, "direction %d: mu must be in [-1, 1] and finite", d);
    } else {
        direction_grid(dirs->n_zen, dirs->n_az, mu, phi);
    }
    cx.assign(n, 0);
    cz.assign(n, 0);
    tap_o.assign((size_t)8 * n, 0);
    tap_w.assign((size_t)4 * n, 0.0);
    for (int d = 0; d < n; ++d) {
        if (streaming == RTLB_STREAM_NEAREST8) {
            if (stream_offset(mu[d], phi[d], plane, &cx[d], &cz[d]))
                return fail(ctx, RTLB_E_AMBIGUOUS_STREAM,
                            "direction %d (mu=%.17g, phi=%.17g) lies between two lattice offsets", d, mu[d],
                            phi[d]);
            tap_o[8 * d] = cx[d];
            tap_o[8 * d + 4] = cz[d];
            tap_w[4 * d] = 1.0;
        } else {
            int sense[2];
            bilinear_taps(mu[d], phi[d], plane, &tap_o[8 * d], &tap_o[8 * d + 4], &tap_w[4 * d], sense);
            cx[d] = sense[0];
            cz[d] = sense[1];
        }
    }
    return RTLB_OK;
}

bool bilinear(const rtlb_ctx *c) { return c->opt.streaming == RTLB_STREAM_BILINEAR; }

void free_ctx_buffers(rtlb_ctx *c)
{
    cudaFree(c->S[0]);
    cudaFree(c->S[1]);
    cudaFree(c->d_dir);
    cudaFree(c->d_dir0);
    cudaFree(c->d_tap_o);
    cudaFree(c->d_tap_w);
    cudaFree(c->d_post);
    cudaFree(c->d_inflow);
    cudaFree(c->d_coef);
    cudaFree(c->d_cls);
    cudaFree(c->d_ZT);
    cudaFree(c->d_Z);
    cudaFree(c->d_tau);
    cudaFree(c->d_alb);
    cudaFree(c->d_scratch);
    cudaFree(c->d_out);
    cudaFree(c->d_flags);
    cudaFree(c->d_stage);
    cudaFree(c->d_rad);
    cudaFreeHost(c->h_out);
    cudaFreeHost(c->h_flags);
    c->adj.release();
    c->adj_tc.release();
    tc_release(c);
}


rtlb_status require_boundary_pairs(rtlb_ctx *c)
{
    if ((c->bc[RTLB_SIDE_TOP] == RTLB_BC_PERIODIC) != (c->bc[RTLB_SIDE_BOTTOM] == RTLB_BC_PERIODIC) ||
        (c->bc[RTLB_SIDE_LEFT] == RTLB_BC_PERIODIC) != (c->bc[RTLB_SIDE_RIGHT] == RTLB_BC_PERIODIC))
        return fail(c, RTLB_E_STATE, "periodic boundaries must be set on both sides of an axis");
    return RTLB_OK;
}

rtlb_status ensure_stage(rtlb_ctx *c)
{
    if (!c->d_stage) CK(c, cudaMalloc(&c->d_stage, c->state_floats() * sizeof(float)), "staging buffer");
    return RTLB_OK;
}

rtlb_status ensure_post(rtlb_ctx *c)
{
    if (!c->d_post) CK(c, cudaMalloc(&c->d_post, c->state_floats() * sizeof(float)), "post-collision buffer");
    return RTLB_OK;
}

StepParams make_params(rtlb_ctx *c)
{
    StepParams p;
    p.S = c->S[c->cur];
    p.S_new = c->S[c->cur ^ 1];
    p.coef = c->d_coef;
    p.cls = c->d_cls;
    p.ZT = c->d_ZT;
    p.dir = c->d_dir;
    p.inflow = c->d_inflow;
    p.nx = c->nx;
    p.nz = c->nz;
    p.n = c->n;
    p.n_phase = c->n_phase;
    for (int k = 0; k < 4; ++k) p.bc[k] = c->bc[k];
    return p;
}

// Bilinear streaming in the gather form: the tensor-core bf16 steps (where
// tc_gather: n in {16, 32}, nx % 128 == 0) gather the four taps of the
// previous step's P while loading their operand, so a run of steps moves the
// state once per step instead of twice (collision pass, then
// k_stream_bilinear).  Measured at 2048^2: 1.34 against 1.69 ms per step at
// n = 32 (bf16), 0.67 against 0.83 ms at n = 16.  The float32 step keeps the
// two passes (gathering in its tile load measured slower: 1.43 against 1.30 ms
// at 1024^2, n = 32; 4.21 against 3.80 ms at n = 64), and so do the n = 64
// tensor-core forms, whose two staging slots cannot hide the windows' latency
// (4.16 against 3.29 ms).
bool gather_form(const rtlb_ctx *c)
{
    return bilinear(c) && c->opt.precision != RTLB_PREC_FP32 && tc_gather(c);
}

cudaError_t gather_into(rtlb_ctx *c, const float *P, float *out, cudaStream_t s)
{
    return launch_stream_bilinear(P, out, c->d_tap_o, c->d_tap_w, c->d_inflow, c->nx, c->nz, c->n, pack_bc(c->bc), s);
}

// The current state S^t: S[cur], or (streaming deferred) the gather of the
// P in S[cur], formed in d_post once per step taken.
rtlb_status state_view(rtlb_ctx *c, cudaStream_t s, const float **out)
{
    if (!c->deferred) {
        *out = c->S[c->cur];
        return RTLB_OK;
    }
    if (!c->view_valid) {
        CK(c, gather_into(c, c->S[c->cur], c->d_post, s), "deferred streaming");
        c->view_valid = true;
    }
    *out = c->d_post;
    return RTLB_OK;
}

// Ends a deferral: S[cur] (and with `prev`, S[cur ^ 1]) then hold states, not
// P; the gathered buffer and the one that held P swap roles.
rtlb_status settle(rtlb_ctx *c, cudaStream_t s, bool prev)
{
    if (c->deferred) {
        const float *v = nullptr;
        const rtlb_status st = state_view(c, s, &v);
        if (st != RTLB_OK) return st;
        std::swap(c->S[c->cur], c->d_post);
        c->deferred = false;
        c->view_valid = false;
    }
    if (prev && c->prev_deferred) {
        const rtlb_status st = ensure_stage(c);
        if (st != RTLB_OK) return st;
        CK(c, gather_into(c, c->S[c->cur ^ 1], c->d_stage, s), "deferred streaming");
        std::swap(c->S[c->cur ^ 1], c->d_stage);
        c->prev_deferred = false;
    }
    return RTLB_OK;
}

// One float32-accurate step from S_in into S_out for the adjoint's forward
// pass and replays: the 3xTF32 tensor-core step when that is the context's
// precision (same accuracy, a third of the time), the CUDA-core float32 step
// otherwise.
cudaError_t fp32_step_into(rtlb_ctx *c, const float *S_in, float *S_out, cudaStream_t s)
{
    StepParams p = make_params(c);
    p.S = S_in;
    p.S_new = S_out;
    const bool tf32 = c->opt.precision == RTLB_PREC_TF32X3;
    auto collide = [&](const StepParams &q) -> cudaError_t {
        if (!tf32) return launch_step_fp32(q, s);
        return tc_step(c, q, s) == RTLB_OK ? cudaSuccess : cudaErrorLaunchFailure;
    };
    if (!bilinear(c)) return collide(p);
    p.dir = c->d_dir0;
    p.S_new = c->d_post;
    cudaError_t e = collide(p);
    if (e != cudaSuccess) return e;
    return launch_stream_bilinear(c->d_post, S_out, c->d_tap_o, c->d_tap_w, c->d_inflow, c->nx, c->nz, c->n,
                                  pack_bc(c->bc), s);
}

}  // namespace

extern "C" {

rtlb_status rtlb_create(const rtlb_grid *grid, const rtlb_directions *dirs, const rtlb_options *opts,
                        rtlb_ctx **out)
{
    if (!out) return RTLB_E_ARG;
    *out = nullptr;
    if (!grid || !dirs) return RTLB_E_ARG;
    if (grid->nx < 1 || grid->nz < 1 || grid->nx > 65535 || grid->nz > 65535) return RTLB_E_SHAPE;
    rtlb_options o{};
    if (opts) o = *opts;
    if (o.precision < RTLB_PREC_FP32 || o.precision > RTLB_PREC_FP8X || o.survival < 0 || o.survival > 1 ||
        o.absorption < 0 || o.absorption > 1)
        return RTLB_E_ARG;
    std::vector<double> mu, phi, tap_w;
    std::vector<int> cx, cz, tap_o;
    rtlb_status st = build_dirs(dirs, o.streaming, o.plane, mu, phi, cx, cz, tap_o, tap_w, nullptr);
    if (st != RTLB_OK) return st;
    if (o.precision != RTLB_PREC_FP32 && !tc_shape_ok(dirs->n_zen * dirs->n_az, o.precision))
        return RTLB_E_UNSUPPORTED;

    rtlb_ctx *c = new (std::nothrow) rtlb_ctx();
    if (!c) return RTLB_E_OOM;
    cudaGetDevice(&c->dev);
    c->nx = grid->nx;
    c->nz = grid->nz;
    c->n_zen = dirs->n_zen;
    c->n_az = dirs->n_az;
    c->n = dirs->n_zen * dirs->n_az;
    c->mu = mu;
    c->phi = phi;
    c->cx = cx;
    c->cz = cz;
    c->tap_o = tap_o;
    c->tap_w.assign(tap_w.begin(), tap_w.end());
    c->opt = o;
    c->inflow.assign((size_t)4 * c->n * 4, 0.0f);
    const size_t bytes = c->state_floats() * sizeof(float);
    const int nblk = residual_blocks(c->state_floats());
    c->scratch_len = nblk;
    std::vector<int> dirbuf(2 * c->n);
    for (int d = 0; d < c->n; ++d) {
        dirbuf[d] = cx[d];
        dirbuf[c->n + d] = cz[d];
    }
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc(&c->S[0], bytes);
    if (e == cudaSuccess) e = cudaMalloc(&c->S[1], bytes);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_dir, dirbuf.size() * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_dir0, dirbuf.size() * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_tap_o, c->tap_o.size() * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_tap_w, c->tap_w.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_inflow, c->inflow.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_scratch, (size_t)3 * nblk * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_out, 8 * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_flags, 4 * sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_out, 8 * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_flags, 4 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->S[0], 0, bytes);
    if (e == cudaSuccess) e = cudaMemset(c->S[1], 0, bytes);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_dir, dirbuf.data(), dirbuf.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(c->d_dir0, 0, dirbuf.size() * sizeof(int));
    if (e == cudaSuccess)
        e = cudaMemcpy(c->d_tap_o, c->tap_o.data(), c->tap_o.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(c->d_tap_w, c->tap_w.data(), c->tap_w.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(c->d_inflow, c->inflow.data(), c->inflow.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        const rtlb_status s = e == cudaErrorMemoryAllocation ? RTLB_E_OOM : RTLB_E_CUDA;
        free_ctx_buffers(c);
        delete c;
        cudaGetLastError();
        return s;
    }
    *out = c;
    return RTLB_OK;
}

void rtlb_destroy(rtlb_ctx *ctx)
{
    if (!ctx) return;
    cudaDeviceSynchronize();
    free_ctx_buffers(ctx);
    delete ctx;
}

const char *rtlb_last_error(const rtlb_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int64_t rtlb_steps_done(const rtlb_ctx *ctx) { return ctx ? ctx->steps : -1; }

rtlb_status rtlb_get_form(const rtlb_ctx *ctx, rtlb_form *out)
{
    if (!ctx || !out) return RTLB_E_ARG;
    *out = rtlb_form{};
    if (!ctx->medium_set) return RTLB_OK;
    int pair = 0, stages = 0;
    if (ctx->opt.precision != RTLB_PREC_FP32 && tc_form(ctx, &pair, &stages)) {
        out->tensor_core = 1;
        out->cta_pair = pair;
        out->stages = stages;
        out->mixed_tiles = tc_mixed_tiles(ctx);
    }
    out->gather_form = gather_form(ctx) ? 1 : 0;
    return RTLB_OK;
}

rtlb_status rtlb_set_medium(rtlb_ctx *c, const float *tau, const float *albedo, const float *emission,
                            int32_t n_phase, const double *phase_tables, const uint8_t *phase_index,
                            void *stream)
{
    if (!c) return RTLB_E_ARG;
    if (!tau || !albedo || !phase_tables) return fail(c, RTLB_E_ARG, "tau, albedo and phase_tables are required");
    if (n_phase < 1 || n_phase > kMaxPhase) return fail(c, RTLB_E_ARG, "n_phase must be in [1, %d]", kMaxPhase);
    const int N4 = 4 * c->n;
    const size_t tsz = (size_t)N4 * N4;
    for (size_t j = 0; j < (size_t)n_phase * tsz; ++j)
        if (!std::isfinite(phase_tables[j])) return fail(c, RTLB_E_NONFINITE, "phase table entry %zu is not finite", j);
    const int ns = (int)c->nsites();
    cudaStream_t s = S(stream);

    // device copies of host inputs
    float *tmp[3] = {nullptr, nullptr, nullptr};
    uint8_t *tmp_cls = nullptr;
    float4 *coef = nullptr;
    uint8_t *cls_dev = nullptr;
    float *ZT = nullptr, *Zr = nullptr, *tau_keep = nullptr, *alb_keep = nullptr;
    auto cleanup = [&]() {
        for (float *t : tmp) cudaFree(t);
        cudaFree(tmp_cls);
        cudaFree(coef);
        cudaFree(cls_dev);
        cudaFree(ZT);
        cudaFree(Zr);
        cudaFree(tau_keep);
        cudaFree(alb_keep);
    };
    const float *in[3] = {tau, albedo, emission};
    const float *dev_in[3] = {nullptr, nullptr, nullptr};
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
        if (!in[k]) continue;
        if (is_device_ptr(in[k])) {
            dev_in[k] = in[k];
        } else {
            e = cudaMalloc(&tmp[k], ns * sizeof(float));
            if (e == cudaSuccess) e = cudaMemcpyAsync(tmp[k], in[k], ns * sizeof(float), cudaMemcpyHostToDevice, s);
            dev_in[k] = tmp[k];
        }
    }
    const uint8_t *dev_cls = nullptr;
    if (e == cudaSuccess && phase_index) {
        if (is_device_ptr(phase_index)) {
            dev_cls = phase_index;
        } else {
            e = cudaMalloc(&tmp_cls, ns);
            if (e == cudaSuccess) e = cudaMemcpyAsync(tmp_cls, phase_index, ns, cudaMemcpyHostToDevice, s);
            dev_cls = tmp_cls;
        }
    }
    std::vector<float> zt((size_t)n_phase * tsz), zr((size_t)n_phase * tsz);
    for (int p = 0; p < n_phase; ++p)
        for (int row = 0; row < N4; ++row)
            for (int col = 0; col < N4; ++col) {
                const float v = (float)phase_tables[(size_t)p * tsz + (size_t)row * N4 + col];
                zt[(size_t)p * tsz + (size_t)col * N4 + row] = v;
                zr[(size_t)p * tsz + (size_t)row * N4 + col] = v;
            }
    if (e == cudaSuccess) e = cudaMalloc(&coef, (size_t)ns * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc(&cls_dev, (size_t)ns);
    if (e == cudaSuccess) e = cudaMalloc(&ZT, zt.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpyAsync(ZT, zt.data(), zt.size() * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMalloc(&Zr, zr.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpyAsync(Zr, zr.data(), zr.size() * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMalloc(&tau_keep, (size_t)ns * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&alb_keep, (size_t)ns * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpyAsync(tau_keep, dev_in[0], (size_t)ns * sizeof(float), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(alb_keep, dev_in[1], (size_t)ns * sizeof(float), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_flags, 0, sizeof(int), s);
    if (e == cudaSuccess)
        e = launch_prep_medium(dev_in[0], dev_in[1], dev_in[2], dev_cls, coef, cls_dev, ns, n_phase,
                               c->opt.survival, c->opt.absorption, c->d_flags, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->h_flags, c->d_flags, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(c, e, "set_medium");
    }
    const int flags = c->h_flags[0];
    if (flags) {
        cleanup();
        if (flags & 1) return fail(c, RTLB_E_NONFINITE, "medium contains NaN or Inf");
        if (flags & 4) return fail(c, RTLB_E_RANGE, "phase_index >= n_phase");
        return fail(c, RTLB_E_RANGE,
                    "medium out of range: need tau >= 0, 0 <= albedo <= 1, emission >= 0, "
                    "albedo*tau <= 1 (linear survival), (1-albedo)*tau <= 1 (Taylor absorption)");
    }
    rtlb_status tst = tc_prepare(c, phase_tables, n_phase, dev_cls, s);
    if (tst != RTLB_OK) {
        cleanup();
        return tst;
    }
    for (float *t : tmp) cudaFree(t);
    cudaFree(tmp_cls);
    cudaFree(c->d_coef);
    cudaFree(c->d_cls);
    cudaFree(c->d_ZT);
    cudaFree(c->d_Z);
    cudaFree(c->d_tau);
    cudaFree(c->d_alb);
    c->d_coef = coef;
    c->d_cls = cls_dev;
    c->d_ZT = ZT;
    c->d_Z = Zr;
    c->d_tau = tau_keep;
    c->d_alb = alb_keep;
    c->n_phase = n_phase;
    c->medium_set = true;
    ++c->medium_gen;
    return RTLB_OK;
}

rtlb_status rtlb_set_boundary(rtlb_ctx *c, int32_t side, int32_t kind, const float *inflow)
{
    if (!c) return RTLB_E_ARG;
    if (side < 0 || side > 3) return fail(c, RTLB_E_ARG, "side must be 0..3");
    if (kind < RTLB_BC_VACUUM || kind > RTLB_BC_INFLOW) return fail(c, RTLB_E_ARG, "bad boundary kind %d", kind);
    if (kind == RTLB_BC_INFLOW && !inflow) return fail(c, RTLB_E_ARG, "INFLOW needs an inflow table");
    std::vector<float> nv = c->inflow;
    float *dst = &nv[(size_t)side * c->n * 4];
    for (int j = 0; j < c->n * 4; ++j) {
        const float v = (kind == RTLB_BC_INFLOW) ? inflow[j] : 0.0f;
        if (!std::isfinite(v)) return fail(c, RTLB_E_NONFINITE, "inflow entry %d is not finite", j);
        dst[j] = v;
    }
    // the deferred streaming of the last step belongs to the old boundary
    rtlb_status sst = settle(c, nullptr, true);
    if (sst != RTLB_OK) return sst;
    CK(c, cudaDeviceSynchronize(), "set_boundary sync");
    CK(c, cudaMemcpy(c->d_inflow, nv.data(), nv.size() * sizeof(float), cudaMemcpyHostToDevice), "inflow upload");
    c->inflow.swap(nv);
    c->bc[side] = kind;
    return RTLB_OK;
}

rtlb_status rtlb_set_state(rtlb_ctx *c, const float *Sin, void *stream)
{
    if (!c || !Sin) return fail(c, RTLB_E_ARG, "null argument");
    cudaStream_t s = S(stream);
    const size_t bytes = c->state_floats() * sizeof(float);
    const float *src = Sin;
    if (!is_device_ptr(Sin)) {
        rtlb_status st = ensure_stage(c);
        if (st != RTLB_OK) return st;
        CK(c, cudaMemcpyAsync(c->d_stage, Sin, bytes, cudaMemcpyHostToDevice, s), "state upload");
        src = c->d_stage;
    }
    CK(c, launch_user_to_dm(src, c->S[c->cur], (int)c->nsites(), c->n, s), "state layout");
    c->steps = 0;
    c->has_prev = false;
    c->deferred = c->prev_deferred = c->view_valid = false;
    return RTLB_OK;
}

rtlb_status rtlb_get_state(rtlb_ctx *c, float *Sout, void *stream)
{
    if (!c || !Sout) return fail(c, RTLB_E_ARG, "null argument");
    cudaStream_t s = S(stream);
    const size_t bytes = c->state_floats() * sizeof(float);
    const float *cur = nullptr;
    rtlb_status st = state_view(c, s, &cur);
    if (st != RTLB_OK) return st;
    if (is_device_ptr(Sout)) {
        CK(c, launch_dm_to_user(cur, Sout, (int)c->nsites(), c->n, s), "state layout");
        return RTLB_OK;
    }
    st = ensure_stage(c);
    if (st != RTLB_OK) return st;
    CK(c, launch_dm_to_user(cur, c->d_stage, (int)c->nsites(), c->n, s), "state layout");
    CK(c, cudaMemcpyAsync(Sout, c->d_stage, bytes, cudaMemcpyDeviceToHost, s), "state download");
    CK(c, cudaStreamSynchronize(s), "state download sync");
    return tc_check_error(c, s);
}

rtlb_status rtlb_step(rtlb_ctx *c, int32_t nsteps, void *stream)
{
    if (!c) return RTLB_E_ARG;
    if (nsteps < 0) return fail(c, RTLB_E_ARG, "nsteps must be >= 0");
    if (!c->medium_set) return fail(c, RTLB_E_STATE, "rtlb_set_medium must come before rtlb_step");
    rtlb_status st = require_boundary_pairs(c);
    if (st != RTLB_OK) return st;
    cudaStream_t s = S(stream);
    if (bilinear(c)) {
        st = ensure_post(c);
        if (st != RTLB_OK) return st;
    }
    const bool gf = gather_form(c);
    if (!gf && c->deferred) {
        st = settle(c, s, true);
        if (st != RTLB_OK) return st;
    }
    for (int t = 0; t < nsteps; ++t) {
        StepParams p = make_params(c);
        if (gf) {
            // gather form: the collision leaves P at its site in the other
            // buffer; with the streaming of the step before deferred, the
            // operand is gathered from the P in S[cur] while loading
            p.dir = c->d_dir0;
            if (c->deferred) {
                p.taps_o = c->d_tap_o;
                p.taps_w = c->d_tap_w;
            }
        } else if (bilinear(c)) {
            // collision in place (zero offsets) into the post-collision buffer,
            // then the four-tap streaming into the next state
            p.dir = c->d_dir0;
            p.S_new = c->d_post;
        }
        cudaError_t e;
        if (c->opt.precision == RTLB_PREC_FP32) {
            e = launch_step_fp32(p, s);
        } else {
            st = tc_step(c, p, s);
            if (st != RTLB_OK) return st;
            e = cudaSuccess;
        }
        if (e == cudaSuccess && bilinear(c) && !gf)
            e = launch_stream_bilinear(c->d_post, c->S[c->cur ^ 1], c->d_tap_o, c->d_tap_w, c->d_inflow, c->nx, c->nz,
                                       c->n, pack_bc(c->bc), s);
        if (e != cudaSuccess) return cuda_fail(c, e, "step launch");
        if (gf) {
            c->prev_deferred = c->deferred;
            c->deferred = true;
            c->view_valid = false;
        }
        c->cur ^= 1;
        c->has_prev = true;
        ++c->steps;
    }
    return RTLB_OK;
}

static rtlb_status residual_now(rtlb_ctx *c, double *res, cudaStream_t s)
{
    {
        const rtlb_status te = tc_check_error(c, s);
        if (te != RTLB_OK) return te;
    }
    const float *cur = nullptr, *prev = c->S[c->cur ^ 1];
    rtlb_status st = state_view(c, s, &cur);
    if (st != RTLB_OK) return st;
    if (c->prev_deferred) {
        st = ensure_stage(c);
        if (st != RTLB_OK) return st;
        CK(c, gather_into(c, c->S[c->cur ^ 1], c->d_stage, s), "deferred streaming");
        prev = c->d_stage;
    }
    CK(c, launch_residual(prev, cur, c->state_floats(), c->d_scratch, c->scratch_len, c->d_out, s), "residual");
    CK(c, cudaMemcpyAsync(c->h_out, c->d_out, 3 * sizeof(double), cudaMemcpyDeviceToHost, s), "residual copy");
    CK(c, cudaStreamSynchronize(s), "residual sync");
    if (c->h_out[2] != 0.0) return fail(c, RTLB_E_NONFINITE, "state contains %.0f non-finite entries", c->h_out[2]);
    *res = c->h_out[1] > 0.0 ? c->h_out[0] / c->h_out[1] : c->h_out[0];
    return RTLB_OK;
}

rtlb_status rtlb_last_residual(rtlb_ctx *c, double *residual, void *stream)
{
    if (!c || !residual) return fail(c, RTLB_E_ARG, "null argument");
    if (!c->has_prev) return fail(c, RTLB_E_STATE, "no step since the state was set");
    return residual_now(c, residual, S(stream));
}

rtlb_status rtlb_run_to_steady(rtlb_ctx *c, double tol, int32_t max_steps, int32_t check_every,
                               int32_t *steps_taken, double *residual, void *stream)
{
    if (!c || !steps_taken || !residual) return fail(c, RTLB_E_ARG, "null argument");
    if (!(tol > 0.0) || max_steps < 1 || check_every < 1) return fail(c, RTLB_E_ARG, "need tol > 0, max_steps >= 1, check_every >= 1");
    cudaStream_t s = S(stream);
    int taken = 0;
    double r = INFINITY;
    while (taken < max_steps) {
        const int k = (max_steps - taken) < check_every ? (max_steps - taken) : check_every;
        rtlb_status st = rtlb_step(c, k, stream);
        if (st != RTLB_OK) return st;
        taken += k;
        st = residual_now(c, &r, s);
        if (st != RTLB_OK) {
            *steps_taken = taken;
            return st;
        }
        if (r < tol) break;
    }
    *steps_taken = taken;
    *residual = r;
    if (!(r < tol)) return fail(c, RTLB_E_NOT_CONVERGED, "residual %.3e after %d steps (tol %.3e)", r, taken, tol);
    return RTLB_OK;
}

// Tensor-core reverse-step state for the current medium (4n = 128): Z^T as
// bf16 hi + lo from the float32 tables (B[c][k] = Z[k][c], K-major), the
// single-class 128-site tiles sorted by class and the mixed ones, and the
// negated streaming offsets.
static rtlb_status prepare_adj_tc(rtlb_ctx *c)
{
    AdjTcState &a = c->adj_tc;
    if (a.gen == c->medium_gen) return RTLB_OK;
    a.release();
    const int n = c->n, N4 = 4 * n, np = c->n_phase, KP = (N4 + 63) / 64 * 64;
    const size_t ns = c->nsites(), tsz = (size_t)N4 * N4, psz = (size_t)N4 * KP;
    std::vector<float> Z((size_t)np * tsz);
    CK(c, cudaMemcpy(Z.data(), c->d_Z, Z.size() * sizeof(float), cudaMemcpyDeviceToHost), "adjoint tables");
    // Z^T rows (one per output of the transposed contraction), K padded with zeros
    std::vector<__nv_bfloat16> hi((size_t)np * psz, __float2bfloat16(0.f)), lo((size_t)np * psz, __float2bfloat16(0.f));
    for (int ph = 0; ph < np; ++ph)
        for (int col = 0; col < N4; ++col)
            for (int k = 0; k < N4; ++k) {
                const float v = Z[(size_t)ph * tsz + (size_t)k * N4 + col];
                const __nv_bfloat16 h = __float2bfloat16(v);
                hi[(size_t)ph * psz + (size_t)col * KP + k] = h;
                lo[(size_t)ph * psz + (size_t)col * KP + k] = __float2bfloat16(v - __bfloat162float(h));
            }
    std::vector<uint8_t> cls(ns);
    CK(c, cudaMemcpy(cls.data(), c->d_cls, ns, cudaMemcpyDeviceToHost), "adjoint classes");
    const int ntiles = (int)((ns + 127) / 128);
    std::vector<int> pure, mixed;
    for (int t = 0; t < ntiles; ++t) {
        const size_t b = (size_t)t * 128, e = std::min(ns, b + 128);
        bool same = true;
        for (size_t k = b + 1; k < e && same; ++k) same = cls[k] == cls[b];
        if (same) pure.push_back(t | ((int)cls[b] << 24));
        else mixed.push_back(t);
    }
    std::stable_sort(pure.begin(), pure.end(), [](int x, int y) { return (x >> 24) < (y >> 24); });
    std::vector<int> dirT(2 * n);
    for (int d = 0; d < n; ++d) {
        dirT[d] = -c->cx[d];
        dirT[n + d] = -c->cz[d];
    }
    CK(c, a.zhi.ensure(hi.size() * 2), "adjoint tables");
    CK(c, a.zlo.ensure(lo.size() * 2), "adjoint tables");
    CK(c, a.pure.ensure(std::max<size_t>(pure.size(), 1) * sizeof(int)), "adjoint tiles");
    CK(c, a.mixed.ensure(std::max<size_t>(mixed.size(), 1) * sizeof(int)), "adjoint tiles");
    CK(c, a.dirT.ensure(dirT.size() * sizeof(int)), "adjoint offsets");
    CK(c, cudaMemcpy(a.zhi.p, hi.data(), hi.size() * 2, cudaMemcpyHostToDevice), "adjoint tables");
    CK(c, cudaMemcpy(a.zlo.p, lo.data(), lo.size() * 2, cudaMemcpyHostToDevice), "adjoint tables");
    if (!pure.empty()) CK(c, cudaMemcpy(a.pure.p, pure.data(), pure.size() * sizeof(int), cudaMemcpyHostToDevice), "adjoint tiles");
    if (!mixed.empty())
        CK(c, cudaMemcpy(a.mixed.p, mixed.data(), mixed.size() * sizeof(int), cudaMemcpyHostToDevice), "adjoint tiles");
    CK(c, cudaMemcpy(a.dirT.p, dirT.data(), dirT.size() * sizeof(int), cudaMemcpyHostToDevice), "adjoint offsets");
    if (!tc_encode_table_map(&a.tmZhi, a.zhi.as<__nv_bfloat16>(), N4, KP, np, N4) ||
        !tc_encode_table_map(&a.tmZlo, a.zlo.as<__nv_bfloat16>(), N4, KP, np, N4))
        return fail(c, RTLB_E_CUDA, "tensor map encoding for the adjoint tables failed");
    a.n_pure = (int)pure.size();
    a.n_mixed = (int)mixed.size();
    a.gen = c->medium_gen;
    return RTLB_OK;
}

rtlb_status rtlb_adjoint(rtlb_ctx *c, int32_t nsteps, int32_t checkpoint_every, const float *dL_dout,
                         float *grad_tau, float *grad_albedo, double *grad_Z, float *grad_S0, void *stream)
{
    if (!c || !dL_dout) return fail(c, RTLB_E_ARG, "null argument");
    if (nsteps < 1 || checkpoint_every < 1) return fail(c, RTLB_E_ARG, "need nsteps >= 1 and checkpoint_every >= 1");
    if (!c->medium_set) return fail(c, RTLB_E_STATE, "rtlb_set_medium must come before rtlb_adjoint");
    if (!adjoint_supported(c->n)) return fail(c, RTLB_E_UNSUPPORTED, "the adjoint needs n in {8, 16, 32, 64}");
    rtlb_status st = require_boundary_pairs(c);
    if (st != RTLB_OK) return st;
    cudaStream_t s = S(stream);
    const size_t L = c->state_floats(), bytes = L * sizeof(float), ns = c->nsites();
    const int K = checkpoint_every, nseg = (nsteps + K - 1) / K, N4 = 4 * c->n;
    const int nslots = adjoint_table_slots();
    const size_t glen = (size_t)c->n_phase * N4 * N4;
    // workspace: grown to this call's sizes (a call that needs no more than
    // the last one allocates nothing); on an allocation failure the whole
    // workspace is released and allocated once more at these sizes
    AdjWork &w = c->adj;
    const size_t dl_bytes = (size_t)c->nx * c->n * 4 * sizeof(float);
    const bool host_dl = !is_device_ptr(dL_dout);
    const bool stage_t = grad_tau && !is_device_ptr(grad_tau), stage_a = grad_albedo && !is_device_ptr(grad_albedo);
    const bool stage_S = grad_S0 && !is_device_ptr(grad_S0);
    const std::pair<DevBuf *, size_t> need[] = {
        {&w.ck, (size_t)nseg * bytes},
        {&w.seg, K > 1 ? (size_t)std::max(K - 1, 2) * bytes : 0},
        {&w.lam, 2 * bytes},
        {&w.bm, bytes},
        {&w.ga, 2 * ns * sizeof(double)},
        {&w.gb, 2 * ns * sizeof(double)},
        {&w.slots, (size_t)nslots * glen * sizeof(double)},
        {&w.G, glen * sizeof(double)},
        {&w.tapT, bilinear(c) ? c->tap_o.size() * sizeof(int) : 0},
        {&w.dl, host_dl ? dl_bytes : 0},
        {&w.gtd, stage_t ? ns * sizeof(float) : 0},
        {&w.gad, stage_a ? ns * sizeof(float) : 0},
        {&w.gS, stage_S ? bytes : 0},
        {&w.cmask, adjoint_chunk_masks_bytes((int)ns)},
        {&w.tpart, adjoint_table_tc_supported(c->n, c->n_phase) ? (size_t)nslots * glen * sizeof(float) : 0},
        {&w.tacc, adjoint_table_tc_supported(c->n, c->n_phase) ? 2 * glen * sizeof(float) : 0},
    };
    auto grow = [&]() -> cudaError_t {
        for (const auto &b : need) {
            const cudaError_t e = b.first->ensure(b.second);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    };
    if (grow() != cudaSuccess) {
        cudaGetLastError();
        w.release();
        const cudaError_t e = grow();
        if (e != cudaSuccess) {
            w.release();
            return cuda_fail(c, e, "adjoint workspace");
        }
    }
    float *ck = w.ck.as<float>(), *seg = w.seg.as<float>(), *lam = w.lam.as<float>(), *bm = w.bm.as<float>();
    float *gtd = w.gtd.as<float>(), *gad = w.gad.as<float>(), *gS = w.gS.as<float>();
    double *ga = w.ga.as<double>(), *gb = w.gb.as<double>(), *slots = w.slots.as<double>(), *G = w.G.as<double>();
    int *tapT = w.tapT.as<int>();
#define AK(call, what)                                \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, (what)); \
    } while (0)
    int bcT[4];
    for (int k = 0; k < 4; ++k) bcT[k] = c->bc[k] == RTLB_BC_PERIODIC ? RTLB_BC_PERIODIC : RTLB_BC_VACUUM;
    // 4n in {32, 64, 128} with nearest-neighbour streaming: the reverse step
    // runs on the tensor cores in the transposed-stream form.  Tiles that mix
    // phase classes take a CUDA-core variant of that form, which exists for
    // 4n = 128 only: at n = 8 and 16 a medium with such tiles keeps the
    // lambda form on the CUDA cores.
    bool nu_form = !bilinear(c) && adjoint_tc_stages(c->n) > 0;
    if (nu_form) {
        st = prepare_adj_tc(c);
        if (st != RTLB_OK) return st;
        if (c->n != 32 && c->adj_tc.n_mixed > 0) nu_form = false;
    }
    if (bilinear(c)) {
        st = ensure_post(c);
        if (st != RTLB_OK) return st;
        st = settle(c, s, false);                   // S^0 in S[cur]
        if (st != RTLB_OK) return st;
        std::vector<int> neg(c->tap_o.size());
        for (size_t k = 0; k < neg.size(); ++k) neg[k] = -c->tap_o[k];
        AK(cudaMemcpy(tapT, neg.data(), neg.size() * sizeof(int), cudaMemcpyHostToDevice), "adjoint taps");
    }
    const float *dl_dev = dL_dout;
    if (host_dl) {
        AK(cudaMemcpyAsync(w.dl.p, dL_dout, dl_bytes, cudaMemcpyHostToDevice, s), "adjoint seed upload");
        dl_dev = w.dl.as<float>();
    }
    // forward in float32, stepping from checkpoint to checkpoint: segment g
    // starts at ck[g] and ends in ck[g + 1] (the last one in the state buffer
    // the context's step count points at), through at most two scratch
    // states in between; no state is copied except S^0.
    const int fin = c->cur ^ (nsteps & 1);
    AK(cudaMemcpyAsync(ck, c->S[c->cur], bytes, cudaMemcpyDeviceToDevice, s), "checkpoint");
    for (int g = 0; g < nseg; ++g) {
        const int len = std::min(K, nsteps - g * K);
        for (int j = 0; j < len; ++j) {
            const float *in = j == 0 ? ck + (size_t)g * L : seg + (size_t)((j - 1) & 1) * L;
            float *out = j + 1 < len ? seg + (size_t)(j & 1) * L
                                     : (g + 1 < nseg ? ck + (size_t)(g + 1) * L : c->S[fin]);
            AK(fp32_step_into(c, in, out, s), "adjoint forward");
        }
    }
    c->cur = fin;
    c->steps += nsteps;
    c->has_prev = true;
    c->deferred = c->prev_deferred = c->view_valid = false;
    // reverse sweep
    AK(cudaMemsetAsync(lam, 0, 2 * bytes, s), "lambda init");
    AK(cudaMemsetAsync(ga, 0, 2 * ns * sizeof(double), s), "g_alpha init");
    AK(cudaMemsetAsync(gb, 0, 2 * ns * sizeof(double), s), "g_beta init");
    AK(cudaMemsetAsync(slots, 0, (size_t)nslots * glen * sizeof(double), s), "slots init");
    const bool table_tc = adjoint_table_tc_supported(c->n, c->n_phase);
    if (table_tc) AK(cudaMemsetAsync(w.tacc.p, 0, 2 * glen * sizeof(float), s), "table sum init");
    const uint32_t *cmask = w.cmask.as<uint32_t>();
    AK(launch_adjoint_chunk_masks(c->d_cls, (int)ns, w.cmask.as<uint32_t>(), s), "chunk class masks");
    int lc = 0;
    if (nu_form) {
        // transposed-stream form: lam[lc] holds nu^t = T^T lambda^{t+1}; each
        // reverse step writes nu^{t-1} (lambda^0 at t = 0) into lam[lc ^ 1]
        AdjTcState &a = c->adj_tc;
        CUtensorMap tmNu[2];
        for (int k = 0; k < 2; ++k)
            if (!tc_encode_state_map(&tmNu[k], lam + (size_t)k * L, ns, c->n))
                return fail(c, RTLB_E_CUDA, "tensor map encoding for the adjoint state failed");
        const int bcbitsT = pack_bc(bcT);
        int sm_count = 148;
        cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, c->dev);
        AK(launch_adjoint_seed_nu(lam, dl_dev, c->d_dir, c->nx, c->nz, c->n, bcbitsT, s), "adjoint seed");
        for (int g = nseg - 1; g >= 0; --g) {
            const int len = std::min(K, nsteps - g * K);
            auto state = [&](int j) -> float * { return j == 0 ? ck + (size_t)g * L : seg + (size_t)(j - 1) * L; };
            for (int j = 0; j + 1 < len; ++j) AK(fp32_step_into(c, state(j), state(j + 1), s), "adjoint recompute");
            for (int j = len - 1; j >= 0; --j) {
                const bool push = g * K + j > 0;
                AdjointParams ap;
                ap.lam_next = lam + (size_t)lc * L;
                ap.lam_out = lam + (size_t)(lc ^ 1) * L;
                ap.beta_mu = lam + (size_t)lc * L;     // nu^t, scaled by beta in the table gradient
                ap.beta_scale = 1;
                ap.S = state(j);
                ap.coef = c->d_coef;
                ap.cls = c->d_cls;
                ap.Z = c->d_Z;
                ap.dir = c->d_dir;
                ap.nx = c->nx;
                ap.nz = c->nz;
                ap.n = c->n;
                ap.n_phase = c->n_phase;
                for (int k = 0; k < 4; ++k) ap.bc[k] = c->bc[k];
                ap.g_alpha = ga;
                ap.g_beta = gb;
                ap.tiles = a.mixed.as<int>();
                ap.dirT = a.dirT.as<int>();
                ap.bcbitsT = bcbitsT;
                ap.push = push ? 1 : 0;
                ap.chunk_mask = cmask;
                ap.table_part = w.tpart.as<float>();
                ap.table_acc = w.tacc.as<float>();
                // the table gradient reads nu^t and S^t, the reverse step's
                // inputs, and nothing it writes: run first, it leaves part of
                // both in L2 for the reverse step
                if (RTLB_ADJ_TABLE_FIRST) AK(launch_adjoint_table(ap, slots, s), "adjoint table gradient");
                if (a.n_pure > 0) {
                    AdjTcLaunch tl;
                    tl.S = state(j);
                    tl.coef = c->d_coef;
                    tl.dirT = a.dirT.as<int>();
                    tl.bcbitsT = bcbitsT;
                    tl.nu_out = lam + (size_t)(lc ^ 1) * L;
                    tl.g_alpha = ga;
                    tl.g_beta = gb;
                    tl.tiles = a.pure.as<int>();
                    tl.n_tiles = a.n_pure;
                    tl.nx = c->nx;
                    tl.nz = c->nz;
                    tl.n = c->n;
                    tl.push = push ? 1 : 0;
                    tl.sm_count = sm_count;
                    AK(launch_adjoint_step_tc(tmNu[lc], a.tmZhi, a.tmZlo, tl, s), "adjoint step (tensor cores)");
                }
                AK(launch_adjoint_step_nu_mixed(ap, a.n_mixed, s), "adjoint step (mixed tiles)");
                if (!RTLB_ADJ_TABLE_FIRST) AK(launch_adjoint_table(ap, slots, s), "adjoint table gradient");
                lc ^= 1;
            }
        }
    } else {
    AK(launch_adjoint_seed(lam, dl_dev, c->d_dir, c->nx, c->nz, c->n, s), "adjoint seed");
    for (int g = nseg - 1; g >= 0; --g) {
        const int len = std::min(K, nsteps - g * K);
        // state j of the segment: the checkpoint for j = 0, recomputed into
        // seg[j - 1] otherwise (a checkpoint every step means no replay)
        auto state = [&](int j) -> float * { return j == 0 ? ck + (size_t)g * L : seg + (size_t)(j - 1) * L; };
        for (int j = 0; j + 1 < len; ++j) AK(fp32_step_into(c, state(j), state(j + 1), s), "adjoint recompute");
        for (int j = len - 1; j >= 0; --j) {
            AdjointParams ap;
            ap.lam_next = lam + (size_t)lc * L;
            if (bilinear(c)) {
                // transposed streaming first: each entry gathers from its four
                // streaming targets (negated taps); content that left through a
                // non-periodic side contributes nothing
                AK(launch_stream_bilinear(lam + (size_t)lc * L, c->d_post, tapT, c->d_tap_w, c->d_inflow, c->nx,
                                          c->nz, c->n, pack_bc(bcT), s),
                   "adjoint transposed streaming");
                ap.lam_next = c->d_post;
            }
            ap.lam_out = lam + (size_t)(lc ^ 1) * L;
            ap.beta_mu = bm;
            ap.S = state(j);
            ap.coef = c->d_coef;
            ap.cls = c->d_cls;
            ap.Z = c->d_Z;
            ap.dir = bilinear(c) ? c->d_dir0 : c->d_dir;
            ap.nx = c->nx;
            ap.nz = c->nz;
            ap.n = c->n;
            ap.n_phase = c->n_phase;
            for (int k = 0; k < 4; ++k) ap.bc[k] = c->bc[k];
            ap.g_alpha = ga;
            ap.g_beta = gb;
            ap.chunk_mask = cmask;
            ap.table_part = w.tpart.as<float>();
            ap.table_acc = w.tacc.as<float>();
            AK(launch_adjoint_step(ap, slots, s), "adjoint step");
            lc ^= 1;
        }
    }
    }
    // outputs
    if (grad_tau || grad_albedo) {
        // a missing output is computed into staging that is not read back
        float *ot = grad_tau && !stage_t ? grad_tau : gtd, *oa = grad_albedo && !stage_a ? grad_albedo : gad;
        if (!ot || !oa) {
            AK(w.gtd.ensure(ns * sizeof(float)), "grad staging");
            AK(w.gad.ensure(ns * sizeof(float)), "grad staging");
            gtd = w.gtd.as<float>();
            gad = w.gad.as<float>();
            if (!ot) ot = gtd;
            if (!oa) oa = gad;
        }
        AK(launch_adjoint_chain(ga, gb, c->d_tau, c->d_alb, (int)ns, c->opt.survival, c->opt.absorption, ot, oa, s),
           "adjoint chain rule");
        if (stage_t) AK(cudaMemcpyAsync(grad_tau, gtd, ns * sizeof(float), cudaMemcpyDeviceToHost, s), "grad_tau");
        if (stage_a)
            AK(cudaMemcpyAsync(grad_albedo, gad, ns * sizeof(float), cudaMemcpyDeviceToHost, s), "grad_albedo");
    }
    if (grad_Z) {
        if (table_tc) AK(launch_adjoint_table_tc_finish(w.tacc.as<float>(), (int)glen, slots, s), "table gradient sum");
        AK(launch_adjoint_fold(slots, nslots, glen, G, s), "table gradient");
        AK(cudaMemcpyAsync(grad_Z, G, glen * sizeof(double), cudaMemcpyDeviceToHost, s), "grad_Z");
    }
    if (grad_S0) {
        if (is_device_ptr(grad_S0)) {
            AK(launch_dm_to_user(lam + (size_t)lc * L, grad_S0, (int)ns, c->n, s), "grad_S0");
        } else {
            AK(launch_dm_to_user(lam + (size_t)lc * L, gS, (int)ns, c->n, s), "grad_S0");
            AK(cudaMemcpyAsync(grad_S0, gS, bytes, cudaMemcpyDeviceToHost, s), "grad_S0 download");
        }
    }
    AK(cudaStreamSynchronize(s), "adjoint sync");
#undef AK
    if (adjoint_table_tc_take_error() > 0) return fail(c, RTLB_E_TIMEOUT, "the table-gradient kernel gave up waiting");
    if (adjoint_step_tc_take_error() > 0) return fail(c, RTLB_E_TIMEOUT, "the tensor-core reverse step gave up waiting");
    if (c->opt.precision == RTLB_PREC_TF32X3) return tc_check_error(c, s);   // the forward's tensor-core steps
    return RTLB_OK;
}

rtlb_status rtlb_release_workspace(rtlb_ctx *c)
{
    if (!c) return RTLB_E_ARG;
    CK(c, cudaDeviceSynchronize(), "release workspace");
    c->adj.release();
    c->adj_tc.release();
    return RTLB_OK;
}

rtlb_status rtlb_radiance_out(rtlb_ctx *c, int32_t side, float *out, void *stream)
{
    if (!c || !out) return fail(c, RTLB_E_ARG, "null argument");
    if (side < 0 || side > 3) return fail(c, RTLB_E_ARG, "side must be 0..3");
    cudaStream_t s = S(stream);
    const int len = (side == RTLB_SIDE_TOP || side == RTLB_SIDE_BOTTOM) ? c->nx : c->nz;
    const size_t bytes = (size_t)len * c->n * 4 * sizeof(float);
    const float *cur = nullptr;
    const rtlb_status vst = state_view(c, s, &cur);
    if (vst != RTLB_OK) return vst;
    if (is_device_ptr(out)) {
        CK(c, launch_radiance_out(cur, out, c->nx, c->nz, c->n, c->d_dir, side, s), "radiance_out");
        return RTLB_OK;
    }
    const size_t need = (size_t)(c->nx > c->nz ? c->nx : c->nz) * c->n * 4;
    if (!c->d_rad) CK(c, cudaMalloc(&c->d_rad, need * sizeof(float)), "radiance staging");
    CK(c, launch_radiance_out(cur, c->d_rad, c->nx, c->nz, c->n, c->d_dir, side, s), "radiance_out");
    CK(c, cudaMemcpyAsync(out, c->d_rad, bytes, cudaMemcpyDeviceToHost, s), "radiance download");
    CK(c, cudaStreamSynchronize(s), "radiance sync");
    return RTLB_OK;
}

rtlb_status rtlb_dop_out(rtlb_ctx *c, int32_t side, float *out, void *stream)
{
    if (!c || !out) return fail(c, RTLB_E_ARG, "null argument");
    if (side < 0 || side > 3) return fail(c, RTLB_E_ARG, "side must be 0..3");
    cudaStream_t s = S(stream);
    const int len = (side == RTLB_SIDE_TOP || side == RTLB_SIDE_BOTTOM) ? c->nx : c->nz;
    const size_t bytes = (size_t)len * c->n * sizeof(float);
    const float *cur = nullptr;
    const rtlb_status vst = state_view(c, s, &cur);
    if (vst != RTLB_OK) return vst;
    if (is_device_ptr(out)) {
        CK(c, launch_dop_out(cur, out, c->nx, c->nz, c->n, c->d_dir, side, s), "dop_out");
        return RTLB_OK;
    }
    const size_t need = (size_t)(c->nx > c->nz ? c->nx : c->nz) * c->n * 4;
    if (!c->d_rad) CK(c, cudaMalloc(&c->d_rad, need * sizeof(float)), "radiance staging");
    CK(c, launch_dop_out(cur, c->d_rad, c->nx, c->nz, c->n, c->d_dir, side, s), "dop_out");
    CK(c, cudaMemcpyAsync(out, c->d_rad, bytes, cudaMemcpyDeviceToHost, s), "dop download");
    CK(c, cudaStreamSynchronize(s), "dop sync");
    return RTLB_OK;
}

rtlb_status rtlb_test_stall_next_step(rtlb_ctx *c)
{
    if (!c) return RTLB_E_ARG;
    if (!c->medium_set) return fail(c, RTLB_E_STATE, "rtlb_set_medium must come before the stall hook");
    if (c->opt.precision == RTLB_PREC_FP32) return fail(c, RTLB_E_UNSUPPORTED, "the stall hook needs a tensor-core precision");
    return tc_arm_stall(c);
}

rtlb_status rtlb_total_intensity(rtlb_ctx *c, double *total, void *stream)
{
    if (!c || !total) return fail(c, RTLB_E_ARG, "null argument");
    cudaStream_t s = S(stream);
    const float *cur = nullptr;
    const rtlb_status vst = state_view(c, s, &cur);
    if (vst != RTLB_OK) return vst;
    CK(c, launch_total_I(cur, c->state_floats() / 4, c->d_scratch, c->scratch_len, c->d_out, s), "total I");
    CK(c, cudaMemcpyAsync(c->h_out, c->d_out, sizeof(double), cudaMemcpyDeviceToHost, s), "total copy");
    CK(c, cudaStreamSynchronize(s), "total sync");
    {
        const rtlb_status te = tc_check_error(c, s);
        if (te != RTLB_OK) return te;
    }
    *total = c->h_out[0];
    return RTLB_OK;
}

rtlb_status rtlb_stream_offsets(const rtlb_directions *dirs, int32_t *cx, int32_t *cz)
{
    if (!cx || !cz) return RTLB_E_ARG;
    std::vector<double> mu, phi, tw;
    std::vector<int> x, z, to;
    rtlb_status st = build_dirs(dirs, RTLB_STREAM_NEAREST8, RTLB_PLANE_XZ, mu, phi, x, z, to, tw, nullptr);
    if (st != RTLB_OK) return st;
    for (size_t d = 0; d < x.size(); ++d) {
        cx[d] = x[d];
        cz[d] = z[d];
    }
    return RTLB_OK;
}

rtlb_status rtlb_stream_taps(const rtlb_directions *dirs, int32_t streaming, int32_t plane, int32_t *ox, int32_t *oz,
                             double *w)
{
    if (!ox || !oz || !w) return RTLB_E_ARG;
    std::vector<double> mu, phi, tw;
    std::vector<int> x, z, to;
    rtlb_status st = build_dirs(dirs, streaming, plane, mu, phi, x, z, to, tw, nullptr);
    if (st != RTLB_OK) return st;
    for (size_t d = 0; d < x.size(); ++d)
        for (int k = 0; k < 4; ++k) {
            ox[4 * d + k] = to[8 * d + k];
            oz[4 * d + k] = to[8 * d + 4 + k];
            w[4 * d + k] = tw[4 * d + k];
        }
    return RTLB_OK;
}

rtlb_status rtlb_phase_rayleigh(const rtlb_directions *dirs, double depol, double *Z_out)
{
    if (!Z_out) return RTLB_E_ARG;
    if (!(depol >= 0.0 && depol < 0.5)) return RTLB_E_RANGE;
    std::vector<double> mu, phi, tw;
    std::vector<int> x, z, to;
    rtlb_status st = build_dirs(dirs, RTLB_STREAM_BILINEAR, RTLB_PLANE_XZ, mu, phi, x, z, to, tw, nullptr);
    if (st != RTLB_OK) return st;
    phase_rayleigh(mu, phi, depol, Z_out);
    return RTLB_OK;
}

rtlb_status rtlb_phase_conserve_intensity(int32_t n, double *Z_inout)
{
    if (!Z_inout) return RTLB_E_ARG;
    if (n < 1 || n > kMaxDirs) return RTLB_E_SHAPE;
    conserve_intensity(n, Z_inout);
    return RTLB_OK;
}

rtlb_status rtlb_phase_hg(const rtlb_directions *dirs, double g, double pol_amp, double *Z_out, double *dZdg_out)
{
    if (!Z_out) return RTLB_E_ARG;
    if (!(g > -1.0 && g < 1.0) || !(std::fabs(pol_amp) <= 1.0)) return RTLB_E_RANGE;
    std::vector<double> mu, phi, tw;
    std::vector<int> x, z, to;
    rtlb_status st = build_dirs(dirs, RTLB_STREAM_BILINEAR, RTLB_PLANE_XZ, mu, phi, x, z, to, tw, nullptr);
    if (st != RTLB_OK) return st;
    phase_hg(mu, phi, g, pol_amp, Z_out, dZdg_out);
    return RTLB_OK;
}

rtlb_status rtlb_phase_hg_grad(const rtlb_directions *dirs, double g, double pol_amp, const double *grad_Z,
                               double *dL_dg)
{
    if (!grad_Z || !dL_dg) return RTLB_E_ARG;
    if (!(g > -1.0 && g < 1.0) || !(std::fabs(pol_amp) <= 1.0)) return RTLB_E_RANGE;
    std::vector<double> mu, phi, tw;
    std::vector<int> x, z, to;
    rtlb_status st = build_dirs(dirs, RTLB_STREAM_BILINEAR, RTLB_PLANE_XZ, mu, phi, x, z, to, tw, nullptr);
    if (st != RTLB_OK) return st;
    const size_t len = 16 * mu.size() * mu.size();
    std::vector<double> Z(len), dZ(len);
    phase_hg(mu, phi, g, pol_amp, Z.data(), dZ.data());
    // chain rule through the table: dL/dg = sum over entries of dL/dZ * dZ/dg,
    // summed in entry order (deterministic)
    double acc = 0.0;
    for (size_t j = 0; j < len; ++j) acc += grad_Z[j] * dZ[j];
    *dL_dg = acc;
    return RTLB_OK;
}

rtlb_status rtlb_phase_mix(const rtlb_directions *dirs, double m, double g, double pol_amp, double *Z_out)
{
    if (!Z_out) return RTLB_E_ARG;
    if (!(m >= 0.0 && m <= 1.0) || !(g > -1.0 && g < 1.0) || !(std::fabs(pol_amp) <= 1.0)) return RTLB_E_RANGE;
    std::vector<double> mu, phi, tw;
    std::vector<int> x, z, to;
    rtlb_status st = build_dirs(dirs, RTLB_STREAM_BILINEAR, RTLB_PLANE_XZ, mu, phi, x, z, to, tw, nullptr);
    if (st != RTLB_OK) return st;
    const size_t len = 16 * mu.size() * mu.size();
    std::vector<double> zr(len), zh(len);
    phase_rayleigh(mu, phi, 0.0, zr.data());
    phase_hg(mu, phi, g, pol_amp, zh.data(), nullptr);
    for (size_t j = 0; j < len; ++j) Z_out[j] = m * zr[j] + (1.0 - m) * zh[j];
    return RTLB_OK;
}

}  // extern "C"
