/*
 * rtlb.h -- C ABI of the B300 polarized lattice-Boltzmann radiative-transfer
 * library (librtlb.so).
 *
 * The library advances the classical lattice form of the polarized radiative
 * transfer equation (Eq. 1) on a 2D (x, z) lattice with n 3D directions, the
 * discrete update of Eq. 2: every site holds a Stokes vector (I, Q, U, V) per
 * direction, and one step applies emission (Eq. 6/8), absorption (Sec. 2.1.4),
 * scattering through rotated phase matrices (Eq. 11-17, 21-25) and streaming to
 * the D2Q9 neighbours (Sec. 2.1.6, boundary handling Sec. 2.1.7).
 *
 * Conventions shared by every call
 *  - Status codes, never exceptions.  On any error the context is unchanged and
 *    rtlb_last_error() describes the cause.
 *  - Pointers marked "host or device" may point to either; the library checks
 *    which with the CUDA runtime.  Pointers marked "device" must be device
 *    memory of the context's GPU.  The library never keeps a caller pointer:
 *    inputs are copied into library-owned buffers before the call returns (for
 *    device inputs: before the stream work the call enqueues completes).
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *    stream-ordered unless marked "synchronizes".
 *  - User state layout S[z][x][d][s], float32, s = I,Q,U,V; d = i_zen*n_az+i_az.
 *  - Lattice: x = 0..nx-1 left to right, z = 0..nz-1 bottom to top.
 */
#ifndef RTLB_H
#define RTLB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rtlb_ctx rtlb_ctx; /* opaque, library-owned */

typedef enum {
    RTLB_OK = 0,
    RTLB_E_ARG = 1,              /* null pointer, bad enum, bad count            */
    RTLB_E_SHAPE = 2,            /* lattice / direction sizes out of range       */
    RTLB_E_RANGE = 3,            /* medium value out of range (tau<0, albedo...) */
    RTLB_E_AMBIGUOUS_STREAM = 4, /* a direction lies between two lattice offsets */
    RTLB_E_STATE = 5,            /* call order (e.g. step before set_medium)     */
    RTLB_E_OOM = 6,              /* device allocation failed                     */
    RTLB_E_CUDA = 7,             /* CUDA runtime / launch error                  */
    RTLB_E_NONFINITE = 8,        /* NaN or Inf in an input or in the state       */
    RTLB_E_NOT_CONVERGED = 9,    /* run_to_steady hit max_steps                  */
    RTLB_E_TIMEOUT = 10,         /* a bounded device wait gave up                */
    RTLB_E_UNSUPPORTED = 11      /* precision form not available for this shape  */
} rtlb_status;

typedef enum { RTLB_SIDE_TOP = 0, RTLB_SIDE_BOTTOM = 1, RTLB_SIDE_LEFT = 2, RTLB_SIDE_RIGHT = 3 } rtlb_side;
typedef enum { RTLB_BC_VACUUM = 0, RTLB_BC_PERIODIC = 1, RTLB_BC_INFLOW = 2 } rtlb_bc;

/* Arithmetic of the scattering contraction (the state is always float32; the
 * unscattered and forward-scattered light are applied in float32 in every form):
 *  FP32     -- float32 FMA on the CUDA cores.
 *  BF16     -- tcgen05 tensor-core MMA, bf16 operands, float32 accumulation.
 *  BF16X3   -- tcgen05, both operands split hi+lo in bf16, three MMAs
 *              (n <= 32: the operands must fit one CTA's shared memory).
 *  BF16X2   -- tcgen05, bf16 state operand and the phase table as bf16 hi+lo,
 *              two MMAs (n = 64 runs on CTA pairs, each holding half the table).
 *  FP8      -- tcgen05 block-scaled MMA (kind::mxf8f6f4): e4m3 operands with
 *              one UE8M0 (power-of-two) scale per 32-element block -- per site
 *              and 8 directions for the state operand beta S~, per table row
 *              and 32 columns for the table -- float32 accumulation.  The
 *              scale of a block is the smallest 2^e with max|block| / 2^e <=
 *              448; values round to nearest even and saturate at +-448.  The
 *              table scales of every phase class stay in tensor memory, which
 *              bounds the classes (n = 64: 12); rtlb_set_medium returns
 *              RTLB_E_UNSUPPORTED beyond that.
 *  TF32X3   -- tcgen05 kind::tf32, both operands split into tf32 hi + lo
 *              (round to nearest; about 22 significand bits each), three MMAs
 *              (hi.hi + hi.lo + lo.hi), float32 accumulation: the accuracy of
 *              the FP32 form on the tensor cores.  The split state operand is
 *              kept in tensor memory.  n in {8, 16, 32} (the split tf32 table
 *              of n = 64 is 512 KB, more than any CTA's shared memory).
 *  FP8X     -- the block-scaled e4m3 MMA with both operands split: the state
 *              operand beta S~ as two e4m3 terms (hi; the remainder with the
 *              scale of its own block maximum), the table as three (each the
 *              e4m3 of what the terms before it left, with its own scale), and
 *              five MMAs (state term a times table term b for a + b <= 2, b <=
 *              2, a <= 1); float32 accumulation.  About the accuracy of BF16X2.
 *              The state terms are kept in tensor memory; with the table
 *              scales of every class resident there too, n = 64 takes at most
 *              2 phase classes (RTLB_E_UNSUPPORTED from rtlb_set_medium
 *              beyond).
 * Tensor-core forms need n in {8, 16, 32, 64} (TF32X3: {8, 16, 32});
 * rtlb_create returns RTLB_E_UNSUPPORTED otherwise.  Tiles of 128 sites that
 * mix phase classes run on the FP32 CUDA-core kernel in every form. */
typedef enum {
    RTLB_PREC_FP32 = 0,
    RTLB_PREC_BF16 = 1,
    RTLB_PREC_BF16X3 = 2,
    RTLB_PREC_BF16X2 = 3,
    RTLB_PREC_FP8 = 4,
    RTLB_PREC_TF32X3 = 5,
    RTLB_PREC_FP8X = 6
} rtlb_precision;

/* Survival of unscattered light over one step: LINEAR = 1 - k_scat dt (Eq. 11
 * as printed), EXP = exp(-k_scat dt).  Absorption: BEER_LAMBERT =
 * exp(-k_abs dt), TAYLOR = 1 - k_abs dt (Sec. 2.1.4). */
typedef enum { RTLB_SURV_LINEAR = 0, RTLB_SURV_EXP = 1 } rtlb_survival;
typedef enum { RTLB_ABS_BEER_LAMBERT = 0, RTLB_ABS_TAYLOR = 1 } rtlb_absorption;

typedef struct { int32_t nx, nz; } rtlb_grid;

/* Angular grid (Sec. 2.1, Eq. 4 text): n = n_zen * n_az directions.  With mu
 * and phi NULL the grid is uniform: mu = -1 + (2 i_zen + 1) / n_zen (equal
 * solid-angle zenith bins, downward first), phi = 2 pi i_az / n_az.  Otherwise
 * mu[n], phi[n] (host) list the directions explicitly (e.g. the azimuth and
 * zenith sets of Tables 1-2). */
typedef struct {
    int32_t n_zen, n_az;
    const double *mu;  /* host, optional, length n */
    const double *phi; /* host, optional, length n */
} rtlb_directions;

/* Streaming of each direction after the collision.
 *  NEAREST8 -- the D2Q9 neighbour offset nearest (by angle) to the direction's
 *              projection on the lattice plane (Sec. 2.1.6).
 *  BILINEAR -- semi-Lagrangian bilinear streaming (Eq. 33-38): over one step a
 *              direction moves l = its projection on the lattice plane (the
 *              paper's dt = dx / c); per axis n0 = floor(l), f = l - n0, and
 *              the field arriving at x is the sum over b_x, b_z in {0, 1} of
 *              w_x(b_x) w_z(b_z) P(x - (n0x + b_x), z - (n0z + b_z)), with
 *              w(0) = 1 - f, w(1) = f.  Components within 1e-12 of an integer
 *              are taken as that integer.  Sources outside the lattice take the
 *              side's ghost value exactly as in NEAREST8.
 * Lattice plane: XZ -- x horizontal, z vertical (the Stokes reference axis),
 * projection (sin(theta) cos(phi), mu); XY -- a horizontal lattice as in the
 * paper's 2D runs (Sec. 3.2), projection (sin(theta) cos(phi),
 * sin(theta) sin(phi)).  Either way the second lattice axis is called z here
 * and "top" is its last row. */
typedef enum { RTLB_STREAM_NEAREST8 = 0, RTLB_STREAM_BILINEAR = 1 } rtlb_streaming;
typedef enum { RTLB_PLANE_XZ = 0, RTLB_PLANE_XY = 1 } rtlb_plane;

/* All-zero options are the defaults: FP32, LINEAR, BEER_LAMBERT, NEAREST8, XZ. */
typedef struct {
    int32_t precision;  /* rtlb_precision  */
    int32_t survival;   /* rtlb_survival   */
    int32_t absorption; /* rtlb_absorption */
    int32_t streaming;  /* rtlb_streaming  */
    int32_t plane;      /* rtlb_plane      */
} rtlb_options;

/* Create a context on the current CUDA device.  With NEAREST8 streaming,
 * computes each direction's D2Q9 offset: the neighbour offset nearest (by
 * angle) to its projection on the lattice plane; a zero projection rests.
 * Returns RTLB_E_AMBIGUOUS_STREAM when a projection lies within 1e-9 (in
 * units of 45 degrees) of the midpoint between two offsets (BILINEAR has no
 * such case).  1 <= nx, nz <= 65535; 1 <= n <= 256.  opts may be NULL (all
 * defaults).  Allocates two state buffers of nx*nz*n*16 bytes (the state
 * starts at zero); BILINEAR adds a third on the first step. */
rtlb_status rtlb_create(const rtlb_grid *grid, const rtlb_directions *dirs,
                        const rtlb_options *opts, rtlb_ctx **out);

/* Medium of Eq. 2 in per-step dimensionless form: tau = k_ext dt (optical depth
 * of one cell and step), albedo = k_scat / k_ext, emission = dt J (added to I of
 * every direction each step, Eq. 6/8; NULL = 0), all [nz][nx] float32, host or
 * device.  phase_tables: host float64 [n_phase][4n][4n], row-major, entry
 * [4o+r][4i+k] maps incoming direction i, Stokes k to outgoing o, Stokes r (the
 * normalized redistribution of Eq. 13-17/25, e.g. from rtlb_phase_rayleigh).
 * phase_index: [nz][nx] uint8 class per site, host or device, NULL = class 0.
 * Checks (RTLB_E_RANGE / RTLB_E_NONFINITE): tau finite and >= 0, albedo in
 * [0, 1], emission finite and >= 0, phase_index < n_phase, LINEAR survival
 * needs albedo*tau <= 1, TAYLOR absorption needs (1-albedo)*tau <= 1.
 * 1 <= n_phase <= 16.  Synchronizes on `stream` (validation result). */
rtlb_status rtlb_set_medium(rtlb_ctx *ctx, const float *tau, const float *albedo,
                            const float *emission, int32_t n_phase,
                            const double *phase_tables, const uint8_t *phase_index,
                            void *stream);

/* Boundary kind of one side (Sec. 2.1.7): VACUUM = absorbing (zero-fill shift),
 * PERIODIC = recycling (shift modulo; must be set on both sides of an axis
 * before stepping), INFLOW = a fixed ghost Stokes vector per direction,
 * inflow[n][4] float32 host (required for INFLOW, ignored otherwise).  Ghost
 * corners belong to the top/bottom side.  Default: VACUUM everywhere. */
rtlb_status rtlb_set_boundary(rtlb_ctx *ctx, int32_t side, int32_t kind, const float *inflow);

/* Replace / read the state S[z][x][d][s] (float32, host or device). */
rtlb_status rtlb_set_state(rtlb_ctx *ctx, const float *S, void *stream);
rtlb_status rtlb_get_state(rtlb_ctx *ctx, float *S_out, void *stream);

/* Advance nsteps >= 0 steps: per step and site, emission, absorption,
 * scattering (the 4n x 4n contraction), then streaming of every direction to
 * its neighbour.  The stored state is the paper's S^t (after streaming); in
 * the gather form of BILINEAR streaming (rtlb_get_form) the context holds the
 * last step's post-collision field and streams it when a reader needs S^t
 * (rtlb_get_state, the readouts, the residual: one extra pass, done once per
 * step taken) or when the next step loads it.  rtlb_set_boundary completes a
 * pending streaming with the old boundary first. */
rtlb_status rtlb_step(rtlb_ctx *ctx, int32_t nsteps, void *stream);

/* Step until the residual max|S^{t+1} - S^t| / max|S^{t+1}| (float64 on the
 * device) is below tol, checking every check_every steps, or max_steps is
 * reached (RTLB_E_NOT_CONVERGED; the state is kept).  Synchronizes. */
rtlb_status rtlb_run_to_steady(rtlb_ctx *ctx, double tol, int32_t max_steps,
                               int32_t check_every, int32_t *steps_taken,
                               double *residual, void *stream);

/* Residual between the current state and the one before the last step
 * (float64, same definition as above).  Synchronizes. */
rtlb_status rtlb_last_residual(rtlb_ctx *ctx, double *residual, void *stream);

/* Radiance leaving through one side: out[len][n][4] float32 (host or device),
 * len = nx for top/bottom and nz for left/right: the state on the boundary row
 * or column for the directions that move out of the domain through that side
 * (NEAREST8: the offset points out; BILINEAR: the displacement component
 * across that side is nonzero and points out), zero for the others. */
rtlb_status rtlb_radiance_out(rtlb_ctx *ctx, int32_t side, float *out, void *stream);

/* Degree of polarization of the radiance leaving through one side (Sec. 3.2.1,
 * Eq. 36): out[len][n] float32 (host or device) = sqrt(Q^2 + U^2 + V^2) / I of
 * the entries rtlb_radiance_out returns, evaluated in float64 and rounded once;
 * zero for the directions that do not leave through that side and where
 * I <= 0.  Errors as rtlb_radiance_out. */
rtlb_status rtlb_dop_out(rtlb_ctx *ctx, int32_t side, float *out, void *stream);

/* Reverse-mode gradients (adjoint of Eq. 2's step: transposed phase-matrix
 * scattering and reversed streaming) of a loss L whose gradient with respect to
 * the top radiance radiance_out(TOP) after nsteps steps is dL_dout[nx][n][4]
 * (host or device).  Starting from the current state S^0 the call runs nsteps
 * float32-accurate steps (the 3xTF32 tensor-core step when the context's
 * precision is TF32X3, the FP32 CUDA-core step for every other precision; the
 * state afterwards is S^N, as after rtlb_step), keeping a checkpoint every
 * checkpoint_every steps,
 * then walks back segment by segment, recomputing each segment's states from
 * its checkpoint.  Outputs (each may be NULL): grad_tau, grad_albedo [nz][nx]
 * float32 (host or device) -- dL/dtau and dL/dalbedo per cell; grad_Z host
 * float64 [n_phase][4n][4n] -- dL/dZ per class table entry (contract with
 * rtlb_phase_hg's dZdg for dL/dg); grad_S0 [nz][nx][n][4] float32 (host or
 * device) -- dL/dS^0.  With BILINEAR streaming the reversed streaming
 * gathers each entry from its four streaming targets with the same weights.
 * Device memory: ceil(nsteps/checkpoint_every) + max(checkpoint_every - 1, 2)
 * + 3 states (checkpoint_every = 1: nsteps + 3, and no step is recomputed;
 * one more for BILINEAR) plus the table-gradient accumulators.  n must be in
 * {8, 16, 32, 64}.  At n in {8, 16, 32} with NEAREST streaming the reverse
 * step's transposed contraction runs on the tensor cores with bf16 hi + lo
 * operands (about 16 significand bits per product, float32 accumulation; the
 * first call after rtlb_set_medium builds the transposed tables) -- at n = 8
 * and 16 only when every 128-site tile of the medium is of one phase class;
 * elsewhere it runs on the CUDA cores in float32.  The table gradient runs on
 * the tensor cores (same split) where n <= 32 and n_phase * 4n <= 512, on the
 * CUDA cores otherwise.  Two identical calls return
 * identical results (no atomics in the sums).  The workspace stays allocated
 * after the call (see rtlb_release_workspace).  Synchronizes. */
rtlb_status rtlb_adjoint(rtlb_ctx *ctx, int32_t nsteps, int32_t checkpoint_every, const float *dL_dout,
                         float *grad_tau, float *grad_albedo, double *grad_Z, float *grad_S0,
                         void *stream);

/* rtlb_adjoint keeps its device workspace (the checkpoints, scratch and
 * adjoint states, accumulators and staging listed above) in the context
 * between calls and grows it only when a call needs more, so repeated calls
 * of the same size allocate nothing.  This frees it (rtlb_destroy does too);
 * the next rtlb_adjoint allocates again.  Synchronizes the device. */
rtlb_status rtlb_release_workspace(rtlb_ctx *ctx);

/* Total I over the lattice and directions, accumulated in float64 on the
 * device.  Synchronizes. */
rtlb_status rtlb_total_intensity(rtlb_ctx *ctx, double *total, void *stream);

/* Steps taken since the last rtlb_set_state (or creation). */
int64_t rtlb_steps_done(const rtlb_ctx *ctx);

/* How the context's steps run, as decided by rtlb_set_medium (all zero before
 * it): tensor_core = 1 for the tcgen05 step kernels (0: CUDA cores, float32);
 * cta_pair = 1 for the CTA-pair form (bf16x2 at n = 64); gather_form = 1 when
 * BILINEAR streaming is gathered while the next step loads its operand (one
 * pass over the state per step: the BF16, BF16X2 and BF16X3 tensor-core steps
 * at n in {16, 32} with nx % 128 == 0 -- other forms run a collision pass and
 * a gather pass; the state a reader sees is the same to the bit);
 * mixed_tiles = the 128-site tiles that mix phase classes (or are left
 * unpaired) and run on the CUDA-core kernel; stages = staging slots of the
 * tensor-core kernel.  RTLB_E_ARG for NULL. */
typedef struct {
    int32_t tensor_core, cta_pair, gather_form, mixed_tiles, stages;
} rtlb_form;
rtlb_status rtlb_get_form(const rtlb_ctx *ctx, rtlb_form *out);

const char *rtlb_last_error(const rtlb_ctx *ctx);
void rtlb_destroy(rtlb_ctx *ctx);

/* ---- many lattices in one launch ----
 *
 * A batch advances many independent contexts (e.g. spectral channels with
 * their own grid, n, medium and tables) with one persistent tensor-core
 * launch per step: the single-class 128-site tiles of all channels form one
 * work list, each item fetching its channel's pointers, TMA maps and tables
 * from a descriptor.  All channels must use the same tensor-core precision
 * (BF16 or BF16X2), n in {8, 16, 32} (n = 8, 16, 32 may be mixed), NEAREST8
 * streaming (RTLB_E_UNSUPPORTED otherwise), have a medium set, live on the
 * same device and stand at the same step parity.
 * Tiles mixing phase classes run on the CUDA-core kernel in the same step.
 * Channels keep working as ordinary contexts (get_state, radiance_out, ...);
 * stepping one alone desynchronizes the batch (rtlb_batch_step then returns
 * RTLB_E_STATE).  Changing a channel's medium or boundaries requires a new
 * batch. */
typedef struct rtlb_batch rtlb_batch;
rtlb_status rtlb_batch_create(int32_t count, rtlb_ctx *const *channels, rtlb_batch **out);

/* Shared-memory pipeline depth of the batch kernel: 2, 4, 6 or 8 16-KB state
 * stages (even: the two converter groups own half each; default 4; other
 * values give RTLB_E_RANGE).  Results do not depend on it. */
rtlb_status rtlb_batch_configure(rtlb_batch *batch, int32_t stages);

/* Work balance of the batch kernel: each CTA takes one contiguous range of
 * the batch's tiles (sorted by n, channel, class), ranges of equal estimated
 * work, a tile counting n + tile_cost directions' worth (default 4; 0 = bytes
 * only).  tile_cost in [0, 64], else RTLB_E_RANGE.  Synchronizes the device
 * (launches in flight read the ranges); results do not depend on it. */
rtlb_status rtlb_batch_balance(rtlb_batch *batch, int32_t tile_cost);

/* Advance every channel nsteps steps on `stream`; pairs of steps replay a
 * captured CUDA graph (one persistent launch per step plus any mixed-tile
 * launches). */
rtlb_status rtlb_batch_step(rtlb_batch *batch, int32_t nsteps, void *stream);

/* Reads (synchronizing) and clears the batch kernel's error flag:
 * RTLB_E_TIMEOUT when a bounded wait gave up. */
rtlb_status rtlb_batch_check(rtlb_batch *batch, void *stream);
const char *rtlb_batch_last_error(const rtlb_batch *batch);
void rtlb_batch_destroy(rtlb_batch *batch);

/* ---- residual without allocation (the paper has no counterpart) ----
 *
 * Same float64 residual as rtlb_last_residual, for callers that must not
 * allocate device memory: code running inside an allocator hook or a host
 * callback (where cudaMalloc is not allowed), processes whose device memory
 * pool is owned and capped by another framework, and latency-bound loops that
 * must never enter the driver's allocator.  Instead of a scratch buffer this
 * call uses a fixed 1.5 MiB array compiled into the library, which every GPU
 * that loads the library holds until the process exits.
 *
 * S_old, S_new: device float32 arrays of `count` entries (any layout, compared
 * elementwise), 16-byte aligned, count a multiple of 4.  out: device, 3
 * doubles, 8-byte aligned: {max|S_new - S_old|, max|S_new|, number of
 * non-finite entries of S_new}; the residual is out[0] / out[1].
 * count > RTLB_NOALLOC_MAX_COUNT returns RTLB_E_SHAPE; null pointers, pointers
 * that are not device (or managed) memory of the current device, bad
 * alignment or count % 4 != 0 return RTLB_E_ARG.  Never calls cudaMalloc /
 * cudaFree.  The first call in a CUDA context (normally: the first on each
 * device, with that device current) looks up the array's device address and
 * may make the driver load the library's device code, which can allocate
 * inside the driver; make that first call before any stream capture and
 * before any use from an allocator hook or host callback.  After a device
 * reset the next call looks the address up again.  All calls share the one
 * array and each overwrites the slots it reads, so two calls that overlap on
 * the GPU (different streams, no ordering) race.  Stream-ordered on `stream`. */
#define RTLB_NOALLOC_MAX_COUNT ((size_t)1 << 30)
rtlb_status rtlb_residual_noalloc(const float *S_old, const float *S_new, size_t count,
                                  double *out, void *stream);

/* ---- test hook of the bounded device waits (the paper has no counterpart) ----
 *
 * Every wait inside the tensor-core kernels gives up after about 2 s; the CTA
 * then drains its in-flight loads and MMAs, frees its tensor memory and
 * returns, and the next call that reads the device error flag
 * (rtlb_get_state, rtlb_last_residual, rtlb_total_intensity, ...) returns
 * RTLB_E_TIMEOUT and clears it.  This arms that path for a test: the next
 * tensor-core step launch of this context leaves the load of one state chunk
 * in its first CTA unissued, so that CTA's converter warps wait for data that
 * never comes.  Nothing is in flight for the skipped chunk, so the launch ends
 * normally after the wait runs out; the state after that step is undefined
 * (set it again) and the context stays usable.  Covers the BF16, BF16X3 and
 * BF16X2 kernels (single CTA and CTA pair); RTLB_E_UNSUPPORTED for FP32 and
 * FP8, RTLB_E_STATE before rtlb_set_medium.  Disarmed after one launch. */
rtlb_status rtlb_test_stall_next_step(rtlb_ctx *ctx);

/* ---- host helpers (float64, no GPU needed) ---- */

/* Per-direction D2Q9 offsets cx[n], cz[n] (host int32) of the grid on the
 * (x, z) plane (NEAREST8). */
rtlb_status rtlb_stream_offsets(const rtlb_directions *dirs, int32_t *cx, int32_t *cz);

/* Streaming taps of every direction for a scheme and plane (rtlb_streaming,
 * rtlb_plane): tap k of direction d moves content by (ox, oz)[4d + k] cells
 * with weight w[4d + k] (host int32 / float64, [n][4]).  BILINEAR lists
 * (b_x, b_z) = (0,0), (1,0), (0,1), (1,1); NEAREST8 puts the offset in tap 0
 * with weight 1 and zero weight on taps 1-3.  Errors as rtlb_create. */
rtlb_status rtlb_stream_taps(const rtlb_directions *dirs, int32_t streaming, int32_t plane, int32_t *ox,
                             int32_t *oz, double *w);

/* Normalized Rayleigh table (Eq. 13-17 with Eq. 16 and the rotation of Eq. 21):
 * Z_out[4n][4n] host float64.  Block (o, i) = R(-psi_o) P~(theta) R(psi_i)
 * divided by sum_o' P~11(theta(o', i)); psi is the angle between the local
 * meridian plane and the scattering plane.  depol in [0, 0.5): molecular
 * depolarization factor (Hansen & Travis 1974 form of the Rayleigh matrix; 0
 * gives Eq. 16 exactly); otherwise RTLB_E_RANGE. */
rtlb_status rtlb_phase_rayleigh(const rtlb_directions *dirs, double depol, double *Z_out);

/* Intensity-conserving correction of a normalized table Z[4n][4n] (host,
 * in place): on a discrete angular grid the I rows of the Q, U, V columns do
 * not sum to zero, so polarized light changes the total intensity even at
 * albedo 1; each such I-row entry Z(o, i)_{I,k} loses Z(o, i)_{I,I} times its
 * column sum, which makes the sums vanish and keeps sum_o Z_{I,I} = 1. */
rtlb_status rtlb_phase_conserve_intensity(int32_t n, double *Z_inout);

/* Henyey-Greenstein weighted Mueller table for cloud cells: HG(theta; g) times
 * [[1,p,0,0],[p,1,0,0],[0,0,q,0],[0,0,0,q]], p = pol_amp sin^2(theta),
 * q = sqrt(1 - p^2), rotated and normalized as above.  dZdg_out (optional,
 * may be NULL) receives the derivative of the normalized table in g. */
rtlb_status rtlb_phase_hg(const rtlb_directions *dirs, double g, double pol_amp,
                          double *Z_out, double *dZdg_out);

/* Gradient of a loss with respect to the asymmetry g of the table above
 * (Eq. 13-17 differentiated in g): dL_dg = sum over entries of
 * grad_Z[4n][4n] * dZ/dg, where grad_Z (host float64) is dL/dZ of that class
 * as rtlb_adjoint returns it; summed in entry order, so identical inputs give
 * identical bits.  Errors as rtlb_phase_hg; grad_Z and dL_dg must be non-NULL. */
rtlb_status rtlb_phase_hg_grad(const rtlb_directions *dirs, double g, double pol_amp,
                               const double *grad_Z, double *dL_dg);

/* Mixture table m * Rayleigh + (1 - m) * HG(g, pol_amp), both normalized as
 * above (so the mixture's weights also sum to one); 0 <= m <= 1. */
rtlb_status rtlb_phase_mix(const rtlb_directions *dirs, double m, double g, double pol_amp,
                           double *Z_out);

#ifdef __cplusplus
}
#endif
#endif /* RTLB_H */
