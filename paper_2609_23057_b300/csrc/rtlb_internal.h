// Internal declarations shared by the library's translation units.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/rtlb.h"

namespace rtlb {

// ---- host geometry / tables (phase.cpp) ----
void direction_grid(int n_zen, int n_az, std::vector<double> &mu, std::vector<double> &phi);
void lattice_projection(double mu, double phi, int plane, double *px, double *pz);
int stream_offset(double mu, double phi, int plane, int *cx, int *cz);  // 1 = tie
void bilinear_taps(double mu, double phi, int plane, int ox[4], int oz[4], double w[4], int sense[2]);
void phase_rayleigh(const std::vector<double> &mu, const std::vector<double> &phi, double rho, double *Z);
void conserve_intensity(int n, double *Z);
void phase_hg(const std::vector<double> &mu, const std::vector<double> &phi, double g,
              double pol_amp, double *Z, double *dZdg);

constexpr int kMaxPhase = 16;
constexpr int kMaxDirs = 256;

// Everything one step kernel needs, passed by value.
struct StepParams {
    const float *S;      // direction-major state [n][nsites][4], nsites = nx*nz
    float *S_new;        // same layout, the other buffer
    const float4 *coef;  // [nsites] {alpha_hi, alpha_lo, beta, emission}
    const uint8_t *cls;  // [nsites] phase class
    const float *ZT;     // [n_phase][4n (k)][4n (col)] float32, Z transposed
    const int *dir;      // [2n] cx then cz
    const float *inflow; // [4 sides][n][4]
    int nx, nz, n, n_phase;
    int bc[4];           // top, bottom, left, right
    // optional: restrict the step to listed tiles of tile_span sites
    const int *tile_list = nullptr;
    int n_tiles = 0, tile_span = 0;
    // optional (bilinear streaming, gather form): S holds the post-collision
    // field P of the step before, and the operand S~ is gathered from its four
    // taps while loading (taps_o [n][8] int, taps_w [n][4] float)
    const int *taps_o = nullptr;
    const float *taps_w = nullptr;
};

// Everything one adjoint step needs (see adjoint.cu).
struct AdjointParams {
    const float *lam_next;  // lambda^{t+1}, direction-major
    float *lam_out;         // lambda^t
    float *beta_mu;         // beta * mu, input of the table-gradient GEMM
    const float *S;         // S^t
    const float4 *coef;
    const uint8_t *cls;
    const float *Z;         // [n_phase][4n][4n] row-major float32 (untransposed)
    const int *dir;
    int nx, nz, n, n_phase;
    int bc[4];
    double *g_alpha, *g_beta;  // [2][nsites] accumulated over the steps (two halves, summed by the chain rule)
    // transposed-stream form (4n = 128): tile list of the CUDA-core kernel,
    // negated offsets and boundary kinds of the push of T^T, push or store in
    // place; the table gradient multiplies its input by beta when beta_scale
    const int *tiles = nullptr;
    const int *dirT = nullptr;
    int bcbitsT = 0;
    int push = 1;
    int beta_scale = 0;
    // class mask of each 32-site chunk (bit c: a site of class c), for the
    // tensor-core table gradient (launch_adjoint_chunk_masks)
    const uint32_t *chunk_mask = nullptr;
    // float32 partial of each CTA of the tensor-core table gradient
    // ([adjoint_table_slots()][n_phase][4n][4n]) and the running sum over the
    // steps as float32 pairs (hi [n_phase][4n][4n], then lo)
    float *table_part = nullptr;
    float *table_acc = nullptr;
};

bool adjoint_supported(int n);
int adjoint_table_slots();
cudaError_t launch_adjoint_step(const AdjointParams &p, double *slots, cudaStream_t s);
cudaError_t launch_adjoint_seed(float *lam, const float *dL_dout, const int *dir, int nx, int nz, int n, cudaStream_t s);
cudaError_t launch_adjoint_chain(const double *ga, const double *gb, const float *tau, const float *alb, int nsites,
                                 int surv_mode, int abs_mode, float *g_tau, float *g_alb, cudaStream_t s);
cudaError_t launch_adjoint_fold(const double *slots, int nslots, size_t len, double *out, cudaStream_t s);
// transposed-stream form (4n = 128): CUDA-core reverse step over the listed
// tiles (p.tiles, n_tiles of them), the table gradient alone, and the seed
// nu^{N-1} = T^T lambda^N
cudaError_t launch_adjoint_step_nu_mixed(const AdjointParams &p, int n_tiles, cudaStream_t s);
cudaError_t launch_adjoint_table(const AdjointParams &p, double *slots, cudaStream_t s);
cudaError_t launch_adjoint_seed_nu(float *nu, const float *dL_dout, const int *dir, int nx, int nz, int n, int bcbits,
                                   cudaStream_t s);
// tensor-core table gradient (adj_table_tc.cu): 4n <= 128, n_phase * 4n <= 512
bool adjoint_table_tc_supported(int n, int n_phase);
cudaError_t launch_adjoint_table_tc(const AdjointParams &p, double *slots, int nslots, cudaStream_t s);
cudaError_t launch_adjoint_chunk_masks(const uint8_t *cls, int nsites, uint32_t *masks, cudaStream_t s);
// slot0[j] += hi[j] + lo[j] (float64) from the running sum of the tensor-core table gradient
cudaError_t launch_adjoint_table_tc_finish(const float *acc, int len, double *slot0, cudaStream_t s);
size_t adjoint_chunk_masks_bytes(int nsites);
int adjoint_table_tc_take_error();

// ---- kernels (launchers return the launch error) ----
cudaError_t launch_user_to_dm(const float *user, float *dm, int nsites, int n, cudaStream_t s);
cudaError_t launch_dm_to_user(const float *dm, float *user, int nsites, int n, cudaStream_t s);
cudaError_t launch_prep_medium(const float *tau, const float *albedo, const float *emis,
                               const uint8_t *cls_in, float4 *coef, uint8_t *cls_out, int nsites,
                               int n_phase, int surv_mode, int abs_mode, int *flags, cudaStream_t s);
cudaError_t launch_step_fp32(const StepParams &p, cudaStream_t s);
cudaError_t launch_residual(const float *a, const float *b, size_t count, double *partials,
                            int nblocks, double *out2, cudaStream_t s);
int residual_blocks(size_t count);
cudaError_t launch_total_I(const float *dm, size_t nvec, double *partials, int nblocks,
                           double *out, cudaStream_t s);
cudaError_t launch_radiance_out(const float *dm, float *out, int nx, int nz, int n,
                                const int *dir, int side, cudaStream_t s);
cudaError_t launch_dop_out(const float *dm, float *out, int nx, int nz, int n, const int *dir, int side,
                           cudaStream_t s);
cudaError_t launch_fill(float *p, size_t count, float v, cudaStream_t s);
// bilinear streaming (k_stream.cu): S(x, d) = sum_k w[d][k] P(x - o[d][k], d) with
// the ghost rule of the boundary kinds; taps_o = [n][8] (ox0..3, oz0..3), taps_w = [n][4]
cudaError_t launch_stream_bilinear(const float *P, float *S, const int *taps_o, const float *taps_w,
                                   const float *inflow, int nx, int nz, int n, int bcbits, cudaStream_t s);

}  // namespace rtlb

namespace rtlb {
// Grow-only device buffer: kept between calls, reallocated only when a call
// needs more than it holds.
struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
    cudaError_t ensure(size_t bytes);
    void release();
    template <class T>
    T *as() const { return static_cast<T *>(p); }
};

// rtlb_adjoint's device workspace (checkpoints, scratch states, adjoint
// states, accumulators and staging), kept in the context between calls.
struct AdjWork {
    DevBuf ck, seg, lam, bm, ga, gb, slots, G, tapT, dl, gtd, gad, gS, cmask, tpart, tacc;
    void release()
    {
        for (DevBuf *b : {&ck, &seg, &lam, &bm, &ga, &gb, &slots, &G, &tapT, &dl, &gtd, &gad, &gS, &cmask, &tpart, &tacc}) b->release();
    }
};

// Tensor-core reverse step state (4n in {32, 64, 128}), built from the medium on the
// first rtlb_adjoint after each rtlb_set_medium: Z^T as bf16 hi and lo with
// their tensor maps, single-class and mixed 128-site tile lists, and the
// negated streaming offsets.
struct AdjTcState {
    DevBuf zhi, zlo, pure, mixed, dirT;
    int n_pure = 0, n_mixed = 0;
    CUtensorMap tmZhi{}, tmZlo{};
    long long gen = -1;                    // medium generation it was built for
    void release()
    {
        for (DevBuf *b : {&zhi, &zlo, &pure, &mixed, &dirT}) b->release();
        gen = -1;
    }
};
}  // namespace rtlb

struct rtlb_ctx {
    int dev = 0;
    int nx = 0, nz = 0, n = 0, n_zen = 0, n_az = 0;
    std::vector<double> mu, phi;
    std::vector<int> cx, cz;      // NEAREST8: offsets; BILINEAR: sense of motion (sign of l)
    std::vector<int> tap_o;       // [n][8] ox0..3, oz0..3 (BILINEAR)
    std::vector<float> tap_w;     // [n][4]
    rtlb_options opt{};
    int bc[4] = {0, 0, 0, 0};
    std::vector<float> inflow;  // [4][n][4]

    // device buffers
    float *S[2] = {nullptr, nullptr};  // direction-major [n][nsites][4]
    int cur = 0;
    int *d_dir = nullptr;         // [2n] cx then cz (see cx, cz above)
    int *d_dir0 = nullptr;        // [2n] zeros: the collision pass of BILINEAR streaming
    int *d_tap_o = nullptr;
    float *d_tap_w = nullptr;
    float *d_post = nullptr;      // BILINEAR: post-collision field before streaming
    float *d_inflow = nullptr;
    float4 *d_coef = nullptr;
    uint8_t *d_cls = nullptr;
    float *d_ZT = nullptr;
    float *d_Z = nullptr;         // untransposed float32 tables (adjoint)
    float *d_tau = nullptr;       // medium kept for the adjoint's chain rule
    float *d_alb = nullptr;
    int n_phase = 0;
    bool medium_set = false;
    double *d_scratch = nullptr;  // reduction partials
    int scratch_len = 0;
    double *d_out = nullptr;      // small device results
    int *d_flags = nullptr;
    double *h_out = nullptr;      // pinned host results
    int *h_flags = nullptr;
    float *d_stage = nullptr;     // user-layout staging for host transfers
    float *d_rad = nullptr;       // radiance_out staging for host transfers
    void *tc = nullptr;           // tensor-core path state (tc.cu)
    rtlb::AdjWork adj;            // rtlb_adjoint workspace (grow-only)
    rtlb::AdjTcState adj_tc;      // tensor-core reverse step tables and tile lists
    long long medium_gen = 0;     // counts rtlb_set_medium calls

    int64_t steps = 0;
    bool has_prev = false;
    // bilinear streaming in the gather form: each step reads the previous
    // step's post-collision field P and gathers its streaming while loading,
    // so the streaming of the last step is deferred -- S[cur] then holds that
    // step's P, and the state S^t is its gather (api.cu: state_view, settle)
    bool deferred = false;
    bool prev_deferred = false;   // the same for S[cur ^ 1] (the residual's previous state)
    bool view_valid = false;      // d_post holds the gather of S[cur]
    std::string err;

    size_t nsites() const { return (size_t)nx * nz; }
    size_t state_floats() const { return nsites() * n * 4; }
};
