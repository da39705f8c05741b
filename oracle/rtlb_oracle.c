/*
 * rtlb_oracle.c -- FP64 CPU oracle for the classical polarized lattice-Boltzmann
 * radiative-transfer time step of "A Quantum-Inspired Two-Dimensional Lattice
 * Polarized Radiative Transfer Simulator" (Zeng, Lin, Omar).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library.  The product path (the CUDA
 * library) shares no code with it: its own table builder, streaming rule and step
 * are written separately.  Everything here is plain, slow and in the order the
 * paper states it; OpenMP only splits the outer loop over lattice rows.
 *
 * Layouts (all row-major, double):
 *   state   S[z][x][d][s]      s = I,Q,U,V ; d = i_zen * n_az + i_az
 *   medium  tau[z][x], albedo[z][x], emis[z][x] (per-step, per-direction, I only),
 *           cls[z][x] (phase-table index)
 *   table   Z[c][4n][4n]        Z[4*o + r][4*i + k] maps incoming (i, k) -> outgoing (o, r)
 *
 * Readings of the paper fixed here (each also listed in the design notes):
 *   - directions: mu = -1 + (2 i_zen + 1)/n_zen (equal solid-angle bins, downward
 *     first), phi = 2 pi i_az / n_az, equal quadrature weights 4 pi / n
 *     (Sec. 2.1, "uniformly distributed zenith and azimuth", omega = 4 pi / n_d).
 *   - streaming offset: the nearest of the 8 D2Q9 neighbour offsets (by angle) of
 *     the (x, z) projection (sin(theta) cos(phi), mu); zero projection rests.
 *   - polarization frame angles psi_in / psi_out: the geometric angle between the
 *     local meridian plane and the scattering plane (Eq. 13 and 15; the literal
 *     azimuth form of Eq. 15 does not reproduce the single-scatter degree of
 *     polarization the paper reports in Sec. 3.2.2).
 *   - normalization (Eq. 17): each 4x4 block is divided by the column sum of the
 *     scalar phase function, so sum_o Z11(o, i) = 1.
 *   - step order: emission, absorption, scattering, streaming (Sec. 2.1, Eq. 6-11,
 *     then the propagation operator).
 *
 * parity of the D1Q2 peak values quoted in Sec. 3.1 (1.806 / 1.475): unpinned --
 * they depend on the set-up of a cited paper that is not reproduced here.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

enum { ORC_SURV_LINEAR = 0, ORC_SURV_EXP = 1 };
enum { ORC_ABS_BEER_LAMBERT = 0, ORC_ABS_TAYLOR = 1 };
enum { ORC_BC_VACUUM = 0, ORC_BC_PERIODIC = 1, ORC_BC_INFLOW = 2 };
enum { ORC_SIDE_TOP = 0, ORC_SIDE_BOTTOM = 1, ORC_SIDE_LEFT = 2, ORC_SIDE_RIGHT = 3 };
enum { ORC_PHASE_RAYLEIGH = 0, ORC_PHASE_HG = 1, ORC_PHASE_RAYLEIGH_DEPOL = 2 };
enum { ORC_PLANE_XZ = 0, ORC_PLANE_XY = 1 };

/* ------------------------------------------------------------------ geometry */

/* Uniform angular grid (Sec. 2.1; Eq. 4 text: directions equally distributed
 * over zenith and azimuth).  Equal solid-angle zenith bins, cell midpoints. */
void orc_direction_grid(int n_zen, int n_az, double *mu, double *phi)
{
    for (int iz = 0; iz < n_zen; ++iz)
        for (int ia = 0; ia < n_az; ++ia) {
            mu[iz * n_az + ia] = -1.0 + (2.0 * iz + 1.0) / n_zen;
            phi[iz * n_az + ia] = 2.0 * ORC_PI * ia / n_az;
        }
}

static void unit_vector(double mu, double phi, double v[3])
{
    double st = sqrt(fmax(0.0, 1.0 - mu * mu));
    v[0] = st * cos(phi);
    v[1] = st * sin(phi);
    v[2] = mu;
}

/* Projection of a direction onto the lattice plane.  ORC_PLANE_XZ: the lattice
 * spans x and the vertical z (the stratification axis), projection
 * (sin(theta) cos(phi), mu).  ORC_PLANE_XY: the lattice is horizontal, as in
 * the paper's 2D experiments (Sec. 3.2), projection (sin(theta) cos(phi),
 * sin(theta) sin(phi)).  The second lattice axis is called z in both cases. */
void orc_lattice_projection(double mu, double phi, int plane, double *px, double *pz)
{
    double v[3];
    unit_vector(mu, phi, v);
    *px = v[0];
    *pz = (plane == ORC_PLANE_XY) ? v[1] : v[2];
}

/* D2Q9 streaming offset of one direction (Sec. 2.1, Fig. 1b/2: propagation along
 * (-1, 0, 1) on both lattice axes): the neighbour offset nearest by angle to
 * the direction's projection on the lattice plane.  Returns 1 when the
 * projection lies exactly between two neighbour offsets (no nearest one). */
int orc_plane_offset(double mu, double phi, int plane, int *cx, int *cz)
{
    static const int ox[8] = {1, 1, 0, -1, -1, -1, 0, 1};
    static const int oz[8] = {0, 1, 1, 1, 0, -1, -1, -1};
    double px, pz;
    orc_lattice_projection(mu, phi, plane, &px, &pz);
    if (hypot(px, pz) < 1e-12) { *cx = 0; *cz = 0; return 0; }
    double t = atan2(pz, px) * (180.0 / ORC_PI) / 45.0;   /* angle in units of 45 deg */
    double f = t - floor(t);
    if (fabs(f - 0.5) < 1e-9) return 1;
    long k = (long)floor(t + 0.5);
    k = ((k % 8) + 8) % 8;
    *cx = ox[k];
    *cz = oz[k];
    return 0;
}

/* The same on the (x, z) plane. */
int orc_stream_offset(double mu, double phi, int *cx, int *cz)
{
    return orc_plane_offset(mu, phi, ORC_PLANE_XZ, cx, cz);
}

/* Semi-Lagrangian bilinear streaming (Eq. 33-34).  Over one step a direction
 * moves l = v dt / dx lattice units; with dt = dx / c (the paper's
 * dt = min(1/N_x, 1/N_y) on a unit domain) l is the direction's projection on
 * the lattice plane.  Per axis the move splits into an integer base n0 and a
 * fraction f in [0, 1): n0 = floor(l), f = l - n0 (Eq. 34 asks 0 <= f < 1,
 * which truncation towards zero would violate for l < 0).  The streamed field
 * is sum over b_x, b_z in {0, 1} of w_x(b_x) w_z(b_z) T_(n0x + b_x, n0z + b_z),
 * w(0) = 1 - f, w(1) = f, where T_c moves content by c cells (the value at x
 * comes from x - c).  A component within 1e-12 of an integer is taken as that
 * integer.  Outputs the four taps in the order (b_x, b_z) = (0,0), (1,0),
 * (0,1), (1,1) and the displacement itself. */
void orc_bilinear_taps(double mu, double phi, int plane, int ox[4], int oz[4], double w[4],
                       double *lx_out, double *lz_out)
{
    double l[2];
    orc_lattice_projection(mu, phi, plane, &l[0], &l[1]);
    int base[2];
    double frac[2];
    for (int a = 0; a < 2; ++a) {
        double r = floor(l[a] + 0.5);
        if (fabs(l[a] - r) < 1e-12) l[a] = r;
        base[a] = (int)floor(l[a]);
        frac[a] = l[a] - base[a];
    }
    for (int bz = 0; bz < 2; ++bz)
        for (int bx = 0; bx < 2; ++bx) {
            int k = 2 * bz + bx;
            ox[k] = base[0] + bx;
            oz[k] = base[1] + bz;
            w[k] = (bx ? frac[0] : 1.0 - frac[0]) * (bz ? frac[1] : 1.0 - frac[1]);
        }
    *lx_out = l[0];
    *lz_out = l[1];
}

/* ----------------------------------------------------- Mueller matrices (4x4) */

/* Stokes frame rotation, Eq. 21/22. */
void orc_rotation(double psi, double R[16])
{
    double c = cos(2.0 * psi), s = sin(2.0 * psi);
    memset(R, 0, 16 * sizeof(double));
    R[0] = 1.0;
    R[5] = c;  R[6] = s;
    R[9] = -s; R[10] = c;
    R[15] = 1.0;
}

/* Normalized Rayleigh matrix P~(theta) of Eq. 16 (without the 3/(8 pi)). */
void orc_rayleigh_matrix(double cos_t, double P[16])
{
    double a = 0.5 * (1.0 + cos_t * cos_t);
    double b = -0.5 * (1.0 - cos_t * cos_t);
    memset(P, 0, 16 * sizeof(double));
    P[0] = a;  P[1] = b;
    P[4] = b;  P[5] = a;
    P[10] = cos_t;
    P[15] = cos_t;
}

/* Henyey-Greenstein weighted Mueller matrix used for cloud cells: the HG
 * scalar phase function times [[1,p,0,0],[p,1,0,0],[0,0,q,0],[0,0,0,q]] with
 * p = pol_amp * sin^2(theta) and q = sqrt(1 - p^2).  (The paper names such
 * matrices as the extension of its Rayleigh kernel to cloud droplets.) */
void orc_hg_matrix(double cos_t, double g, double pol_amp, double P[16])
{
    double h = (1.0 - g * g) / pow(1.0 + g * g - 2.0 * g * cos_t, 1.5);
    double p = pol_amp * (1.0 - cos_t * cos_t);
    double q = sqrt(fmax(0.0, 1.0 - p * p));
    memset(P, 0, 16 * sizeof(double));
    P[0] = h;      P[1] = h * p;
    P[4] = h * p;  P[5] = h;
    P[10] = h * q;
    P[15] = h * q;
}

/* Rayleigh matrix with molecular depolarization factor rho (Hansen & Travis
 * 1974, Sec. 2): with D = (1 - rho) / (1 + rho / 2) and D' = (1 - 2 rho) /
 * (1 - rho), and in the normalization of Eq. 16's P~ (2/3 of the phase matrix
 * whose (1,1) element averages to one over the sphere),
 *   P11 = D (1 + c^2) / 2 + (2/3)(1 - D),  P12 = P21 = -D (1 - c^2) / 2,
 *   P22 = D (1 + c^2) / 2,  P33 = D c,  P44 = D D' c.
 * rho = 0 gives Eq. 16. */
void orc_rayleigh_depol_matrix(double cos_t, double rho, double P[16])
{
    double D = (1.0 - rho) / (1.0 + 0.5 * rho);
    double Dp = (1.0 - 2.0 * rho) / (1.0 - rho);
    double c2 = cos_t * cos_t;
    memset(P, 0, 16 * sizeof(double));
    P[0] = 0.5 * D * (1.0 + c2) + (2.0 / 3.0) * (1.0 - D);
    P[1] = -0.5 * D * (1.0 - c2);
    P[4] = P[1];
    P[5] = 0.5 * D * (1.0 + c2);
    P[10] = D * cos_t;
    P[15] = D * Dp * cos_t;
}

static void matmul4(const double A[16], const double B[16], double C[16])
{
    double T[16];
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            double acc = 0.0;
            for (int k = 0; k < 4; ++k) acc += A[4 * r + k] * B[4 * k + c];
            T[4 * r + c] = acc;
        }
    memcpy(C, T, sizeof(T));
}

/* Angle from the meridian-plane axis of direction (mu, phi) to the in-plane
 * axis n x Omega of the scattering plane with unit normal n, measured towards
 * the azimuthal axis (Eq. 13/15, geometric reading). */
static double frame_angle(const double nrm[3], double mu, double phi)
{
    double om[3], par[3], per[3], p[3];
    unit_vector(mu, phi, om);
    double st = sqrt(fmax(0.0, 1.0 - mu * mu));
    par[0] = mu * cos(phi); par[1] = mu * sin(phi); par[2] = -st;
    per[0] = -sin(phi);     per[1] = cos(phi);      per[2] = 0.0;
    p[0] = nrm[1] * om[2] - nrm[2] * om[1];
    p[1] = nrm[2] * om[0] - nrm[0] * om[2];
    p[2] = nrm[0] * om[1] - nrm[1] * om[0];
    double x = p[0] * par[0] + p[1] * par[1] + p[2] * par[2];
    double y = p[0] * per[0] + p[1] * per[1] + p[2] * per[2];
    return atan2(y, x);
}

/* One rotation-phase-rotation block (Eq. 13): M = R(-psi_out) P~(theta) R(psi_in),
 * theta from Eq. 14.  *w receives the scalar phase function P~11 used by the
 * Eq. 17 weights.  Parallel and antiparallel pairs take psi = 0. */
void orc_rpr_block(double mu_o, double phi_o, double mu_i, double phi_i,
                   int kind, double g, double pol_amp, double M[16], double *w)
{
    double vo[3], vi[3], n[3], P[16], Ri[16], Ro[16];
    unit_vector(mu_o, phi_o, vo);
    unit_vector(mu_i, phi_i, vi);
    double cos_t = vo[0] * vi[0] + vo[1] * vi[1] + vo[2] * vi[2];
    if (cos_t > 1.0) cos_t = 1.0;
    if (cos_t < -1.0) cos_t = -1.0;
    if (kind == ORC_PHASE_RAYLEIGH) orc_rayleigh_matrix(cos_t, P);
    else if (kind == ORC_PHASE_RAYLEIGH_DEPOL) orc_rayleigh_depol_matrix(cos_t, g, P);   /* g carries rho */
    else orc_hg_matrix(cos_t, g, pol_amp, P);
    *w = P[0];
    n[0] = vi[1] * vo[2] - vi[2] * vo[1];
    n[1] = vi[2] * vo[0] - vi[0] * vo[2];
    n[2] = vi[0] * vo[1] - vi[1] * vo[0];
    double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    double psi_i = 0.0, psi_o = 0.0;
    if (nn > 1e-12) {
        n[0] /= nn; n[1] /= nn; n[2] /= nn;
        psi_i = frame_angle(n, mu_i, phi_i);
        psi_o = frame_angle(n, mu_o, phi_o);
    }
    orc_rotation(psi_i, Ri);
    orc_rotation(-psi_o, Ro);
    double T[16];
    matmul4(P, Ri, T);
    matmul4(Ro, T, M);
}

/* Full 4n x 4n redistribution table (Eq. 13-17, 25): Z(o, i) = M(o, i) / N(i),
 * N(i) = sum_o P~11(theta(o, i)) (equal quadrature weights cancel). */
void orc_phase_table(int n, const double *mu, const double *phi,
                     int kind, double g, double pol_amp, double *Z)
{
    int K = 4 * n;
    double *wcol = (double *)calloc((size_t)n, sizeof(double));
    for (int o = 0; o < n; ++o)
        for (int i = 0; i < n; ++i) {
            double M[16], w;
            orc_rpr_block(mu[o], phi[o], mu[i], phi[i], kind, g, pol_amp, M, &w);
            wcol[i] += w;
            for (int r = 0; r < 4; ++r)
                for (int k = 0; k < 4; ++k)
                    Z[(size_t)(4 * o + r) * K + 4 * i + k] = M[4 * r + k];
        }
    for (int row = 0; row < K; ++row)
        for (int i = 0; i < n; ++i)
            for (int k = 0; k < 4; ++k)
                Z[(size_t)row * K + 4 * i + k] /= wcol[i];
    free(wcol);
}

/* Intensity-conserving variant of a normalized table: on a discrete grid the
 * Q -> I column sums sum_o Z12(o, i) are not zero, so polarized light changes
 * the total intensity at albedo 1.  Subtract Z11(o, i) * sum_o' Z12(o', i) from
 * every Z12(o, i) (and likewise for the U and V columns), which makes those
 * sums vanish while keeping sum_o Z11 = 1. */
void orc_conserve_intensity(int n, double *Z)
{
    int K = 4 * n;
    for (int i = 0; i < n; ++i)
        for (int k = 1; k < 4; ++k) {
            double sum = 0.0;
            for (int o = 0; o < n; ++o) sum += Z[(size_t)(4 * o) * K + 4 * i + k];
            for (int o = 0; o < n; ++o)
                Z[(size_t)(4 * o) * K + 4 * i + k] -= Z[(size_t)(4 * o) * K + 4 * i] * sum;
        }
}

/* ---------------------------------------------------------------- time step */

/* Post-collision state P of one site: emission (Eq. 6/8), absorption
 * (Sec. 2.1.4, Beer-Lambert or first-order Taylor), scattering (Eq. 11/12). */
static void collide_site(int n, const double *Zc, double tau, double w0, double e,
                         int surv_mode, int abs_mode, const double *S, double *P,
                         double *Se)
{
    int K = 4 * n;
    for (int j = 0; j < K; ++j) Se[j] = S[j];
    for (int d = 0; d < n; ++d) Se[4 * d] += e;                     /* emission */
    double kabs = (1.0 - w0) * tau, ksca = w0 * tau;
    double A = (abs_mode == ORC_ABS_TAYLOR) ? 1.0 - kabs : exp(-kabs);
    for (int j = 0; j < K; ++j) Se[j] *= A;                          /* absorption */
    double s = (surv_mode == ORC_SURV_EXP) ? exp(-ksca) : 1.0 - ksca;
    for (int row = 0; row < K; ++row) {                              /* scattering */
        double red = 0.0;
        for (int col = 0; col < K; ++col) red += Zc[(size_t)row * K + col] * Se[col];
        P[row] = s * Se[row] + (1.0 - s) * red;
    }
}

/* Value streamed into (x, z, d) from the upstream cell (x - cx, z - cz): interior,
 * periodic wrap ("shifts taken modulo"), or the side's ghost value (vacuum = 0,
 * inflow = the side's Stokes vector).  Ghost corners belong to the top/bottom
 * side.  Returns a pointer into P or into the inflow table, or NULL for zero. */
static const double *upstream(int nx, int nz, int n, int x, int z, int d, int cx, int cz,
                              const int *bc, const double *inflow, const double *P)
{
    int xs = x - cx, zs = z - cz;
    if (bc[ORC_SIDE_LEFT] == ORC_BC_PERIODIC) xs = ((xs % nx) + nx) % nx;
    if (bc[ORC_SIDE_TOP] == ORC_BC_PERIODIC) zs = ((zs % nz) + nz) % nz;
    int side = -1;
    if (zs >= nz) side = ORC_SIDE_TOP;
    else if (zs < 0) side = ORC_SIDE_BOTTOM;
    else if (xs < 0) side = ORC_SIDE_LEFT;
    else if (xs >= nx) side = ORC_SIDE_RIGHT;
    if (side < 0) return P + (((size_t)zs * nx + xs) * n + d) * 4;
    if (bc[side] == ORC_BC_INFLOW) return inflow + ((size_t)side * n + d) * 4;
    return NULL;
}

/* Streaming of the post-collision field P into S_out (weighted taps, see
 * orc_step). */
static void stream_all(int nx, int nz, int n, int ntap, const int *tx, const int *tz, const double *tw,
                       const int *bc, const double *inflow, const double *P, double *S_out)
{
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int x = 0; x < nx; ++x)
            for (int d = 0; d < n; ++d) {
                double *dst = S_out + (((size_t)z * nx + x) * n + d) * 4;
                for (int s = 0; s < 4; ++s) dst[s] = 0.0;
                for (int k = 0; k < ntap; ++k) {
                    int j = d * ntap + k;
                    const double *src = upstream(nx, nz, n, x, z, d, tx[j], tz[j], bc, inflow, P);
                    if (src)
                        for (int s = 0; s < 4; ++s) dst[s] += tw[j] * src[s];
                }
            }
}

/* One full step S_in -> S_out (emission, absorption, scattering, streaming).
 * Streaming of direction d is the weighted sum of ntap translations: tap k
 * moves content by (tx, tz)[d * ntap + k] cells with weight tw[d * ntap + k]
 * (one tap of weight 1 for the nearest-offset scheme, the four taps of
 * orc_bilinear_taps for the semi-Lagrangian one).  bc[4] = kinds of top,
 * bottom, left, right; periodic must be set on both sides of an axis.
 * inflow[4][n][4] holds the ghost Stokes vectors. */
void orc_step(int nx, int nz, int n, int ntap, const int *tx, const int *tz, const double *tw,
              const double *tau, const double *albedo, const double *emis, const int *cls,
              const double *Z, int surv_mode, int abs_mode, const int *bc,
              const double *inflow, const double *S_in, double *S_out)
{
    int K = 4 * n;
    size_t nsite = (size_t)nx * nz;
    double *P = (double *)malloc(nsite * K * sizeof(double));
#pragma omp parallel
    {
        double *Se = (double *)malloc((size_t)K * sizeof(double));
#pragma omp for schedule(static)
        for (int z = 0; z < nz; ++z)
            for (int x = 0; x < nx; ++x) {
                size_t st = (size_t)z * nx + x;
                const double *Zc = Z + (size_t)(cls ? cls[st] : 0) * K * K;
                collide_site(n, Zc, tau[st], albedo[st], emis ? emis[st] : 0.0,
                             surv_mode, abs_mode, S_in + st * K, P + st * K, Se);
            }
        free(Se);
    }
    stream_all(nx, nz, n, ntap, tx, tz, tw, bc, inflow, P, S_out);
    free(P);
}

/* Run nsteps steps in place on S (ping-pong through a scratch copy). */
void orc_run(int nx, int nz, int n, int ntap, const int *tx, const int *tz, const double *tw,
             const double *tau, const double *albedo, const double *emis, const int *cls,
             const double *Z, int surv_mode, int abs_mode, const int *bc,
             const double *inflow, double *S, int nsteps)
{
    size_t len = (size_t)nx * nz * n * 4;
    double *T = (double *)malloc(len * sizeof(double));
    for (int t = 0; t < nsteps; ++t) {
        orc_step(nx, nz, n, ntap, tx, tz, tw, tau, albedo, emis, cls, Z, surv_mode, abs_mode, bc,
                 inflow, S, T);
        memcpy(S, T, len * sizeof(double));
    }
    free(T);
}

/* ------------------------------------------------- FP8 block-scaled form */

/* Nearest e4m3 value of x (OCP 8-bit floating point, E4M3: 4 exponent bits
 * with bias 7, 3 mantissa bits, subnormals spaced 2^-9, largest finite value
 * 448), ties to even; larger magnitudes saturate to 448. */
double orc_e4m3(double x)
{
    double a = fabs(x);
    if (a == 0.0) return x;
    int E;
    frexp(a, &E);                       /* a in [2^(E-1), 2^E) */
    int b = E - 1;
    if (b < -6) b = -6;                 /* below the normal range the spacing stays 2^-9 */
    double q = ldexp(1.0, b - 3);       /* spacing of 3 mantissa bits in binade b */
    double r = nearbyint(a / q) * q;    /* default rounding: ties to even */
    if (r > 448.0) r = 448.0;
    return copysign(r, x);
}

/* Power-of-two block scale 2^e (UE8M0): the smallest e with amax / 2^e <= 448,
 * clamped to [-127, 127]; -127 for amax = 0 and, when fp32_floor is set, for
 * amax below the float32 normal range. */
int orc_fp8_exponent(double amax, int fp32_floor)
{
    if (!(amax > 0.0)) return -127;
    if (fp32_floor && amax < ldexp(1.0, -126)) return -127;
    int E;
    double f = frexp(amax, &E);         /* amax = (2 f) 2^(E - 1), 2 f in [1, 2) */
    int e = (E - 1) - 8 + (2.0 * f > 1.75 ? 1 : 0);
    if (e < -127) e = -127;
    if (e > 127) e = 127;
    return e;
}

/* One step in the FP8 block-scaled precision form of the contraction: an
 * emulation, in float64, of the CUDA library's FP8 precision, written from
 * that form's definition.  It reproduces the form's quantization choices (it
 * is not the paper's method: orc_step is); tests use it to check that the
 * kernel implements the form, and orc_step to measure what the form costs in
 * accuracy.  The paper fixes no low-precision arithmetic; the form is:
 *   - state operand: S~ = S + e rounded to float32 (S holds float32 values),
 *     beta rounded to float32, b = beta S~ rounded to float32; per site and
 *     block of 8 directions (32 values) the scale 2^ea from the block's
 *     largest |b| (float32 floor), each value e4m3(b 2^-ea) 2^ea;
 *   - table: for each class whose forward blocks Z(i, i) are c_i I (within
 *     1e-14 |c_i|), the float32 c_i is taken out and applied exactly, the
 *     remainder c_i - float32(c_i) staying on the diagonal; the rest of the
 *     table is quantized per row and block of 32 columns the same way (scale
 *     from the block's largest |value|, no float32 floor);
 *   - P = alpha S~ + beta c_i S~ + sum of the quantized products (exact here;
 *     the tensor core accumulates them in float32), then streaming as in
 *     orc_step.  n must be a multiple of 8. */
void orc_step_fp8(int nx, int nz, int n, int ntap, const int *tx, const int *tz, const double *tw,
                  const double *tau, const double *albedo, const double *emis, const int *cls,
                  const double *Z, int n_phase, int surv_mode, int abs_mode, const int *bc,
                  const double *inflow, const double *S_in, double *S_out)
{
    int K = 4 * n;
    size_t nsite = (size_t)nx * nz;
    double *Bq = (double *)malloc((size_t)n_phase * K * K * sizeof(double));
    double *fw = (double *)calloc((size_t)n_phase * n, sizeof(double));
    for (int c = 0; c < n_phase; ++c) {
        const double *Zc = Z + (size_t)c * K * K;
        double *B = Bq + (size_t)c * K * K;
        memcpy(B, Zc, (size_t)K * K * sizeof(double));
        int diag = 1;
        for (int i = 0; i < n && diag; ++i) {
            double ci = Zc[(size_t)(4 * i) * K + 4 * i];
            for (int a = 0; a < 4 && diag; ++a)
                for (int b = 0; b < 4; ++b) {
                    double want = (a == b) ? ci : 0.0;
                    if (fabs(Zc[(size_t)(4 * i + a) * K + 4 * i + b] - want) > 1e-14 * fabs(ci)) {
                        diag = 0;
                        break;
                    }
                }
        }
        if (diag)
            for (int i = 0; i < n; ++i) {
                double ci = Zc[(size_t)(4 * i) * K + 4 * i];
                fw[(size_t)c * n + i] = (double)(float)ci;
                for (int a = 0; a < 4; ++a) B[(size_t)(4 * i + a) * K + 4 * i + a] = ci - (double)(float)ci;
            }
        for (int row = 0; row < K; ++row)
            for (int blk = 0; blk < K / 32; ++blk) {
                double *v = B + (size_t)row * K + 32 * blk;
                double amax = 0.0;
                for (int k = 0; k < 32; ++k) amax = fmax(amax, fabs(v[k]));
                int e = orc_fp8_exponent(amax, 0);
                for (int k = 0; k < 32; ++k) v[k] = ldexp(orc_e4m3(ldexp(v[k], -e)), e);
            }
    }
    double *P = (double *)malloc(nsite * K * sizeof(double));
#pragma omp parallel
    {
        float *st = (float *)malloc((size_t)K * sizeof(float));
        double *aq = (double *)malloc((size_t)K * sizeof(double));
#pragma omp for schedule(static)
        for (int z = 0; z < nz; ++z)
            for (int x = 0; x < nx; ++x) {
                size_t site = (size_t)z * nx + x;
                int c = cls ? cls[site] : 0;
                const double *S = S_in + site * K;
                float e = (float)(emis ? emis[site] : 0.0);
                for (int k = 0; k < K; ++k) st[k] = (float)S[k];
                for (int d = 0; d < n; ++d) st[4 * d] = st[4 * d] + e;
                double t = tau[site], w = albedo[site];
                double kabs = (1.0 - w) * t, ksca = w * t;
                double A = (abs_mode == ORC_ABS_TAYLOR) ? 1.0 - kabs : exp(-kabs);
                double s = (surv_mode == ORC_SURV_EXP) ? exp(-ksca) : 1.0 - ksca;
                double alpha = A * s;
                float beta = (float)(A * (1.0 - s));
                for (int blk = 0; blk < n / 8; ++blk) {
                    float amax = 0.0f;
                    for (int k = 32 * blk; k < 32 * blk + 32; ++k) amax = fmaxf(amax, fabsf(beta * st[k]));
                    int ea = orc_fp8_exponent((double)amax, 1);
                    float inv = (float)ldexp(1.0, -ea);
                    for (int k = 32 * blk; k < 32 * blk + 32; ++k) {
                        float b = beta * st[k];
                        aq[k] = ldexp(orc_e4m3((double)(b * inv)), ea);
                    }
                }
                const double *B = Bq + (size_t)c * K * K;
                double *out = P + site * K;
                for (int row = 0; row < K; ++row) {
                    double acc = 0.0;
                    for (int k = 0; k < K; ++k) acc += B[(size_t)row * K + k] * aq[k];
                    out[row] = alpha * st[row] + (double)beta * fw[(size_t)c * n + row / 4] * st[row] + acc;
                }
            }
        free(st);
        free(aq);
    }
    stream_all(nx, nz, n, ntap, tx, tz, tw, bc, inflow, P, S_out);
    free(P);
    free(Bq);
    free(fw);
}

/* One step in the split FP8 precision form of the contraction: an
 * emulation, in float64, of the CUDA library's FP8X precision, written from
 * that form's definition (the paper fixes no low-precision arithmetic).  The
 * form, against orc_step_fp8's single e4m3 operands:
 *   - state operand: b = beta S~ as in orc_step_fp8 (float32 roundings); per
 *     site and block of 8 directions the scale 2^e0 from the block's largest
 *     |b| (float32 floor), hi term q0 = e4m3(b 2^-e0); the remainder
 *     r = b 2^-e0 - q0 (exact) gets its own scale 2^d from its block's
 *     largest |r| (float32 floor), lo term q1 = e4m3(r 2^-d); the two terms
 *     are q0 2^e0 and q1 2^(e0 + d), the lo term zero when e0 + d < -127;
 *   - table (forward blocks taken out as in orc_step_fp8): three terms per row
 *     and block of 32 columns, each e4m3 with the scale of the remainder left
 *     by the terms before it (from the block's largest |remainder|, no float32
 *     floor);
 *   - products kept: state term a times table term b for (a, b) in (0,0),
 *     (0,1), (0,2), (1,0), (1,1); the dropped (1,2) is below 2^-12 of a
 *     product.  P = alpha S~ + beta c_i S~ + their sum (exact here), then
 *     streaming as in orc_step.  n must be a multiple of 8. */
void orc_step_fp8x(int nx, int nz, int n, int ntap, const int *tx, const int *tz, const double *tw,
                   const double *tau, const double *albedo, const double *emis, const int *cls,
                   const double *Z, int n_phase, int surv_mode, int abs_mode, const int *bc,
                   const double *inflow, const double *S_in, double *S_out)
{
    int K = 4 * n;
    size_t nsite = (size_t)nx * nz;
    size_t tsz = (size_t)K * K;
    double *Bt = (double *)malloc((size_t)3 * n_phase * tsz * sizeof(double));   /* [term][class][K][K] */
    double *fw = (double *)calloc((size_t)n_phase * n, sizeof(double));
    double *rem = (double *)malloc(tsz * sizeof(double));
    for (int c = 0; c < n_phase; ++c) {
        const double *Zc = Z + (size_t)c * tsz;
        memcpy(rem, Zc, tsz * sizeof(double));
        int diag = 1;
        for (int i = 0; i < n && diag; ++i) {
            double ci = Zc[(size_t)(4 * i) * K + 4 * i];
            for (int a = 0; a < 4 && diag; ++a)
                for (int b = 0; b < 4; ++b) {
                    double want = (a == b) ? ci : 0.0;
                    if (fabs(Zc[(size_t)(4 * i + a) * K + 4 * i + b] - want) > 1e-14 * fabs(ci)) {
                        diag = 0;
                        break;
                    }
                }
        }
        if (diag)
            for (int i = 0; i < n; ++i) {
                double ci = Zc[(size_t)(4 * i) * K + 4 * i];
                fw[(size_t)c * n + i] = (double)(float)ci;
                for (int a = 0; a < 4; ++a) rem[(size_t)(4 * i + a) * K + 4 * i + a] = ci - (double)(float)ci;
            }
        for (int t = 0; t < 3; ++t) {
            double *B = Bt + ((size_t)t * n_phase + c) * tsz;
            for (int row = 0; row < K; ++row)
                for (int blk = 0; blk < K / 32; ++blk) {
                    double *r = rem + (size_t)row * K + 32 * blk;
                    double *q = B + (size_t)row * K + 32 * blk;
                    double amax = 0.0;
                    for (int k = 0; k < 32; ++k) amax = fmax(amax, fabs(r[k]));
                    int e = orc_fp8_exponent(amax, 0);
                    for (int k = 0; k < 32; ++k) {
                        q[k] = ldexp(orc_e4m3(ldexp(r[k], -e)), e);
                        r[k] -= q[k];
                    }
                }
        }
    }
    static const int pairs[5][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 0}, {1, 1}};
    double *P = (double *)malloc(nsite * K * sizeof(double));
#pragma omp parallel
    {
        float *st = (float *)malloc((size_t)K * sizeof(float));
        double *aq = (double *)malloc((size_t)2 * K * sizeof(double));   /* [term][K] */
#pragma omp for schedule(static)
        for (int z = 0; z < nz; ++z)
            for (int x = 0; x < nx; ++x) {
                size_t site = (size_t)z * nx + x;
                int c = cls ? cls[site] : 0;
                const double *S = S_in + site * K;
                float e = (float)(emis ? emis[site] : 0.0);
                for (int k = 0; k < K; ++k) st[k] = (float)S[k];
                for (int d = 0; d < n; ++d) st[4 * d] = st[4 * d] + e;
                double t = tau[site], w = albedo[site];
                double kabs = (1.0 - w) * t, ksca = w * t;
                double A = (abs_mode == ORC_ABS_TAYLOR) ? 1.0 - kabs : exp(-kabs);
                double s = (surv_mode == ORC_SURV_EXP) ? exp(-ksca) : 1.0 - ksca;
                double alpha = A * s;
                float beta = (float)(A * (1.0 - s));
                for (int blk = 0; blk < n / 8; ++blk) {
                    float amax = 0.0f;
                    for (int k = 32 * blk; k < 32 * blk + 32; ++k) amax = fmaxf(amax, fabsf(beta * st[k]));
                    int e0 = orc_fp8_exponent((double)amax, 1);
                    double r[32], rmax = 0.0;
                    for (int k = 0; k < 32; ++k) {
                        double bs = ldexp((double)(beta * st[32 * blk + k]), -e0);   /* exact scaling */
                        double q0 = orc_e4m3(bs);
                        aq[32 * blk + k] = ldexp(q0, e0);
                        r[k] = bs - q0;
                        rmax = fmax(rmax, fabs(r[k]));
                    }
                    int d = orc_fp8_exponent(rmax, 1);
                    for (int k = 0; k < 32; ++k)
                        aq[K + 32 * blk + k] = (e0 + d < -127) ? 0.0 : ldexp(orc_e4m3(ldexp(r[k], -d)), e0 + d);
                }
                double *out = P + site * K;
                for (int row = 0; row < K; ++row) {
                    double acc = 0.0;
                    for (int p = 0; p < 5; ++p) {
                        const double *B = Bt + ((size_t)pairs[p][1] * n_phase + c) * tsz + (size_t)row * K;
                        const double *a = aq + (size_t)pairs[p][0] * K;
                        for (int k = 0; k < K; ++k) acc += B[k] * a[k];
                    }
                    out[row] = alpha * st[row] + (double)beta * fw[(size_t)c * n + row / 4] * st[row] + acc;
                }
            }
        free(st);
        free(aq);
    }
    stream_all(nx, nz, n, ntap, tx, tz, tw, bc, inflow, P, S_out);
    free(P);
    free(Bt);
    free(fw);
    free(rem);
}

/* Steady-state residual: max |S_new - S_old| / max |S_new| over all entries. */
double orc_residual(size_t len, const double *S_old, const double *S_new)
{
    double dmax = 0.0, vmax = 0.0;
    for (size_t j = 0; j < len; ++j) {
        double d = fabs(S_new[j] - S_old[j]), v = fabs(S_new[j]);
        if (d > dmax) dmax = d;
        if (v > vmax) vmax = v;
    }
    return vmax > 0.0 ? dmax / vmax : dmax;
}

/* Iterate to the steady state of Eq. 1 (time derivative zero): step until the
 * residual falls below tol or max_steps is reached.  Returns steps taken. */
int orc_run_to_steady(int nx, int nz, int n, int ntap, const int *tx, const int *tz,
                      const double *tw, const double *tau, const double *albedo, const double *emis,
                      const int *cls, const double *Z, int surv_mode, int abs_mode,
                      const int *bc, const double *inflow, double *S, double tol,
                      int max_steps, double *residual)
{
    size_t len = (size_t)nx * nz * n * 4;
    double *T = (double *)malloc(len * sizeof(double));
    int t = 0;
    double r = INFINITY;
    while (t < max_steps) {
        orc_step(nx, nz, n, ntap, tx, tz, tw, tau, albedo, emis, cls, Z, surv_mode, abs_mode, bc,
                 inflow, S, T);
        r = orc_residual(len, S, T);
        memcpy(S, T, len * sizeof(double));
        ++t;
        if (r < tol) break;
    }
    free(T);
    *residual = r;
    return t;
}

/* Outgoing radiance on one side: the state on the boundary row/column for the
 * directions that move out through that side; zero for the other directions.
 * (cx, cz) is each direction's sense of motion per axis (-1, 0, +1): its
 * offset in the nearest-offset scheme, the sign of its displacement in the
 * bilinear one.  out[len][n][4], len = nx (top/bottom) or nz. */
void orc_radiance_out(int nx, int nz, int n, const int *cx, const int *cz, int side,
                      const double *S, double *out)
{
    int len = (side == ORC_SIDE_TOP || side == ORC_SIDE_BOTTOM) ? nx : nz;
    for (int p = 0; p < len; ++p)
        for (int d = 0; d < n; ++d) {
            int x, z, leaves;
            switch (side) {
            case ORC_SIDE_TOP:    x = p; z = nz - 1; leaves = cz[d] == 1; break;
            case ORC_SIDE_BOTTOM: x = p; z = 0;      leaves = cz[d] == -1; break;
            case ORC_SIDE_LEFT:   x = 0; z = p;      leaves = cx[d] == -1; break;
            default:              x = nx - 1; z = p; leaves = cx[d] == 1; break;
            }
            const double *src = S + (((size_t)z * nx + x) * n + d) * 4;
            double *dst = out + ((size_t)p * n + d) * 4;
            for (int s = 0; s < 4; ++s) dst[s] = leaves ? src[s] : 0.0;
        }
}

/* Degree of polarization, sqrt(Q^2 + U^2 + V^2) / I (Sec. 3.2.1). */
double orc_dop(const double *stokes)
{
    double I = stokes[0];
    double p = sqrt(stokes[1] * stokes[1] + stokes[2] * stokes[2] + stokes[3] * stokes[3]);
    return I != 0.0 ? p / I : 0.0;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ adjoint */

/* Derivatives of the per-site step coefficients alpha = A s, beta = A (1 - s)
 * with respect to the extinction optical depth tau and the albedo w
 * (k_abs dt = (1 - w) tau, k_scat dt = w tau; Sec. 2.1.4 and Eq. 11). */
static void coef_derivatives(double tau, double w, int surv_mode, int abs_mode, double *alpha,
                             double *beta, double *da_dt, double *da_dw, double *db_dt, double *db_dw)
{
    double kabs = (1.0 - w) * tau, ksca = w * tau;
    double A, dA, s, ds;        /* dA = dA/dkabs, ds = ds/dksca */
    if (abs_mode == ORC_ABS_TAYLOR) { A = 1.0 - kabs; dA = -1.0; }
    else { A = exp(-kabs); dA = -A; }
    if (surv_mode == ORC_SURV_EXP) { s = exp(-ksca); ds = -s; }
    else { s = 1.0 - ksca; ds = -1.0; }
    *alpha = A * s;
    *beta = A * (1.0 - s);
    /* dkabs/dtau = 1 - w, dkabs/dw = -tau, dksca/dtau = w, dksca/dw = tau */
    *da_dt = dA * (1.0 - w) * s + A * ds * w;
    *da_dw = dA * (-tau) * s + A * ds * tau;
    *db_dt = dA * (1.0 - w) * (1.0 - s) - A * ds * w;
    *db_dw = dA * (-tau) * (1.0 - s) - A * ds * tau;
}

/* Reverse-mode gradient of L = <dL_dout, radiance_out(top, S^N)> after
 * nsteps steps from S0, with respect to tau and albedo per cell, every
 * phase-table entry, and the initial state.  All intermediate states are
 * kept (small lattices only).  The step is affine,
 *   S^{t+1} = T (C S^t + c0) + b,  C = blockdiag(alpha I + beta Z_c),
 * so lambda^t = C^T T^T lambda^{t+1}; T^T pulls from each entry's streaming
 * targets with the taps' weights (zero where the content left through a
 * non-periodic side).  Taps as in orc_step; sense_z[d] = +1 marks the
 * directions that leave through the top (the radiance_out rows). */
void orc_adjoint(int nx, int nz, int n, int ntap, const int *tx, const int *tz, const double *tw,
                 const int *sense_z, const double *tau, const double *albedo, const double *emis, const int *cls,
                 const double *Z, int n_phase, int surv_mode, int abs_mode, const int *bc,
                 const double *inflow, const double *S0, int nsteps, const double *dL_dout,
                 double *grad_tau, double *grad_albedo, double *grad_Z, double *grad_S0)
{
    int K = 4 * n;
    size_t nsite = (size_t)nx * nz, len = nsite * K;
    double *states = (double *)malloc((size_t)(nsteps + 1) * len * sizeof(double));
    memcpy(states, S0, len * sizeof(double));
    for (int t = 0; t < nsteps; ++t)
        orc_step(nx, nz, n, ntap, tx, tz, tw, tau, albedo, emis, cls, Z, surv_mode, abs_mode, bc,
                 inflow, states + (size_t)t * len, states + (size_t)(t + 1) * len);
    double *lam = (double *)calloc(len, sizeof(double));
    double *mu = (double *)malloc(len * sizeof(double));
    double *ga = (double *)calloc(nsite, sizeof(double));
    double *gb = (double *)calloc(nsite, sizeof(double));
    memset(grad_Z, 0, (size_t)n_phase * K * K * sizeof(double));
    /* seed: the top row's outgoing directions */
    for (int x = 0; x < nx; ++x)
        for (int d = 0; d < n; ++d)
            if (sense_z[d] == 1)
                for (int s = 0; s < 4; ++s)
                    lam[(((size_t)(nz - 1) * nx + x) * n + d) * 4 + s] = dL_dout[((size_t)x * n + d) * 4 + s];
    int per_x = bc[ORC_SIDE_LEFT] == ORC_BC_PERIODIC, per_z = bc[ORC_SIDE_TOP] == ORC_BC_PERIODIC;
    double *Se = (double *)malloc((size_t)K * sizeof(double));
    double *ZTm = (double *)malloc((size_t)K * sizeof(double));
    for (int t = nsteps - 1; t >= 0; --t) {
        const double *St = states + (size_t)t * len;
        /* mu = T^T lambda */
        for (int z = 0; z < nz; ++z)
            for (int x = 0; x < nx; ++x)
                for (int d = 0; d < n; ++d) {
                    double *dst = mu + (((size_t)z * nx + x) * n + d) * 4;
                    for (int s = 0; s < 4; ++s) dst[s] = 0.0;
                    for (int k = 0; k < ntap; ++k) {
                        int j = d * ntap + k;
                        int xt = x + tx[j], zt = z + tz[j];
                        if (per_x) xt = ((xt % nx) + nx) % nx;
                        if (per_z) zt = ((zt % nz) + nz) % nz;
                        if (xt >= 0 && xt < nx && zt >= 0 && zt < nz)
                            for (int s = 0; s < 4; ++s)
                                dst[s] += tw[j] * lam[(((size_t)zt * nx + xt) * n + d) * 4 + s];
                    }
                }
        /* lambda = C^T mu, and the parameter gradients of this step */
        for (size_t st = 0; st < nsite; ++st) {
            int c = cls ? cls[st] : 0;
            const double *Zc = Z + (size_t)c * K * K;
            double alpha, beta, a1, a2, b1, b2;
            coef_derivatives(tau[st], albedo[st], surv_mode, abs_mode, &alpha, &beta, &a1, &a2, &b1, &b2);
            const double *m = mu + st * K;
            for (int j = 0; j < K; ++j) Se[j] = St[st * K + j];
            for (int d = 0; d < n; ++d) Se[4 * d] += emis ? emis[st] : 0.0;
            for (int k = 0; k < K; ++k) {
                double acc = 0.0;
                for (int row = 0; row < K; ++row) acc += Zc[(size_t)row * K + k] * m[row];
                ZTm[k] = acc;
            }
            double sa = 0.0, sb = 0.0;
            for (int k = 0; k < K; ++k) {
                sa += m[k] * Se[k];
                sb += ZTm[k] * Se[k];
                lam[st * K + k] = alpha * m[k] + beta * ZTm[k];
            }
            ga[st] += sa;
            gb[st] += sb;
            double *G = grad_Z + (size_t)c * K * K;
            for (int row = 0; row < K; ++row)
                for (int k = 0; k < K; ++k) G[(size_t)row * K + k] += beta * m[row] * Se[k];
        }
    }
    for (size_t st = 0; st < nsite; ++st) {
        double alpha, beta, a1, a2, b1, b2;
        coef_derivatives(tau[st], albedo[st], surv_mode, abs_mode, &alpha, &beta, &a1, &a2, &b1, &b2);
        grad_tau[st] = ga[st] * a1 + gb[st] * b1;
        grad_albedo[st] = ga[st] * a2 + gb[st] * b2;
    }
    if (grad_S0) memcpy(grad_S0, lam, len * sizeof(double));
    free(states); free(lam); free(mu); free(ga); free(gb); free(Se); free(ZTm);
}
