// Host-side (float64) geometry and phase-matrix tables of the library.
//
// Angular grid (Sec. 2.1): n = n_zen x n_az directions with equal quadrature
// weights 4 pi / n; the uniform grid uses equal solid-angle zenith bins (cell
// midpoints in mu) and equally spaced azimuths.
//
// Redistribution table (Eq. 13-17, 21-25): block (o, i) maps the Stokes vector
// of incoming direction i, referred to its meridian plane, to outgoing
// direction o: rotate into the scattering plane, apply the single-scattering
// Mueller matrix at the scattering angle, rotate back into the outgoing
// meridian plane.  The frame angle psi is the angle between the meridian plane
// and the scattering plane; the block is divided by the sum over outgoing
// directions of its (1,1) element, so the weights of Eq. 17 sum to one.
#include <cmath>
#include <cstring>
#include <vector>

#include "rtlb_internal.h"

namespace rtlb {

static const double kPi = 3.14159265358979323846;

void direction_grid(int n_zen, int n_az, std::vector<double> &mu, std::vector<double> &phi)
{
    const int n = n_zen * n_az;
    mu.assign(n, 0.0);
    phi.assign(n, 0.0);
    for (int d = 0; d < n; ++d) {
        const int iz = d / n_az, ia = d % n_az;
        mu[d] = (2.0 * iz + 1.0 - n_zen) / n_zen;
        phi[d] = (2.0 * kPi / n_az) * ia;
    }
}

void lattice_projection(double mu, double phi, int plane, double *px, double *pz)
{
    const double st = std::sqrt(std::fmax(0.0, 1.0 - mu * mu));
    *px = st * std::cos(phi);
    *pz = plane == RTLB_PLANE_XY ? st * std::sin(phi) : mu;
}

// Nearest D2Q9 offset by angle, found by folding the projection into the first
// octant: the smaller-over-larger component angle delta in [0, 45] deg picks an
// axis offset (delta < 22.5) or a diagonal one (delta > 22.5).
int stream_offset(double mu, double phi, int plane, int *cx, int *cz)
{
    double px, pz;
    lattice_projection(mu, phi, plane, &px, &pz);
    const double ax = std::fabs(px), az = std::fabs(pz);
    if (std::sqrt(ax * ax + az * az) < 1e-12) {
        *cx = 0;
        *cz = 0;
        return 0;
    }
    const double delta = std::atan2(std::fmin(ax, az), std::fmax(ax, az));  // [0, pi/4]
    const double half = kPi / 8.0;
    if (std::fabs(delta - half) < (kPi / 4.0) * 1e-9) return 1;  // between two offsets
    const int sx = px > 0 ? 1 : (px < 0 ? -1 : 0);
    const int sz = pz > 0 ? 1 : (pz < 0 ? -1 : 0);
    if (delta > half) {
        *cx = sx;
        *cz = sz;
    } else if (ax >= az) {
        *cx = sx;
        *cz = 0;
    } else {
        *cx = 0;
        *cz = sz;
    }
    return 0;
}

// Semi-Lagrangian taps: per axis the displacement l (snapped to an integer
// when within 1e-12 of one) splits into n0 = floor(l) and f = l - n0; the two
// axis stencils {n0: 1 - f, n0 + 1: f} multiply into four taps, b_x fastest.
void bilinear_taps(double mu, double phi, int plane, int ox[4], int oz[4], double w[4], int sense[2])
{
    double l[2];
    lattice_projection(mu, phi, plane, &l[0], &l[1]);
    int n0[2];
    double f[2];
    for (int a = 0; a < 2; ++a) {
        const double r = std::nearbyint(l[a]);
        if (std::fabs(l[a] - r) < 1e-12) l[a] = r;
        n0[a] = (int)std::floor(l[a]);
        f[a] = l[a] - n0[a];
        sense[a] = l[a] > 0.0 ? 1 : (l[a] < 0.0 ? -1 : 0);
    }
    for (int k = 0; k < 4; ++k) {
        const int bx = k & 1, bz = k >> 1;
        ox[k] = n0[0] + bx;
        oz[k] = n0[1] + bz;
        w[k] = (bx ? f[0] : 1.0 - f[0]) * (bz ? f[1] : 1.0 - f[1]);
    }
}

namespace {

struct Vec3 {
    double x, y, z;
};
inline Vec3 cross(const Vec3 &a, const Vec3 &b)
{
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
inline double dot(const Vec3 &a, const Vec3 &b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

struct Dir {
    Vec3 om, par, per;  // propagation, meridian-plane axis, azimuthal axis
};

Dir make_dir(double mu, double phi)
{
    const double st = std::sqrt(std::fmax(0.0, 1.0 - mu * mu));
    const double c = std::cos(phi), s = std::sin(phi);
    return {{st * c, st * s, mu}, {mu * c, mu * s, -st}, {-s, c, 0.0}};
}

// cos(2 psi), sin(2 psi) of the frame angle from the meridian axis to the
// scattering-plane axis n x omega (measured towards the azimuthal axis).
void frame_cs(const Vec3 &nrm, const Dir &d, double *c2, double *s2)
{
    const Vec3 p = cross(nrm, d.om);
    const double c = dot(p, d.par), s = dot(p, d.per);
    *c2 = c * c - s * s;
    *s2 = 2.0 * s * c;
}

// Single-scattering matrix in the scattering plane, stored as its distinct
// entries: [[a,b,0,0],[b,a2,0,0],[0,0,cu,0],[0,0,0,cv]].
struct Scat {
    double a, b, a2, cu, cv;
};

// Rayleigh matrix with molecular depolarization rho in the normalization of
// Eq. 16's P~ (Hansen & Travis 1974): the anisotropic part is weighted by
// D = (1 - rho) / (1 + rho / 2), an isotropic (2/3)(1 - D) joins the (1,1)
// element, and circular polarization is further reduced by
// D' = (1 - 2 rho) / (1 - rho).  rho = 0 is Eq. 16.
Scat rayleigh(double ct, double rho)
{
    const double c2 = ct * ct;
    const double D = (1.0 - rho) / (1.0 + 0.5 * rho);
    const double Dv = D * (1.0 - 2.0 * rho) / (1.0 - rho);
    const double an = 0.5 * D * (1.0 + c2);
    return {an + (2.0 / 3.0) * (1.0 - D), -0.5 * D * (1.0 - c2), an, D * ct, Dv * ct};
}

double hg_phase(double ct, double g) { return (1.0 - g * g) / std::pow(1.0 + g * g - 2.0 * g * ct, 1.5); }

double hg_phase_dg(double ct, double g)
{
    const double den = 1.0 + g * g - 2.0 * g * ct;
    return -2.0 * g / std::pow(den, 1.5) - 1.5 * (1.0 - g * g) * (2.0 * g - 2.0 * ct) / std::pow(den, 2.5);
}

// Rotated block M = R(-psi_o) S R(psi_i), written out entry by entry for the
// structure of S (only the I/Q and Q/U couplings rotate; V passes through).
void rotated_block(const Scat &S, double ci, double si, double co, double so, double M[16])
{
    M[0] = S.a;
    M[1] = S.b * ci;
    M[2] = S.b * si;
    M[3] = 0.0;
    M[4] = co * S.b;
    M[5] = co * S.a2 * ci + so * S.cu * si;
    M[6] = co * S.a2 * si - so * S.cu * ci;
    M[7] = 0.0;
    M[8] = so * S.b;
    M[9] = so * S.a2 * ci - co * S.cu * si;
    M[10] = so * S.a2 * si + co * S.cu * ci;
    M[11] = 0.0;
    M[12] = 0.0;
    M[13] = 0.0;
    M[14] = 0.0;
    M[15] = S.cv;
}

enum Kind { kRayleigh, kHG };

// Fills the un-normalized blocks (and optionally their g-derivative, HG only),
// then normalizes each incoming column.
void build_table(const std::vector<double> &mu, const std::vector<double> &phi, Kind kind,
                 double g, double pol_amp, double rho, double *Z, double *dZ)
{
    const int n = (int)mu.size();
    const size_t K = 4 * (size_t)n;
    std::vector<Dir> dirs(n);
    for (int d = 0; d < n; ++d) dirs[d] = make_dir(mu[d], phi[d]);
    std::vector<double> colsum(n, 0.0), colsum_dg(n, 0.0);
    std::vector<double> unit(16 * (size_t)n * n), hval((size_t)n * n), hdg((size_t)n * n);
    for (int i = 0; i < n; ++i) {
        for (int o = 0; o < n; ++o) {
            const Dir &Di = dirs[i], &Do = dirs[o];
            double ct = dot(Do.om, Di.om);
            ct = std::fmin(1.0, std::fmax(-1.0, ct));
            Vec3 nrm = cross(Di.om, Do.om);
            const double nn = std::sqrt(dot(nrm, nrm));
            double ci = 1.0, si = 0.0, co = 1.0, so = 0.0;
            if (nn > 1e-12) {
                nrm = {nrm.x / nn, nrm.y / nn, nrm.z / nn};
                frame_cs(nrm, Di, &ci, &si);
                frame_cs(nrm, Do, &co, &so);
            }
            Scat S;
            double weight, weight_dg = 0.0;
            if (kind == kRayleigh) {
                S = rayleigh(ct, rho);
                weight = S.a;
            } else {
                const double p = pol_amp * (1.0 - ct * ct);
                const double q = std::sqrt(std::fmax(0.0, 1.0 - p * p));
                S = {1.0, p, 1.0, q, q};
                weight = hg_phase(ct, g);
                weight_dg = hg_phase_dg(ct, g);
            }
            double *blk = &unit[16 * ((size_t)o * n + i)];
            rotated_block(S, ci, si, co, so, blk);
            // Rayleigh blocks carry their weight inside S (a); HG blocks are
            // the unit structure scaled by the HG phase function.
            const double scale = (kind == kRayleigh) ? 1.0 : weight;
            hval[(size_t)o * n + i] = scale;
            hdg[(size_t)o * n + i] = weight_dg;
            colsum[i] += weight;
            colsum_dg[i] += weight_dg;
        }
    }
    for (int o = 0; o < n; ++o)
        for (int i = 0; i < n; ++i) {
            const double *blk = &unit[16 * ((size_t)o * n + i)];
            const double h = hval[(size_t)o * n + i], N = colsum[i];
            for (int r = 0; r < 4; ++r)
                for (int k = 0; k < 4; ++k) {
                    const size_t idx = (4 * (size_t)o + r) * K + 4 * (size_t)i + k;
                    Z[idx] = blk[4 * r + k] * h / N;
                    if (dZ) {
                        const double hd = hdg[(size_t)o * n + i], Nd = colsum_dg[i];
                        dZ[idx] = blk[4 * r + k] * (hd / N - h * Nd / (N * N));
                    }
                }
        }
}

}  // namespace

void phase_rayleigh(const std::vector<double> &mu, const std::vector<double> &phi, double rho, double *Z)
{
    build_table(mu, phi, kRayleigh, 0.0, 0.0, rho, Z, nullptr);
}

void conserve_intensity(int n, double *Z)
{
    // Per incoming (direction, Stokes k = Q, U, V) column, remove the part of
    // the I row that does not sum to zero, in proportion to the I -> I
    // weights (which sum to one).
    const size_t K = 4 * (size_t)n;
    for (int i = 0; i < n; ++i)
        for (int k = 1; k < 4; ++k) {
            const size_t col = 4 * (size_t)i + k, col_i = 4 * (size_t)i;
            double excess = 0.0;
            for (int o = 0; o < n; ++o) excess += Z[4 * (size_t)o * K + col];
            for (int o = 0; o < n; ++o) Z[4 * (size_t)o * K + col] -= excess * Z[4 * (size_t)o * K + col_i];
        }
}

void phase_hg(const std::vector<double> &mu, const std::vector<double> &phi, double g,
              double pol_amp, double *Z, double *dZdg)
{
    build_table(mu, phi, kHG, g, pol_amp, 0.0, Z, dZdg);
}

}  // namespace rtlb
