/*
 * CPU ORACLE for the matrix-free rectangular-prism gravity operator.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load or call this file.  The
 * CUDA library never links, includes or calls it, and it shares no code,
 * header, table or constant generator with the CUDA path.
 *
 * What it computes, in plain FP64, one prism at a time (8 corner terms per
 * cell, no node sharing, no blocking, no fusion):
 *
 *   Eq. 2-3   Psi(x,y,z) = z*atan(x*y/(z*R)) - x*ln(R+y) - y*ln(R+x),
 *             R = sqrt(x^2+y^2+z^2), coordinates = prism vertex minus station.
 *   Eq. 1     dg = gamma*rho * sum_{p,q,r in {1,2}} (-1)^(p+q+r) Psi(x_p,y_q,z_r)
 *   Eq. 4-6   d_i = sum_k G_ik rho_k   (d = G m)
 *             adjoint (G^T r)_k = sum_i G_ik r_i  (optionally times (zc_k+z0)^2)
 *             diag_i = sum_k G_ik^2 (zc_k+z0)^2 (the diagonal of G W^-2 G^T)
 *
 * Readings of points the paper leaves open (Section 2.1 and Section 2.3):
 *   - z is depth, positive down; index 1 is the lower coordinate of each
 *     pair, so the parity sum is positive for a positive contrast below the
 *     station (g_z reported positive down).
 *   - gamma = 6.67430e-11 m^3 kg^-1 s^-2 (CODATA 2018; the paper names gamma
 *     but prints no value).  Output unit mGal (1 mGal = 1e-5 m/s^2).
 *   - "singularity-robust formulation" (Section 2.3, unspecified) is read as
 *     the exact identity R + y = (x^2 + z^2)/(R - y), used whenever y < 0 so
 *     that ln(R+y) never suffers cancellation (same for R + x), plus the
 *     limits x*ln(.) -> 0 at x = 0, y*ln(.) -> 0 at y = 0, z*atan(.) -> 0 at
 *     z = 0 and Psi(0,0,0) = 0.
 *
 * Parity pins (tests/test_oracle_pins.py) tie this code to things it does not
 * share: the point-mass limit, an independent Gauss-Legendre Newton
 * integral, the on-axis solid-angle closed form (and its Bouguer-slab limit),
 * superposition, symmetry, z-mirror, finite-difference check of the mixed
 * third derivative of Psi, the exact transpose, and the x/y edge assignment
 * and cell ordering k = i + nx (j + ny l), one cell at a time on a mesh with
 * nx != ny and unequal spacings against the Newton integral of that cell's box.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_GAMMA 6.67430e-11
#define ORACLE_SI_TO_MGAL 1.0e5

static int g_threads = 0;

void oracle_set_threads(int n) { g_threads = n; }

int oracle_get_threads(void) {
#ifdef _OPENMP
    return g_threads > 0 ? g_threads : omp_get_max_threads();
#else
    return 1;
#endif
}

double oracle_gamma(void) { return ORACLE_GAMMA; }

/* ln(R + a) with the cancellation-free form when a < 0; b2 = sum of the
 * squares of the two other coordinates (R^2 - a^2). */
static double log_R_plus(double R, double a, double b2) {
    if (a >= 0.0) return log(R + a);
    return log(b2 / (R - a));
}

/* Eq. 2 with R from Eq. 3. */
double oracle_psi(double x, double y, double z) {
    double x2 = x * x, y2 = y * y, z2 = z * z;
    double R = sqrt(x2 + y2 + z2);
    if (R == 0.0) return 0.0;
    double t_atan = 0.0, t_lx = 0.0, t_ly = 0.0;
    if (z != 0.0) t_atan = z * atan((x * y) / (z * R));
    if (x != 0.0) t_lx = x * log_R_plus(R, y, x2 + z2);
    if (y != 0.0) t_ly = y * log_R_plus(R, x, y2 + z2);
    return t_atan - t_lx - t_ly;
}

/* Eq. 1 without gamma*rho: sum over the 8 vertices of the prism
 * [x1,x2] x [y1,y2] x [z1,z2] (station at the origin) with parity sign
 * (-1)^(p+q+r), p = 1 for x1 and p = 2 for x2 (same for q, r). */
double oracle_prism(double x1, double x2, double y1, double y2, double z1, double z2) {
    const double xs[2] = {x1, x2}, ys[2] = {y1, y2}, zs[2] = {z1, z2};
    double s = 0.0;
    for (int p = 1; p <= 2; ++p)
        for (int q = 1; q <= 2; ++q)
            for (int r = 1; r <= 2; ++r) {
                double sigma = ((p + q + r) % 2 == 0) ? 1.0 : -1.0;
                s += sigma * oracle_psi(xs[p - 1], ys[q - 1], zs[r - 1]);
            }
    return s;
}

/* G_ik in mGal per (kg/m^3): prism (i_x, j_y, l_z) seen from station s. */
static double g_entry(const double *xe, const double *ye, const double *ze,
                      int i, int j, int l, double sx, double sy, double sz) {
    return ORACLE_GAMMA * ORACLE_SI_TO_MGAL *
           oracle_prism(xe[i] - sx, xe[i + 1] - sx,
                        ye[j] - sy, ye[j + 1] - sy,
                        ze[l] - sz, ze[l + 1] - sz);
}

/* Eq. 5-6: d = G m.  m has nx*ny*nz entries, k = i + nx*(j + ny*l). */
void oracle_forward(int nx, int ny, int nz, const double *xe, const double *ye,
                    const double *ze, int n, const double *sx, const double *sy,
                    const double *sz, const double *m, double *d) {
    int nt = oracle_get_threads();
    (void)nt;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (int s = 0; s < n; ++s) {
        double acc = 0.0;
        for (int l = 0; l < nz; ++l)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    size_t k = (size_t)i + (size_t)nx * ((size_t)j + (size_t)ny * l);
                    if (m[k] == 0.0) continue;
                    acc += g_entry(xe, ye, ze, i, j, l, sx[s], sy[s], sz[s]) * m[k];
                }
        d[s] = acc;
    }
}

/* Depth weight squared W^-2 = (zc + z0)^2, zc = cell-centre depth below the
 * mesh top (reading of the paper's Li & Oldenburg depth weighting, Section 2.2). */
static double depth_w2(const double *ze, int l, double z0) {
    double zc = 0.5 * (ze[l] + ze[l + 1]) - ze[0];
    return (zc + z0) * (zc + z0);
}

/* (G^T r)_k, times (zc_k + z0)^2 when depth_weighted != 0. */
void oracle_adjoint(int nx, int ny, int nz, const double *xe, const double *ye,
                    const double *ze, int n, const double *sx, const double *sy,
                    const double *sz, const double *r, double *out,
                    int depth_weighted, double z0) {
    int nt = oracle_get_threads();
    (void)nt;
    long long M = (long long)nx * ny * nz;
#pragma omp parallel for schedule(dynamic, 64) num_threads(nt)
    for (long long k = 0; k < M; ++k) {
        int i = (int)(k % nx);
        int j = (int)((k / nx) % ny);
        int l = (int)(k / ((long long)nx * ny));
        double acc = 0.0;
        for (int s = 0; s < n; ++s) {
            if (r[s] == 0.0) continue;
            acc += g_entry(xe, ye, ze, i, j, l, sx[s], sy[s], sz[s]) * r[s];
        }
        out[k] = depth_weighted ? acc * depth_w2(ze, l, z0) : acc;
    }
}

/* Explicit dense G, row-major [n][M]. */
void oracle_G(int nx, int ny, int nz, const double *xe, const double *ye,
              const double *ze, int n, const double *sx, const double *sy,
              const double *sz, double *G) {
    int nt = oracle_get_threads();
    (void)nt;
    long long M = (long long)nx * ny * nz;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (int s = 0; s < n; ++s)
        for (int l = 0; l < nz; ++l)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    long long k = i + (long long)nx * (j + (long long)ny * l);
                    G[(long long)s * M + k] = g_entry(xe, ye, ze, i, j, l, sx[s], sy[s], sz[s]);
                }
}

/* diag_i = sum_k G_ik^2 (zc_k + z0)^2 : diagonal of G W^-2 G^T. */
void oracle_diag(int nx, int ny, int nz, const double *xe, const double *ye,
                 const double *ze, int n, const double *sx, const double *sy,
                 const double *sz, double z0, double *diag) {
    int nt = oracle_get_threads();
    (void)nt;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (int s = 0; s < n; ++s) {
        double acc = 0.0;
        for (int l = 0; l < nz; ++l) {
            double w2 = depth_w2(ze, l, z0);
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    double g = g_entry(xe, ye, ze, i, j, l, sx[s], sy[s], sz[s]);
                    acc += g * g * w2;
                }
        }
        diag[s] = acc;
    }
}
