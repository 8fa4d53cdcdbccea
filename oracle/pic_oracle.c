/*
 * FP64 CPU oracle for the electromagnetic PIC hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * definition that the CUDA library is checked against.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it; the
 * product library never links, calls or reads anything here, and this file
 * shares no code, header or table with it.
 *
 * What it computes (the paper names the methods and gives no equations for
 * them; each function restates the cited method from its mathematics):
 *   - order-p B-spline particle shapes, p = 1..3 (3rd-order shapes are the
 *     paper's choice, Sec. 4.1.1),
 *   - momentum-conserving field gather from the staggered Yee lattice
 *     (Yee staggering: Sec. 2.4, SyncNodal paragraph),
 *   - relativistic Boris push and position advance,
 *   - Esirkepov charge-conserving current deposition (Sec. 3.4.1 and the
 *     roofline figure caption of Sec. 3.4.2 cite Esirkepov 2001),
 *   - nodal charge deposition (Sec. 3.4.1, "charge and current deposition"),
 *   - Yee FDTD E/B update with periodic boundaries (Sec. 2.4 and Sec. 4.1.1),
 *   - one full PIC step in the order gather -> push -> advance -> deposit ->
 *     field update (fused gather+push, Sec. 3.1),
 *   - reductions used as diagnostics (Sec. 2.6).
 *
 * Conventions: normalised units c = eps0 = mu0 = 1.  Node i sits at x = i*dx;
 * the grid is periodic with length L = n*dx.  Array element [i][j][k]
 * (k fastest) holds the component at its staggered location just above node
 * (i,j,k):  Ex(i+1/2,j,k) Ey(i,j+1/2,k) Ez(i,j,k+1/2)  Bx(i,j+1/2,k+1/2)
 * By(i+1/2,j,k+1/2) Bz(i+1/2,j+1/2,k);  J like E;  rho nodal.
 * Particle momenta are u = gamma*v, stored at half steps.
 *
 * Compiled with -ffp-contract=off so results do not depend on whether the
 * host compiler fuses multiply-adds.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "pic_oracle.h"

/* Mutation switch for the oracle's own self-test: the test suite rebuilds
 * this file with -DORC_MUTANT=k to plant one known mistake and checks that
 * the pins catch it.  The default build defines no mutant. */
#ifndef ORC_MUTANT
#define ORC_MUTANT 0
#endif

/* ------------------------------------------------------------------ */
/* indexing                                                            */
/* ------------------------------------------------------------------ */

static int64_t wrapi(int64_t i, int64_t n) {
    int64_t r = i % n;
    return r < 0 ? r + n : r;
}

static int64_t idx3(const orc_grid* g, int64_t i, int64_t j, int64_t k) {
    return (wrapi(i, g->n[0]) * g->n[1] + wrapi(j, g->n[1])) * g->n[2] + wrapi(k, g->n[2]);
}

/* With z open, a node outside [0, nz) along z holds no field and takes no current. */
static int outside(const orc_grid* g, int64_t k) { return g->zopen && (k < 0 || k >= g->n[2]); }

static double fetch(const orc_grid* g, const double* F, int64_t i, int64_t j, int64_t k) {
    return outside(g, k) ? 0.0 : F[idx3(g, i, j, k)];
}

static void add_to(const orc_grid* g, double* F, int64_t i, int64_t j, int64_t k, double v) {
    if (!outside(g, k)) F[idx3(g, i, j, k)] += v;
}

/* Staggering (in units of the cell size) of each field component along
 * each axis: rows Ex Ey Ez Bx By Bz. */
static const double STAG[6][3] = {
    {0.5, 0.0, 0.0}, {0.0, 0.5, 0.0}, {0.0, 0.0, 0.5},
    {0.0, 0.5, 0.5}, {0.5, 0.0, 0.5}, {0.5, 0.5, 0.0},
};

/* ------------------------------------------------------------------ */
/* shapes: cardinal B-splines                                          */
/* ------------------------------------------------------------------ */

/* s_p(xi): the order-p cardinal B-spline (the (p+1)-fold convolution of the
 * unit box), centred on 0, support |xi| < (p+1)/2; p = 0 is the unit box on
 * [-1/2, 1/2) (used by the energy-conserving gather at order 1). */
double orc_shape(int p, double xi) {
    if (p == 0) return (xi >= -0.5 && xi < 0.5) ? 1.0 : 0.0; /* the unit box, half-open */
    double a = fabs(xi);
    switch (p) {
    case 1:
        return a < 1.0 ? 1.0 - a : 0.0;
    case 2:
        if (a <= 0.5) return 0.75 - a * a;
        if (a < 1.5) { double t = 1.5 - a; return 0.5 * t * t; }
        return 0.0;
    case 3:
        if (a <= 1.0) {
#if ORC_MUTANT == 1
            return (4.0 - 6.0 * a * a + 3.0 * a * a * a) / 6.0 + 1e-3 * a * a * (1.0 - a); /* planted: wrong inner piece */
#else
            return (4.0 - 6.0 * a * a + 3.0 * a * a * a) / 6.0;
#endif
        }
        if (a < 2.0) { double t = 2.0 - a; return t * t * t / 6.0; }
        return 0.0;
    default:
        return 0.0;
    }
}

/* ------------------------------------------------------------------ */
/* gather                                                              */
/* ------------------------------------------------------------------ */

/* Momentum-conserving gather: every component is interpolated with the
 * order-p shape along all three axes at its own staggered location,
 *   F_c(x) = sum_{ijk} s_p(x/dx - i - dx_c) s_p(y/dy - j - dy_c) s_p(z/dz - k - dz_c) F_c[ijk].
 * The node ranges below cover the support with room to spare; nodes outside
 * the support contribute exactly zero. */
static void gather_orders(const orc_grid* g, int p, int energy, const double* const F[6], double x, double y,
                          double z, double EB[6]) {
    enum { NR = 8 };
    const double pos[3] = {x / g->d[0], y / g->d[1], z / g->d[2]};
    for (int c = 0; c < 6; ++c) {
        /* per axis: the first node of a range that covers the support, and the weights on it */
        int64_t first[3];
        double wt[3][NR];
        for (int a = 0; a < 3; ++a) {
#if ORC_MUTANT == 2
            const double sh = pos[a] - (c == 0 && a == 0 ? 0.0 : STAG[c][a]); /* planted: Ex not staggered */
#else
            const double sh = pos[a] - STAG[c][a];
#endif
#if ORC_MUTANT == 9
            const int order = (energy && STAG[c][a] != 0.0 && c != 1) ? p - 1 : p; /* planted: E_y keeps order p */
#else
            const int order = (energy && STAG[c][a] != 0.0) ? p - 1 : p;
#endif
            first[a] = (int64_t)floor(sh - 0.5 * (order + 1)) - 1;
            for (int r = 0; r < NR; ++r) wt[a][r] = orc_shape(order, sh - (double)(first[a] + r));
        }
        double acc = 0.0;
        for (int r0 = 0; r0 < NR; ++r0)
            for (int r1 = 0; r1 < NR; ++r1)
                for (int r2 = 0; r2 < NR; ++r2) {
                    const double wgt = wt[0][r0] * wt[1][r1] * wt[2][r2];
                    if (wgt == 0.0) continue;
                    acc += wgt * fetch(g, F[c], first[0] + r0, first[1] + r1, first[2] + r2);
                }
        EB[c] = acc;
    }
}

void orc_gather(const orc_grid* g, int p, const double* const F[6],
                double x, double y, double z, double EB[6]) {
    gather_orders(g, p, 0, F, x, y, z, EB);
}

/* Energy-conserving gather (Sec. 4.2 lists it among the plasma-acceleration
 * run's options): along every axis where a component is staggered the shape
 * order drops to p - 1, the order of the Esirkepov current along its own
 * direction, so that sum_cells J . E dV equals q w v . E(particle) as the
 * step shrinks; unstaggered axes keep order p. */
void orc_gather_ec(const orc_grid* g, int p, const double* const F[6],
                   double x, double y, double z, double EB[6]) {
    gather_orders(g, p, 1, F, x, y, z, EB);
}

/* ------------------------------------------------------------------ */
/* Boris push                                                          */
/* ------------------------------------------------------------------ */

/* Relativistic Boris rotation, u = gamma*v:
 *   k = q dt/(2m); u- = u + kE; g- = sqrt(1+|u-|^2); t = kB/g-;
 *   s = 2t/(1+|t|^2); u' = u- + u- x t; u+ = u- + u' x s; u_new = u+ + kE. */
void orc_boris(double q, double m, double dt, const double E[3], const double B[3], double u[3]) {
    const double k = q * dt / (2.0 * m);
    double um[3] = {u[0] + k * E[0], u[1] + k * E[1], u[2] + k * E[2]};
    const double gm = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
    double t[3] = {k * B[0] / gm, k * B[1] / gm, k * B[2] / gm};
    const double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    double s[3] = {2.0 * t[0] / (1.0 + t2), 2.0 * t[1] / (1.0 + t2), 2.0 * t[2] / (1.0 + t2)};
    double up[3] = {um[0] + (um[1] * t[2] - um[2] * t[1]),
                    um[1] + (um[2] * t[0] - um[0] * t[2]),
                    um[2] + (um[0] * t[1] - um[1] * t[0])};
    double upl[3] = {um[0] + (up[1] * s[2] - up[2] * s[1]),
                     um[1] + (up[2] * s[0] - up[0] * s[2]),
                     um[2] + (up[0] * s[1] - up[1] * s[0])};
#if ORC_MUTANT == 3
    u[0] = upl[0]; u[1] = upl[1]; u[2] = upl[2]; /* planted: second half kick dropped */
#else
    u[0] = upl[0] + k * E[0];
    u[1] = upl[1] + k * E[1];
    u[2] = upl[2] + k * E[2];
#endif
}

/* Vay's pusher (Vay 2008, named among the plasma-acceleration run's options
 * in Sec. 4.2), u = gamma*v:
 *   u^{n+1/2} = u^{n-1/2} + (q dt/m) (E + (v^{n-1/2} + v^{n+1/2})/2 x B),
 * solved as u' = u + (q dt/m)(E + v x B/2) with v = u/gamma, tau = (q dt/2m) B,
 * u* = u'.tau, sigma = 1 + |u'|^2 - |tau|^2,
 * gamma_new = sqrt((sigma + sqrt(sigma^2 + 4 (|tau|^2 + u*^2)))/2),
 * t = tau/gamma_new, s = 1/(1 + |t|^2), u_new = s (u' + (u'.t) t + u' x t). */
void orc_vay(double q, double m, double dt, const double E[3], const double B[3], double u[3]) {
    const double k = q * dt / m;
    const double g0 = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const double v[3] = {u[0] / g0, u[1] / g0, u[2] / g0};
    const double vxB[3] = {v[1] * B[2] - v[2] * B[1], v[2] * B[0] - v[0] * B[2], v[0] * B[1] - v[1] * B[0]};
    double up[3];
#if ORC_MUTANT == 10
    for (int a = 0; a < 3; ++a) up[a] = u[a] + k * E[a]; /* planted: explicit half of v x B dropped */
#else
    for (int a = 0; a < 3; ++a) up[a] = u[a] + k * (E[a] + 0.5 * vxB[a]);
#endif
    const double tau[3] = {0.5 * k * B[0], 0.5 * k * B[1], 0.5 * k * B[2]};
    const double tau2 = tau[0] * tau[0] + tau[1] * tau[1] + tau[2] * tau[2];
    const double ustar = up[0] * tau[0] + up[1] * tau[1] + up[2] * tau[2];
    const double sigma = 1.0 + up[0] * up[0] + up[1] * up[1] + up[2] * up[2] - tau2;
    const double gnew = sqrt(0.5 * (sigma + sqrt(sigma * sigma + 4.0 * (tau2 + ustar * ustar))));
    const double t[3] = {tau[0] / gnew, tau[1] / gnew, tau[2] / gnew};
    const double s = 1.0 / (1.0 + t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    const double ut = up[0] * t[0] + up[1] * t[1] + up[2] * t[2];
    const double uxt[3] = {up[1] * t[2] - up[2] * t[1], up[2] * t[0] - up[0] * t[2], up[0] * t[1] - up[1] * t[0]};
    for (int a = 0; a < 3; ++a) u[a] = s * (up[a] + ut * t[a] + uxt[a]);
}

/* x^{n+1} = x^n + dt u/gamma with gamma = sqrt(1+|u|^2); no wrap. */
void orc_advance(double dt, const double u[3], double x[3]) {
    const double gi = 1.0 / sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
#if ORC_MUTANT == 8
    (void)gi;
    x[0] += dt * u[0]; /* planted: momentum used as velocity */
    x[1] += dt * u[1];
    x[2] += dt * u[2];
#else
    x[0] += dt * u[0] * gi;
    x[1] += dt * u[1] * gi;
    x[2] += dt * u[2] * gi;
#endif
}

/* Periodic wrap into [0, L); a value that rounds to L maps to 0. */
double orc_wrap(double x, double L) {
    if (x >= L) x -= L;
    else if (x < 0.0) x += L;
    if (x >= L) x = 0.0;
    return x;
}

/* ------------------------------------------------------------------ */
/* Esirkepov current deposition                                       */
/* ------------------------------------------------------------------ */

/* Charge-conserving deposit of one particle (charge*weight = qw) moving
 * from x0 to x1 (unwrapped, |x1-x0| < one cell per axis) during dt.
 * Per axis, S0(i) = s_p(x0/d - i), S1(i) = s_p(x1/d - i) on the common
 * window of p+2 nodes starting at floor(min(x0,x1)/d - (p+1)/2) + 1, and
 * dS = S1 - S0.  Esirkepov's decomposition
 *   Wx = dSx [S0y S0z + 1/2 dSy S0z + 1/2 S0y dSz + 1/3 dSy dSz]  (and cyclic)
 * gives Jx(i+1/2,j,k) = -(qw/(dt dy dz)) sum_{i'<=i} Wx(i',j,k) over the window,
 * added with periodic wrap of the node indices. */
void orc_deposit_esirkepov(const orc_grid* g, int p, double dt, double qw,
                           const double x0[3], const double x1[3], double* const J[3]) {
    enum { MAXW = 5 };
    const int nw = p + 2;
    int64_t b[3];
    double S0[3][MAXW], dS[3][MAXW];
    for (int a = 0; a < 3; ++a) {
        const double p0 = x0[a] / g->d[a], p1 = x1[a] / g->d[a];
        const double mn = p0 < p1 ? p0 : p1;
#if ORC_MUTANT == 4
        b[a] = (int64_t)floor(mn - 0.5 * (p + 1)) + 2; /* planted: window start one node high */
#else
        b[a] = (int64_t)floor(mn - 0.5 * (p + 1)) + 1;
#endif
        for (int w = 0; w < nw; ++w) {
            const double node = (double)(b[a] + w);
            S0[a][w] = orc_shape(p, p0 - node);
            dS[a][w] = orc_shape(p, p1 - node) - S0[a][w];
        }
    }
    const double dV = g->d[0] * g->d[1] * g->d[2];
    for (int comp = 0; comp < 3; ++comp) {
        /* axis `comp` carries the cumulative sum; (t1,t2) are the transverse axes in cyclic order */
        const int t1 = (comp + 1) % 3, t2 = (comp + 2) % 3;
        const double coef = -qw * g->d[comp] / (dt * dV);
        for (int w1 = 0; w1 < nw; ++w1) {
            for (int w2 = 0; w2 < nw; ++w2) {
#if ORC_MUTANT == 5
                const double Q = S0[t1][w1] * S0[t2][w2] + 0.5 * dS[t1][w1] * S0[t2][w2] +
                                 0.5 * S0[t1][w1] * dS[t2][w2] + 0.5 * dS[t1][w1] * dS[t2][w2]; /* planted: 1/2 for 1/3 */
#else
                const double Q = S0[t1][w1] * S0[t2][w2] + 0.5 * dS[t1][w1] * S0[t2][w2] +
                                 0.5 * S0[t1][w1] * dS[t2][w2] + (1.0 / 3.0) * dS[t1][w1] * dS[t2][w2];
#endif
                double run = 0.0;
                for (int w0 = 0; w0 < nw; ++w0) {
                    run += dS[comp][w0] * Q;
                    int64_t node[3];
                    node[comp] = b[comp] + w0;
                    node[t1] = b[t1] + w1;
                    node[t2] = b[t2] + w2;
                    add_to(g, J[comp], node[0], node[1], node[2], coef * run);
                }
            }
        }
    }
}

/* Nodal charge density of one particle: rho(i,j,k) += qw S_x S_y S_z / dV. */
void orc_deposit_rho(const orc_grid* g, int p, double qw, const double x[3], double* rho) {
    enum { NR = 8 };
    const double half = 0.5 * (p + 1);
    const double dV = g->d[0] * g->d[1] * g->d[2];
    int64_t first[3];
    double wt[3][NR];
    for (int a = 0; a < 3; ++a) {
        const double pos = x[a] / g->d[a];
        first[a] = (int64_t)floor(pos - half) - 1;
        for (int r = 0; r < NR; ++r) wt[a][r] = orc_shape(p, pos - (double)(first[a] + r));
    }
    for (int r0 = 0; r0 < NR; ++r0)
        for (int r1 = 0; r1 < NR; ++r1)
            for (int r2 = 0; r2 < NR; ++r2) {
                const double wgt = wt[0][r0] * wt[1][r1] * wt[2][r2];
                if (wgt == 0.0) continue;
#if ORC_MUTANT == 14
                add_to(g, rho, first[0] + r0, first[1] + r1, first[2] + r2, qw * wgt);
#else
                add_to(g, rho, first[0] + r0, first[1] + r1, first[2] + r2, qw * wgt / dV);
#endif
            }
}

/* ------------------------------------------------------------------ */
/* Yee FDTD                                                            */
/* ------------------------------------------------------------------ */

/* B <- B - h curl E, forward differences (B sits half a cell above E):
 *   Bx(i,j+1/2,k+1/2) -= h[(Ez(i,j+1,k+1/2)-Ez(i,j,k+1/2))/dy - (Ey(i,j+1/2,k+1)-Ey(i,j+1/2,k))/dz] and cyclic. */
void orc_yee_b(const orc_grid* g, double h, const double* const E[3], double* const B[3]) {
    const int64_t nx = g->n[0], ny = g->n[1], nz = g->n[2];
    const double ix = 1.0 / g->d[0], iy = 1.0 / g->d[1], iz = 1.0 / g->d[2];
    for (int64_t i = 0; i < nx; ++i)
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t k = 0; k < nz; ++k) {
                const int64_t c = idx3(g, i, j, k);
                const double dEz_dy = (E[2][idx3(g, i, j + 1, k)] - E[2][c]) * iy;
                const double dEy_dz = (fetch(g, E[1], i, j, k + 1) - E[1][c]) * iz;
                const double dEx_dz = (fetch(g, E[0], i, j, k + 1) - E[0][c]) * iz;
                const double dEz_dx = (E[2][idx3(g, i + 1, j, k)] - E[2][c]) * ix;
                const double dEy_dx = (E[1][idx3(g, i + 1, j, k)] - E[1][c]) * ix;
                const double dEx_dy = (E[0][idx3(g, i, j + 1, k)] - E[0][c]) * iy;
                B[0][c] -= h * (dEz_dy - dEy_dz);
#if ORC_MUTANT == 6
                B[1][c] -= h * (dEx_dz + dEz_dx); /* planted: sign of one curl term */
#else
                B[1][c] -= h * (dEx_dz - dEz_dx);
#endif
                B[2][c] -= h * (dEy_dx - dEx_dy);
            }
}

/* E <- E + dt (curl B - J), backward differences (E sits half a cell below B):
 *   Ex(i+1/2,j,k) += dt[(Bz(i+1/2,j+1/2,k)-Bz(i+1/2,j-1/2,k))/dy - (By(i+1/2,j,k+1/2)-By(i+1/2,j,k-1/2))/dz - Jx] and cyclic. */
void orc_yee_e(const orc_grid* g, double dt, double* const E[3], const double* const B[3],
               const double* const J[3]) {
    const int64_t nx = g->n[0], ny = g->n[1], nz = g->n[2];
    const double ix = 1.0 / g->d[0], iy = 1.0 / g->d[1], iz = 1.0 / g->d[2];
    for (int64_t i = 0; i < nx; ++i)
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t k = 0; k < nz; ++k) {
                const int64_t c = idx3(g, i, j, k);
                const double dBz_dy = (B[2][c] - B[2][idx3(g, i, j - 1, k)]) * iy;
                const double dBy_dz = (B[1][c] - fetch(g, B[1], i, j, k - 1)) * iz;
                const double dBx_dz = (B[0][c] - fetch(g, B[0], i, j, k - 1)) * iz;
                const double dBz_dx = (B[2][c] - B[2][idx3(g, i - 1, j, k)]) * ix;
                const double dBy_dx = (B[1][c] - B[1][idx3(g, i - 1, j, k)]) * ix;
                const double dBx_dy = (B[0][c] - B[0][idx3(g, i, j - 1, k)]) * iy;
#if ORC_MUTANT == 7
                E[0][c] += dt * ((dBz_dy - dBy_dz) + J[0][c]); /* planted: sign of the current */
#else
                E[0][c] += dt * ((dBz_dy - dBy_dz) - J[0][c]);
#endif
                E[1][c] += dt * ((dBx_dz - dBz_dx) - J[1][c]);
                E[2][c] += dt * ((dBy_dx - dBx_dy) - J[2][c]);
            }
}

/* B <- B - h curl E with the Cole-Karkkainen stencil (the CKC solver named
 * for the plasma-acceleration run, Sec. 4.2), for cubic cells: every forward
 * difference in curl E is averaged over the two directions transverse to it
 * with weights (1/4, 1/2, 1/4) x (1/4, 1/2, 1/4), e.g. for d Ez/dy at
 * (i, j+1/2, k+1/2)
 *   sum_{a,b in -1..1} w_a w_b (Ez(i+a, j+1, k+b+1/2) - Ez(i+a, j, k+b+1/2)) / dy,
 * w_0 = 1/2, w_{+-1} = 1/4.  Along-axis variations are untouched (the
 * weights sum to 1); the scheme is stable up to dt = dx. */
static double dfwd_ckc(const orc_grid* g, const double* F, int axis, int64_t i, int64_t j, int64_t k) {
#if ORC_MUTANT == 11
    static const double w[3] = {1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0}; /* planted: box average instead of (1/4,1/2,1/4) */
#else
    static const double w[3] = {0.25, 0.5, 0.25};
#endif
    const int t1 = (axis + 1) % 3, t2 = (axis + 2) % 3;
    double acc = 0.0;
    for (int a = -1; a <= 1; ++a)
        for (int b = -1; b <= 1; ++b) {
            int64_t p0[3] = {i, j, k};
            p0[t1] += a;
            p0[t2] += b;
            int64_t p1[3] = {p0[0], p0[1], p0[2]};
            p1[axis] += 1;
            acc += w[a + 1] * w[b + 1] * (fetch(g, F, p1[0], p1[1], p1[2]) - fetch(g, F, p0[0], p0[1], p0[2]));
        }
    return acc / g->d[axis];
}

void orc_yee_b_ckc(const orc_grid* g, double h, const double* const E[3], double* const B[3]) {
    const int64_t nx = g->n[0], ny = g->n[1], nz = g->n[2];
    const int64_t C = nx * ny * nz;
    double* nb[3];
    for (int c = 0; c < 3; ++c) nb[c] = (double*)malloc((size_t)C * sizeof(double));
    for (int64_t i = 0; i < nx; ++i)
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t k = 0; k < nz; ++k) {
                const int64_t c = idx3(g, i, j, k);
                nb[0][c] = B[0][c] - h * (dfwd_ckc(g, E[2], 1, i, j, k) - dfwd_ckc(g, E[1], 2, i, j, k));
                nb[1][c] = B[1][c] - h * (dfwd_ckc(g, E[0], 2, i, j, k) - dfwd_ckc(g, E[2], 0, i, j, k));
                nb[2][c] = B[2][c] - h * (dfwd_ckc(g, E[1], 0, i, j, k) - dfwd_ckc(g, E[0], 1, i, j, k));
            }
    for (int c = 0; c < 3; ++c) {
        memcpy(B[c], nb[c], (size_t)C * sizeof(double));
        free(nb[c]);
    }
}

/* One step with the CKC B update (E update as in Yee). */
void orc_yee_step_ckc(const orc_grid* g, double dt, double* const E[3], double* const B[3],
                      const double* const J[3]) {
    orc_yee_b_ckc(g, 0.5 * dt, (const double* const*)E, B);
    orc_yee_e(g, dt, E, (const double* const*)B, J);
    orc_yee_b_ckc(g, 0.5 * dt, (const double* const*)E, B);
}

/* One Yee step: B half step, E full step with the current, B half step. */
void orc_yee_step(const orc_grid* g, double dt, double* const E[3], double* const B[3],
                  const double* const J[3]) {
    orc_yee_b(g, 0.5 * dt, (const double* const*)E, B);
    orc_yee_e(g, dt, E, (const double* const*)B, J);
    orc_yee_b(g, 0.5 * dt, (const double* const*)E, B);
}

/* ------------------------------------------------------------------ */
/* full PIC step                                                       */
/* ------------------------------------------------------------------ */

/* One step for one species: gather E^n, B^n at x^n (plus the optional
 * external drive E_ext = drive_amp * y_hat * cos(drive_k x - drive_k t)),
 * Boris u^{n-1/2} -> u^{n+1/2}, advance x^n -> x^{n+1}, Esirkepov J^{n+1/2}
 * (J is zeroed first), periodic wrap of x^{n+1}, then the Yee update.
 * With z open, z^{n+1} is not wrapped: a particle that left [0, Lz) keeps
 * its outside position (its current inside the grid was deposited) and the
 * caller removes it.  fields = {Ex,Ey,Ez,Bx,By,Bz,Jx,Jy,Jz}. */
void orc_pic_step(const orc_grid* g, int p, double dt, double q, double m, int64_t np,
                  double* x, double* y, double* z, double* ux, double* uy, double* uz,
                  const double* w, double* const fields[9],
                  double drive_amp, double drive_k, double t) {
    orc_pic_step_alg(g, p, dt, q, m, np, x, y, z, ux, uy, uz, w, fields, drive_amp, drive_k, t, 0, 0);
}

/* The same step with a choice of pusher (0 Boris, 1 Vay) and gather
 * (0 momentum-conserving, 1 energy-conserving). */
void orc_pic_step_alg(const orc_grid* g, int p, double dt, double q, double m, int64_t np,
                      double* x, double* y, double* z, double* ux, double* uy, double* uz,
                      const double* w, double* const fields[9],
                      double drive_amp, double drive_k, double t, int pusher, int gather) {
    orc_pic_step_full(g, p, dt, q, m, np, x, y, z, ux, uy, uz, w, fields, drive_amp, drive_k, t, pusher, gather, 0);
}

/* The step with the fields the particles gather from given separately (F:
 * Ex..Bz as gathered; fields: the ones the Yee update advances). */
static void step_impl(const orc_grid* g, int p, double dt, double q, double m, int64_t np, double* x, double* y,
                      double* z, double* ux, double* uy, double* uz, const double* w, double* const fields[9],
                      const double* const F[6], double drive_amp, double drive_k, double t, int pusher, int gather,
                      int solver);

/* The same with a choice of field solver too (0 Yee, 1 CKC). */
void orc_pic_step_full(const orc_grid* g, int p, double dt, double q, double m, int64_t np,
                       double* x, double* y, double* z, double* ux, double* uy, double* uz,
                       const double* w, double* const fields[9],
                       double drive_amp, double drive_k, double t, int pusher, int gather, int solver) {
    const double* const F[6] = {fields[0], fields[1], fields[2], fields[3], fields[4], fields[5]};
    step_impl(g, p, dt, q, m, np, x, y, z, ux, uy, uz, w, fields, F, drive_amp, drive_k, t, pusher, gather, solver);
}

/* Digital filter along z applied to E and B before the gather (the Godfrey
 * filter of the paper's plasma-acceleration run, Sec. 4.2; the paper gives no
 * coefficients, so this is the compensated binomial form of that family of
 * filters): npass passes of the stencil (1/4, 1/2, 1/4), then one
 * compensation pass (-npass/4, 1 + npass/2, -npass/4); each pass reads the
 * previous one's output, periodic along z, or zero beyond the z ends when z
 * is open.  On a periodic Fourier mode e^{i k z} one pass multiplies by
 * cos^2(k dz/2), the compensation by 1 + npass sin^2(k dz/2): the transfer
 * function cos^(2 npass)(k dz/2) (1 + npass sin^2(k dz/2)) is 1 at k = 0, 0 at
 * the Nyquist mode and 1 - O(k^4) for long waves.  npass = 0: a copy. */
void orc_filter_z(const orc_grid* g, int npass, const double* in, double* out) {
    const int64_t C = (int64_t)g->n[0] * g->n[1] * g->n[2];
    double* tmp = (double*)malloc((size_t)C * sizeof(double));
    memcpy(out, in, (size_t)C * sizeof(double));
    for (int pass = 0; pass <= npass && npass > 0; ++pass) {
        double a, b; /* stencil (a, b, a) */
        if (pass < npass) {
            a = 0.25;
            b = 0.5;
        } else {
#if ORC_MUTANT == 15
            a = 0.25 * npass; /* planted: compensation with the wrong sign */
#else
            a = -0.25 * npass;
#endif
            b = 1.0 - 2.0 * a;
        }
        memcpy(tmp, out, (size_t)C * sizeof(double));
        for (int64_t i = 0; i < g->n[0]; ++i)
            for (int64_t j = 0; j < g->n[1]; ++j)
                for (int64_t k = 0; k < g->n[2]; ++k)
                    out[idx3(g, i, j, k)] = a * fetch(g, tmp, i, j, k - 1) + b * tmp[idx3(g, i, j, k)] +
                                            a * fetch(g, tmp, i, j, k + 1);
    }
    free(tmp);
}

/* The step with the particles gathering from E and B filtered along z by
 * orc_filter_z (npass passes); the Yee update advances the unfiltered fields. */
void orc_pic_step_filtered(const orc_grid* g, int p, double dt, double q, double m, int64_t np, double* x,
                           double* y, double* z, double* ux, double* uy, double* uz, const double* w,
                           double* const fields[9], double drive_amp, double drive_k, double t, int pusher,
                           int gather, int solver, int npass) {
    const int64_t C = (int64_t)g->n[0] * g->n[1] * g->n[2];
    double* buf = (double*)malloc(6 * (size_t)C * sizeof(double));
    const double* F[6];
    for (int c = 0; c < 6; ++c) {
        orc_filter_z(g, npass, fields[c], buf + c * C);
        F[c] = buf + c * C;
    }
    step_impl(g, p, dt, q, m, np, x, y, z, ux, uy, uz, w, fields, F, drive_amp, drive_k, t, pusher, gather, solver);
    free(buf);
}

static void step_impl(const orc_grid* g, int p, double dt, double q, double m, int64_t np, double* x, double* y,
                      double* z, double* ux, double* uy, double* uz, const double* w, double* const fields[9],
                      const double* const F[6], double drive_amp, double drive_k, double t, int pusher, int gather,
                      int solver) {
    const int64_t C = (int64_t)g->n[0] * g->n[1] * g->n[2];
    double* const E[3] = {fields[0], fields[1], fields[2]};
    double* const B[3] = {fields[3], fields[4], fields[5]};
    double* const J[3] = {fields[6], fields[7], fields[8]};
    const double L[3] = {g->n[0] * g->d[0], g->n[1] * g->d[1], g->n[2] * g->d[2]};
    for (int c = 0; c < 3; ++c) memset(J[c], 0, (size_t)C * sizeof(double));
    for (int64_t n = 0; n < np; ++n) {
        double EB[6];
        if (gather) orc_gather_ec(g, p, F, x[n], y[n], z[n], EB);
        else orc_gather(g, p, F, x[n], y[n], z[n], EB);
        if (drive_amp != 0.0) EB[1] += drive_amp * cos(drive_k * x[n] - drive_k * t);
        double u[3] = {ux[n], uy[n], uz[n]};
        if (pusher) orc_vay(q, m, dt, EB, EB + 3, u);
        else orc_boris(q, m, dt, EB, EB + 3, u);
        double x0[3] = {x[n], y[n], z[n]};
        double x1[3] = {x[n], y[n], z[n]};
        orc_advance(dt, u, x1);
#if ORC_MUTANT == 16
        orc_deposit_esirkepov(g, p, dt, q * w[n > 0 ? n - 1 : n], x0, x1, J); /* another particle's weight */
#else
        orc_deposit_esirkepov(g, p, dt, q * w[n], x0, x1, J);
#endif
        x[n] = orc_wrap(x1[0], L[0]);
        y[n] = orc_wrap(x1[1], L[1]);
        z[n] = g->zopen ? x1[2] : orc_wrap(x1[2], L[2]); /* z open: left unwrapped, the caller removes it */
        ux[n] = u[0];
        uy[n] = u[1];
        uz[n] = u[2];
    }
    if (solver) orc_yee_step_ckc(g, dt, E, B, (const double* const*)J);
    else orc_yee_step(g, dt, E, B, (const double* const*)J);
}

/* ------------------------------------------------------------------ */
/* diagnostics                                                         */
/* ------------------------------------------------------------------ */

/* Nodal divergence of an edge-centred (E-like) vector field:
 * div(i,j,k) = (Fx[i]-Fx[i-1])/dx + (Fy[j]-Fy[j-1])/dy + (Fz[k]-Fz[k-1])/dz. */
void orc_div_edge(const orc_grid* g, const double* const F[3], double* out) {
    for (int64_t i = 0; i < g->n[0]; ++i)
        for (int64_t j = 0; j < g->n[1]; ++j)
            for (int64_t k = 0; k < g->n[2]; ++k) {
                const int64_t c = idx3(g, i, j, k);
                out[c] = (F[0][c] - F[0][idx3(g, i - 1, j, k)]) / g->d[0] +
                         (F[1][c] - F[1][idx3(g, i, j - 1, k)]) / g->d[1] +
                         (F[2][c] - fetch(g, F[2], i, j, k - 1)) / g->d[2];
            }
}

/* Cell-centred divergence of a face-centred (B-like) vector field:
 * div(i+1/2,j+1/2,k+1/2) = (Bx[i+1]-Bx[i])/dx + (By[j+1]-By[j])/dy + (Bz[k+1]-Bz[k])/dz. */
void orc_div_face(const orc_grid* g, const double* const F[3], double* out) {
    for (int64_t i = 0; i < g->n[0]; ++i)
        for (int64_t j = 0; j < g->n[1]; ++j)
            for (int64_t k = 0; k < g->n[2]; ++k) {
                const int64_t c = idx3(g, i, j, k);
                out[c] = (F[0][idx3(g, i + 1, j, k)] - F[0][c]) / g->d[0] +
                         (F[1][idx3(g, i, j + 1, k)] - F[1][c]) / g->d[1] +
                         (fetch(g, F[2], i, j, k + 1) - F[2][c]) / g->d[2];
            }
}

/* Field energy 1/2 sum (|E|^2 + |B|^2) dV and kinetic energy sum w m (gamma-1)
 * (the in-situ reductions of Sec. 2.6; energy density |E|^2/2 + |B|^2/2 in
 * these units). */
double orc_field_energy(const orc_grid* g, const double* const F[6]) {
    const int64_t C = (int64_t)g->n[0] * g->n[1] * g->n[2];
    double s = 0.0;
    for (int c = 0; c < 6; ++c)
        for (int64_t i = 0; i < C; ++i) s += F[c][i] * F[c][i];
#if ORC_MUTANT == 12
    return 0.5 * s;
#else
    return 0.5 * s * g->d[0] * g->d[1] * g->d[2];
#endif
}

double orc_kinetic_energy(double m, int64_t np, const double* ux, const double* uy, const double* uz,
                          const double* w) {
    double s = 0.0;
    for (int64_t n = 0; n < np; ++n) {
        const double u2 = ux[n] * ux[n] + uy[n] * uy[n] + uz[n] * uz[n];
#if ORC_MUTANT == 13
        s += w[n] * m * sqrt(1.0 + u2);
#else
        s += w[n] * m * (sqrt(1.0 + u2) - 1.0);
#endif
    }
    return s;
}

/* ------------------------------------------------------------------ */
/* batched wrappers (one call per particle array, for the Python side) */
/* ------------------------------------------------------------------ */

void orc_gather_many(const orc_grid* g, int p, const double* const F[6], int64_t np,
                     const double* x, const double* y, const double* z, double* out /* [np][6] */) {
    for (int64_t n = 0; n < np; ++n) orc_gather(g, p, F, x[n], y[n], z[n], out + 6 * n);
}

void orc_gather_ec_many(const orc_grid* g, int p, const double* const F[6], int64_t np, const double* x,
                        const double* y, const double* z, double* out /* [np][6] */) {
    for (int64_t n = 0; n < np; ++n) orc_gather_ec(g, p, F, x[n], y[n], z[n], out + 6 * n);
}

void orc_vay_many(double q, double m, double dt, int64_t np, const double* EB /* [np][6] */, double* ux,
                  double* uy, double* uz) {
    for (int64_t n = 0; n < np; ++n) {
        double u[3] = {ux[n], uy[n], uz[n]};
        orc_vay(q, m, dt, EB + 6 * n, EB + 6 * n + 3, u);
        ux[n] = u[0];
        uy[n] = u[1];
        uz[n] = u[2];
    }
}

void orc_boris_many(double q, double m, double dt, int64_t np, const double* EB /* [np][6] */,
                    double* ux, double* uy, double* uz) {
    for (int64_t n = 0; n < np; ++n) {
        double u[3] = {ux[n], uy[n], uz[n]};
        orc_boris(q, m, dt, EB + 6 * n, EB + 6 * n + 3, u);
        ux[n] = u[0];
        uy[n] = u[1];
        uz[n] = u[2];
    }
}

void orc_deposit_many(const orc_grid* g, int p, double dt, double q, int64_t np,
                      const double* x0, const double* y0, const double* z0,
                      const double* x1, const double* y1, const double* z1,
                      const double* w, double* const J[3]) {
    for (int64_t n = 0; n < np; ++n) {
        const double a[3] = {x0[n], y0[n], z0[n]}, b[3] = {x1[n], y1[n], z1[n]};
        orc_deposit_esirkepov(g, p, dt, q * w[n], a, b, J);
    }
}

void orc_rho_many(const orc_grid* g, int p, double q, int64_t np, const double* x, const double* y,
                  const double* z, const double* w, double* rho) {
    for (int64_t n = 0; n < np; ++n) {
        const double a[3] = {x[n], y[n], z[n]};
        orc_deposit_rho(g, p, q * w[n], a, rho);
    }
}
