/*
 * FP64 CPU oracle: discrete adjoint of the PIC step (pic_oracle.c).
 *
 * TEST INFRASTRUCTURE ONLY (see pic_oracle.c).  It differentiates exactly the
 * oracle's forward map, step by step in reverse, with the cell index and the
 * Esirkepov window treated as locally constant (the derivative of floor() is
 * taken as zero) and the periodic wrap as the identity.
 *
 * Loss: L = 1/2 sum_cells (|E^N|^2 + |B^N|^2) dV after N steps.  Outputs:
 * dL/dA for the amplitude A of the external drive E_y += A cos(k x - k t_n),
 * and dL/du for the initial momenta u^{-1/2}.
 *
 * Reverse of one step (forward: gather -> Boris -> advance -> Esirkepov ->
 * Yee), given the adjoints of x^{n+1}, u^{n+1/2}, E^{n+1}, B^{n+1}:
 *   Yee:      lamB' = lamB^{n+1};  lamE' = lamE^{n+1} - h C^T lamB';
 *             lamJ = -dt lamE';  lamB1/2 = lamB' + dt C'^T lamE';
 *             lamB^n = lamB1/2;  lamE^n = lamE' - h C^T lamB1/2
 *             (C: E -> curl E at B sites, C': B -> curl B at E sites, h = dt/2);
 *   deposit:  lamx0 += (dJ/dx0)^T lamJ, lamx1 += (dJ/dx1)^T lamJ;
 *   advance:  lamx0 += lamx1, lamu += dt (I/g - u u^T/g^3) lamx1;
 *   Boris:    lamu^{n-1/2}, lamE_p, lamB_p by the reverse sweep of the rotation;
 *   gather:   lamF += weights * lamEB_p, lamx0 += (d weights/dx)^T (F lamEB_p),
 *             drive: lamA += lamE_y,p cos(k x - k t), lamx += -A k sin(..) lamE_y,p.
 * Periodic grids only (orc_grid.zopen = 0).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "pic_oracle.h"

static int64_t wrapi_a(int64_t i, int64_t n) {
    int64_t r = i % n;
    return r < 0 ? r + n : r;
}

static int64_t idx3_a(const orc_grid* g, int64_t i, int64_t j, int64_t k) {
    return (wrapi_a(i, g->n[0]) * g->n[1] + wrapi_a(j, g->n[1])) * g->n[2] + wrapi_a(k, g->n[2]);
}

static const double STAG_A[6][3] = {
    {0.5, 0.0, 0.0}, {0.0, 0.5, 0.0}, {0.0, 0.0, 0.5},
    {0.0, 0.5, 0.5}, {0.5, 0.0, 0.5}, {0.5, 0.5, 0.0},
};

/* s_p'(xi), the derivative of the order-p B-spline (0 at the knots where it
 * jumps, the average of the one-sided values there). */
double orc_dshape(int p, double xi) {
    const double a = fabs(xi), sg = xi < 0.0 ? -1.0 : 1.0;
    switch (p) {
    case 1:
        return a < 1.0 && a > 0.0 ? -sg : 0.0;
    case 2:
        if (a <= 0.5) return -2.0 * xi;
        if (a < 1.5) return -sg * (1.5 - a);
        return 0.0;
    case 3:
        if (a <= 1.0) return sg * (-12.0 * a + 9.0 * a * a) / 6.0;
        if (a < 2.0) { const double t = 2.0 - a; return -sg * 3.0 * t * t / 6.0; }
        return 0.0;
    default:
        return 0.0;
    }
}

/* ------------------------------------------------------------------ */
/* gather adjoint                                                      */
/* ------------------------------------------------------------------ */

/* For EB_c = sum_nodes w(x) F_c[node]: lamF_c[node] += w lamEB_c and
 * lam_x[a] += lamEB_c sum_nodes dw/dx_a F_c[node]. */
void orc_gather_adj(const orc_grid* g, int p, const double* const F[6], double* const lamF[6],
                    const double x[3], const double lamEB[6], double lam_x[3]) {
    enum { NR = 8 };
    const double half = 0.5 * (p + 1);
    for (int c = 0; c < 6; ++c) {
        if (lamEB[c] == 0.0) continue;
        int64_t first[3];
        double wt[3][NR], dw[3][NR];
        for (int a = 0; a < 3; ++a) {
            const double sh = x[a] / g->d[a] - STAG_A[c][a];
            first[a] = (int64_t)floor(sh - half) - 1;
            for (int r = 0; r < NR; ++r) {
                wt[a][r] = orc_shape(p, sh - (double)(first[a] + r));
                dw[a][r] = orc_dshape(p, sh - (double)(first[a] + r)) / g->d[a];
            }
        }
        double gx[3] = {0.0, 0.0, 0.0};
        for (int r0 = 0; r0 < NR; ++r0)
            for (int r1 = 0; r1 < NR; ++r1)
                for (int r2 = 0; r2 < NR; ++r2) {
                    const int64_t node = idx3_a(g, first[0] + r0, first[1] + r1, first[2] + r2);
                    const double w = wt[0][r0] * wt[1][r1] * wt[2][r2];
                    if (w != 0.0) lamF[c][node] += w * lamEB[c];
                    const double f = F[c][node];
                    gx[0] += dw[0][r0] * wt[1][r1] * wt[2][r2] * f;
                    gx[1] += wt[0][r0] * dw[1][r1] * wt[2][r2] * f;
                    gx[2] += wt[0][r0] * wt[1][r1] * dw[2][r2] * f;
                }
        for (int a = 0; a < 3; ++a) lam_x[a] += lamEB[c] * gx[a];
    }
}

/* ------------------------------------------------------------------ */
/* Boris adjoint                                                       */
/* ------------------------------------------------------------------ */

static void cross(const double a[3], const double b[3], double o[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

/* Reverse sweep of orc_boris: given the forward inputs (u_old, E, B) and the
 * adjoint of the result, return the adjoints of u_old, E and B. */
void orc_boris_adj(double q, double m, double dt, const double E[3], const double B[3], const double u_old[3],
                   const double lam_unew[3], double lam_uold[3], double lam_E[3], double lam_B[3]) {
    const double k = q * dt / (2.0 * m);
    /* forward intermediates */
    double um[3], t[3], s[3], up[3], tmp[3];
    for (int a = 0; a < 3; ++a) um[a] = u_old[a] + k * E[a];
    const double gm = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
    for (int a = 0; a < 3; ++a) t[a] = k * B[a] / gm;
    const double tt = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    const double sc = 2.0 / (1.0 + tt);
    for (int a = 0; a < 3; ++a) s[a] = sc * t[a];
    cross(um, t, tmp);
    for (int a = 0; a < 3; ++a) up[a] = um[a] + tmp[a];
    /* reverse */
    double g_upl[3], g_um[3], g_up[3], g_s[3], g_t[3];
    for (int a = 0; a < 3; ++a) {
        g_upl[a] = lam_unew[a];
        lam_E[a] = k * lam_unew[a];
        g_um[a] = g_upl[a];
    }
    /* upl = um + up x s */
    cross(s, g_upl, g_up);   /* d/dup of (up x s).g = s x g */
    cross(g_upl, up, g_s);   /* d/ds  of (up x s).g = g x up */
    /* up = um + um x t */
    cross(t, g_up, tmp);
    for (int a = 0; a < 3; ++a) g_um[a] += g_up[a] + tmp[a];
    cross(g_up, um, g_t);
    /* s = sc t, sc = 2/(1+tt) */
    double g_sc = 0.0;
    for (int a = 0; a < 3; ++a) {
        g_t[a] += sc * g_s[a];
        g_sc += g_s[a] * t[a];
    }
    const double g_tt = -0.5 * sc * sc * g_sc;
    for (int a = 0; a < 3; ++a) g_t[a] += 2.0 * t[a] * g_tt;
    /* t = k B / gm */
    double g_gm = 0.0;
    for (int a = 0; a < 3; ++a) {
        lam_B[a] = (k / gm) * g_t[a];
        g_gm -= t[a] * g_t[a] / gm;
    }
    /* gm = sqrt(1 + |um|^2) */
    for (int a = 0; a < 3; ++a) g_um[a] += um[a] / gm * g_gm;
    /* um = u + k E */
    for (int a = 0; a < 3; ++a) {
        lam_uold[a] = g_um[a];
        lam_E[a] += k * g_um[a];
    }
}

/* ------------------------------------------------------------------ */
/* Esirkepov adjoint                                                   */
/* ------------------------------------------------------------------ */

/* Adjoint of orc_deposit_esirkepov for one particle: lam_x0 += (dJ/dx0)^T lamJ
 * and lam_x1 += (dJ/dx1)^T lamJ, the window start held fixed. */
void orc_deposit_adj(const orc_grid* g, int p, double dt, double qw, const double x0[3], const double x1[3],
                     const double* const lamJ[3], double lam_x0[3], double lam_x1[3]) {
    enum { MAXW = 5 };
    const int nw = p + 2;
    int64_t b[3];
    double S0[3][MAXW], dS[3][MAXW], dS0[3][MAXW], dS1[3][MAXW];
    double gS0[3][MAXW], gdS[3][MAXW];
    for (int a = 0; a < 3; ++a) {
        const double p0 = x0[a] / g->d[a], p1 = x1[a] / g->d[a];
        const double mn = p0 < p1 ? p0 : p1;
        b[a] = (int64_t)floor(mn - 0.5 * (p + 1)) + 1;
        for (int w = 0; w < nw; ++w) {
            const double node = (double)(b[a] + w);
            S0[a][w] = orc_shape(p, p0 - node);
            dS[a][w] = orc_shape(p, p1 - node) - S0[a][w];
            dS0[a][w] = orc_dshape(p, p0 - node) / g->d[a];
            dS1[a][w] = orc_dshape(p, p1 - node) / g->d[a];
            gS0[a][w] = 0.0;
            gdS[a][w] = 0.0;
        }
    }
    const double dV = g->d[0] * g->d[1] * g->d[2];
    for (int comp = 0; comp < 3; ++comp) {
        const int t1 = (comp + 1) % 3, t2 = (comp + 2) % 3;
        const double coef = -qw * g->d[comp] / (dt * dV);
        double gcum[MAXW] = {0.0};
        for (int w1 = 0; w1 < nw; ++w1)
            for (int w2 = 0; w2 < nw; ++w2) {
                const double Q = S0[t1][w1] * S0[t2][w2] + 0.5 * dS[t1][w1] * S0[t2][w2] +
                                 0.5 * S0[t1][w1] * dS[t2][w2] + (1.0 / 3.0) * dS[t1][w1] * dS[t2][w2];
                double run = 0.0, gQ = 0.0;
                for (int w0 = 0; w0 < nw; ++w0) {
                    run += dS[comp][w0];
                    int64_t node[3];
                    node[comp] = b[comp] + w0;
                    node[t1] = b[t1] + w1;
                    node[t2] = b[t2] + w2;
                    const double M = coef * lamJ[comp][idx3_a(g, node[0], node[1], node[2])];
                    /* J += coef * run * Q */
                    gQ += M * run;
                    gcum[w0] += M * Q;
                }
                gS0[t1][w1] += gQ * (S0[t2][w2] + 0.5 * dS[t2][w2]);
                gdS[t1][w1] += gQ * (0.5 * S0[t2][w2] + (1.0 / 3.0) * dS[t2][w2]);
                gS0[t2][w2] += gQ * (S0[t1][w1] + 0.5 * dS[t1][w1]);
                gdS[t2][w2] += gQ * (0.5 * S0[t1][w1] + (1.0 / 3.0) * dS[t1][w1]);
            }
        /* run(w0) = sum_{w' <= w0} dS[comp][w'] */
        double acc = 0.0;
        for (int w = nw - 1; w >= 0; --w) {
            acc += gcum[w];
            gdS[comp][w] += acc;
        }
    }
    /* S1 = S0 + dS */
    for (int a = 0; a < 3; ++a)
        for (int w = 0; w < nw; ++w) {
            lam_x0[a] += (gS0[a][w] - gdS[a][w]) * dS0[a][w];
            lam_x1[a] += gdS[a][w] * dS1[a][w];
        }
}

/* ------------------------------------------------------------------ */
/* Yee adjoint                                                         */
/* ------------------------------------------------------------------ */

/* out_E += C^T lamB: the transpose of the forward-difference curl of
 * orc_yee_b, written as the scatter of each B-site term onto the E values it
 * read. */
static void curlE_T(const orc_grid* g, const double* const lamB[3], double* const outE[3]) {
    const double ix = 1.0 / g->d[0], iy = 1.0 / g->d[1], iz = 1.0 / g->d[2];
    for (int64_t i = 0; i < g->n[0]; ++i)
        for (int64_t j = 0; j < g->n[1]; ++j)
            for (int64_t k = 0; k < g->n[2]; ++k) {
                const int64_t c = idx3_a(g, i, j, k);
                /* (curl E)_x = (Ez[j+1]-Ez)/dy - (Ey[k+1]-Ey)/dz */
                const double bx = lamB[0][c], by = lamB[1][c], bz = lamB[2][c];
                outE[2][idx3_a(g, i, j + 1, k)] += bx * iy;
                outE[2][c] -= bx * iy;
                outE[1][idx3_a(g, i, j, k + 1)] -= bx * iz;
                outE[1][c] += bx * iz;
                /* (curl E)_y = (Ex[k+1]-Ex)/dz - (Ez[i+1]-Ez)/dx */
                outE[0][idx3_a(g, i, j, k + 1)] += by * iz;
                outE[0][c] -= by * iz;
                outE[2][idx3_a(g, i + 1, j, k)] -= by * ix;
                outE[2][c] += by * ix;
                /* (curl E)_z = (Ey[i+1]-Ey)/dx - (Ex[j+1]-Ex)/dy */
                outE[1][idx3_a(g, i + 1, j, k)] += bz * ix;
                outE[1][c] -= bz * ix;
                outE[0][idx3_a(g, i, j + 1, k)] -= bz * iy;
                outE[0][c] += bz * iy;
            }
}

/* out_B += C'^T lamE: the transpose of the backward-difference curl of orc_yee_e. */
static void curlB_T(const orc_grid* g, const double* const lamE[3], double* const outB[3]) {
    const double ix = 1.0 / g->d[0], iy = 1.0 / g->d[1], iz = 1.0 / g->d[2];
    for (int64_t i = 0; i < g->n[0]; ++i)
        for (int64_t j = 0; j < g->n[1]; ++j)
            for (int64_t k = 0; k < g->n[2]; ++k) {
                const int64_t c = idx3_a(g, i, j, k);
                const double ex = lamE[0][c], ey = lamE[1][c], ez = lamE[2][c];
                /* (curl B)_x = (Bz - Bz[j-1])/dy - (By - By[k-1])/dz */
                outB[2][c] += ex * iy;
                outB[2][idx3_a(g, i, j - 1, k)] -= ex * iy;
                outB[1][c] -= ex * iz;
                outB[1][idx3_a(g, i, j, k - 1)] += ex * iz;
                /* (curl B)_y = (Bx - Bx[k-1])/dz - (Bz - Bz[i-1])/dx */
                outB[0][c] += ey * iz;
                outB[0][idx3_a(g, i, j, k - 1)] -= ey * iz;
                outB[2][c] -= ey * ix;
                outB[2][idx3_a(g, i - 1, j, k)] += ey * ix;
                /* (curl B)_z = (By - By[i-1])/dx - (Bx - Bx[j-1])/dy */
                outB[1][c] += ez * ix;
                outB[1][idx3_a(g, i - 1, j, k)] -= ez * ix;
                outB[0][c] -= ez * iy;
                outB[0][idx3_a(g, i, j - 1, k)] += ez * iy;
            }
}

/* Reverse of orc_yee_step, in place on lamE, lamB (adjoints of E^{n+1},
 * B^{n+1} on entry, of E^n, B^n on exit); lamJ receives the adjoint of J. */
void orc_yee_step_adj(const orc_grid* g, double dt, double* const lamE[3], double* const lamB[3],
                      double* const lamJ[3]) {
    const int64_t C = g->n[0] * g->n[1] * g->n[2];
    const double h = 0.5 * dt;
    double* tmp = (double*)calloc((size_t)(3 * C), sizeof(double));
    double* const T[3] = {tmp, tmp + C, tmp + 2 * C};
    /* B' = B1/2 - h C E'  ->  lamE' = lamE - h C^T lamB */
    curlE_T(g, (const double* const*)lamB, T);
    for (int a = 0; a < 3; ++a)
        for (int64_t i = 0; i < C; ++i) lamE[a][i] -= h * T[a][i];
    /* E' = E + dt (C' B1/2 - J)  ->  lamJ = -dt lamE', lamB1/2 = lamB' + dt C'^T lamE' */
    memset(tmp, 0, (size_t)(3 * C) * sizeof(double));
    curlB_T(g, (const double* const*)lamE, T);
    for (int a = 0; a < 3; ++a)
        for (int64_t i = 0; i < C; ++i) {
            lamJ[a][i] = -dt * lamE[a][i];
            lamB[a][i] += dt * T[a][i];
        }
    /* B1/2 = B - h C E  ->  lamE -= h C^T lamB1/2, lamB unchanged */
    memset(tmp, 0, (size_t)(3 * C) * sizeof(double));
    curlE_T(g, (const double* const*)lamB, T);
    for (int a = 0; a < 3; ++a)
        for (int64_t i = 0; i < C; ++i) lamE[a][i] -= h * T[a][i];
    free(tmp);
}

/* ------------------------------------------------------------------ */
/* full adjoint                                                        */
/* ------------------------------------------------------------------ */

/* Runs nsteps forward from the given state (particles x..w, E and B in
 * fields[0..5]; J ignored) with the drive (A, kd), storing every state, then
 * the reverse sweep for L = 1/2 sum(|E|^2+|B|^2) dV at the end.  Writes
 * dL/dA, dL/du^{-1/2} (3 np, component-major: ux then uy then uz) and the loss;
 * the particles and fields are left at the final forward state. */
void orc_pic_adjoint(const orc_grid* g, int p, double dt, double q, double m, int64_t np, double* x, double* y,
                     double* z, double* ux, double* uy, double* uz, const double* w, double* const fields[9],
                     int nsteps, double A, double kd, double* dL_dA, double* dL_du, double* loss) {
    const int64_t C = g->n[0] * g->n[1] * g->n[2];
    const double dV = g->d[0] * g->d[1] * g->d[2];
    const double L[3] = {g->n[0] * g->d[0], g->n[1] * g->d[1], g->n[2] * g->d[2]};
    /* stored states: particles (x, y, z, ux, uy, uz) and E, B before each step */
    double* ps = (double*)malloc((size_t)(nsteps * 6 * np + 1) * sizeof(double));
    double* fs = (double*)malloc((size_t)(nsteps * 6 * C + 1) * sizeof(double));
    for (int n = 0; n < nsteps; ++n) {
        double* P = ps + (size_t)n * 6 * np;
        memcpy(P + 0 * np, x, (size_t)np * sizeof(double));
        memcpy(P + 1 * np, y, (size_t)np * sizeof(double));
        memcpy(P + 2 * np, z, (size_t)np * sizeof(double));
        memcpy(P + 3 * np, ux, (size_t)np * sizeof(double));
        memcpy(P + 4 * np, uy, (size_t)np * sizeof(double));
        memcpy(P + 5 * np, uz, (size_t)np * sizeof(double));
        for (int c = 0; c < 6; ++c) memcpy(fs + ((size_t)n * 6 + c) * C, fields[c], (size_t)C * sizeof(double));
        orc_pic_step(g, p, dt, q, m, np, x, y, z, ux, uy, uz, w, fields, A, kd, (double)n * dt);
    }
    double l = 0.0;
    for (int c = 0; c < 6; ++c)
        for (int64_t i = 0; i < C; ++i) l += fields[c][i] * fields[c][i];
    *loss = 0.5 * l * dV;

    /* adjoint state */
    double* lf = (double*)calloc((size_t)(9 * C), sizeof(double));
    double* const lamE[3] = {lf, lf + C, lf + 2 * C};
    double* const lamB[3] = {lf + 3 * C, lf + 4 * C, lf + 5 * C};
    double* const lamJ[3] = {lf + 6 * C, lf + 7 * C, lf + 8 * C};
    double* lp = (double*)calloc((size_t)(6 * np), sizeof(double)); /* lam x (3), lam u (3) */
    for (int c = 0; c < 3; ++c)
        for (int64_t i = 0; i < C; ++i) {
            lamE[c][i] = fields[c][i] * dV;
            lamB[c][i] = fields[3 + c][i] * dV;
        }
    double gA = 0.0;
    double* lamF_gather = (double*)calloc((size_t)(6 * C), sizeof(double));
    for (int n = nsteps - 1; n >= 0; --n) {
        const double* P = ps + (size_t)n * 6 * np;
        const double* Fn[6];
        for (int c = 0; c < 6; ++c) Fn[c] = fs + ((size_t)n * 6 + c) * C;
        const double t = (double)n * dt;
        orc_yee_step_adj(g, dt, lamE, lamB, lamJ);
        memset(lamF_gather, 0, (size_t)(6 * C) * sizeof(double));
        double* const lamFg[6] = {lamF_gather, lamF_gather + C, lamF_gather + 2 * C,
                                  lamF_gather + 3 * C, lamF_gather + 4 * C, lamF_gather + 5 * C};
        for (int64_t i = 0; i < np; ++i) {
            const double x0[3] = {P[i], P[np + i], P[2 * np + i]};
            const double u_old[3] = {P[3 * np + i], P[4 * np + i], P[5 * np + i]};
            /* forward recomputation */
            double EB[6];
            orc_gather(g, p, Fn, x0[0], x0[1], x0[2], EB);
            const double ph = kd * x0[0] - kd * t;
            EB[1] += A * cos(ph); /* the forward adds it only for A != 0, where it is A cos */
            double u[3] = {u_old[0], u_old[1], u_old[2]};
            orc_boris(q, m, dt, EB, EB + 3, u);
            double x1[3] = {x0[0], x0[1], x0[2]};
            orc_advance(dt, u, x1);
            /* adjoints of the step's outputs */
            double lx1[3] = {lp[i], lp[np + i], lp[2 * np + i]};          /* lam x^{n+1} (wrap: identity) */
            double lu[3] = {lp[3 * np + i], lp[4 * np + i], lp[5 * np + i]}; /* lam u^{n+1/2} */
            double lx0[3] = {0.0, 0.0, 0.0};
            /* deposit */
            orc_deposit_adj(g, p, dt, q * w[i], x0, x1, (const double* const*)lamJ, lx0, lx1);
            /* advance x1 = x0 + dt u / gamma */
            const double gam = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
            const double udl = u[0] * lx1[0] + u[1] * lx1[1] + u[2] * lx1[2];
            for (int a = 0; a < 3; ++a) {
                lx0[a] += lx1[a];
                lu[a] += dt * (lx1[a] / gam - u[a] * udl / (gam * gam * gam));
            }
            /* Boris */
            double luo[3], lE[3], lB[3];
            orc_boris_adj(q, m, dt, EB, EB + 3, u_old, lu, luo, lE, lB);
            /* drive */
            gA += lE[1] * cos(ph);
            lx0[0] += lE[1] * A * (-kd) * sin(ph);
            /* gather */
            const double lEB[6] = {lE[0], lE[1], lE[2], lB[0], lB[1], lB[2]};
            orc_gather_adj(g, p, Fn, lamFg, x0, lEB, lx0);
            lp[i] = lx0[0];
            lp[np + i] = lx0[1];
            lp[2 * np + i] = lx0[2];
            lp[3 * np + i] = luo[0];
            lp[4 * np + i] = luo[1];
            lp[5 * np + i] = luo[2];
        }
        for (int c = 0; c < 3; ++c)
            for (int64_t i = 0; i < C; ++i) {
                lamE[c][i] += lamFg[c][i];
                lamB[c][i] += lamFg[3 + c][i];
            }
        (void)L;
    }
    *dL_dA = gA;
    memcpy(dL_du, lp + 3 * np, (size_t)(3 * np) * sizeof(double));
    free(lamF_gather);
    free(lp);
    free(lf);
    free(ps);
    free(fs);
}

/* Helpers for the self-tests: the Yee curls and their transposes as
 * stand-alone maps on whole arrays. */
void orc_curlE(const orc_grid* g, const double* const E[3], double* const out[3]) {
    double* const B[3] = {out[0], out[1], out[2]};
    const int64_t C = g->n[0] * g->n[1] * g->n[2];
    for (int a = 0; a < 3; ++a) memset(B[a], 0, (size_t)C * sizeof(double));
    orc_yee_b(g, -1.0, E, B); /* B -= (-1) curl E  ->  B = curl E */
}

void orc_curlE_T(const orc_grid* g, const double* const lamB[3], double* const out[3]) {
    const int64_t C = g->n[0] * g->n[1] * g->n[2];
    for (int a = 0; a < 3; ++a) memset(out[a], 0, (size_t)C * sizeof(double));
    curlE_T(g, lamB, out);
}

void orc_curlB_T(const orc_grid* g, const double* const lamE[3], double* const out[3]) {
    const int64_t C = g->n[0] * g->n[1] * g->n[2];
    for (int a = 0; a < 3; ++a) memset(out[a], 0, (size_t)C * sizeof(double));
    curlB_T(g, lamE, out);
}
