/*
 * Multi-threaded FP64 CPU baseline of the PIC step (OpenMP).
 *
 * TEST INFRASTRUCTURE ONLY, like pic_oracle.c: a CPU baseline that the
 * benchmark times on the host cores and that the test suite checks against
 * the serial oracle.  The product library never links, calls or reads it.
 *
 * It follows the paper's CPU current deposition (Sec. 3.4.1): the particles
 * are split among the threads, each thread deposits into its own copy of the
 * current arrays (so no two threads add to the same memory), and the copies
 * are then summed into J.  Here each thread takes one contiguous block of the
 * particles and the copies are summed in thread order, a fixed order for a
 * fixed thread count.  Everything else is the serial oracle's arithmetic per
 * particle and per cell (gather, push, advance and wrap call the oracle's own
 * functions; the Yee loops restate its formulas cell by cell, which has no
 * order of additions to change), so the result equals the serial oracle's up
 * to the order in which J is summed.
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <string.h>

#include "pic_oracle.h"

static int64_t mt_wrap(int64_t i, int64_t n) {
    const int64_t r = i % n;
    return r < 0 ? r + n : r;
}

static int64_t mt_idx(const orc_grid* g, int64_t i, int64_t j, int64_t k) {
    return (mt_wrap(i, g->n[0]) * g->n[1] + mt_wrap(j, g->n[1])) * g->n[2] + mt_wrap(k, g->n[2]);
}

/* z open: no field beyond the z ends */
static double mt_fetch(const orc_grid* g, const double* F, int64_t i, int64_t j, int64_t k) {
    return (g->zopen && (k < 0 || k >= g->n[2])) ? 0.0 : F[mt_idx(g, i, j, k)];
}

/* B <- B - h curl E (forward differences), cell by cell in parallel. */
static void mt_yee_b(const orc_grid* g, double h, double* const E[3], double* const B[3]) {
    const int64_t nx = g->n[0], ny = g->n[1], nz = g->n[2];
    const double ix = 1.0 / g->d[0], iy = 1.0 / g->d[1], iz = 1.0 / g->d[2];
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nx; ++i)
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t k = 0; k < nz; ++k) {
                const int64_t c = mt_idx(g, i, j, k);
                const double dEz_dy = (E[2][mt_idx(g, i, j + 1, k)] - E[2][c]) * iy;
                const double dEy_dz = (mt_fetch(g, E[1], i, j, k + 1) - E[1][c]) * iz;
                const double dEx_dz = (mt_fetch(g, E[0], i, j, k + 1) - E[0][c]) * iz;
                const double dEz_dx = (E[2][mt_idx(g, i + 1, j, k)] - E[2][c]) * ix;
                const double dEy_dx = (E[1][mt_idx(g, i + 1, j, k)] - E[1][c]) * ix;
                const double dEx_dy = (E[0][mt_idx(g, i, j + 1, k)] - E[0][c]) * iy;
                B[0][c] -= h * (dEz_dy - dEy_dz);
                B[1][c] -= h * (dEx_dz - dEz_dx);
                B[2][c] -= h * (dEy_dx - dEx_dy);
            }
}

/* E <- E + dt (curl B - J) (backward differences), cell by cell in parallel. */
static void mt_yee_e(const orc_grid* g, double dt, double* const E[3], double* const B[3], double* const J[3]) {
    const int64_t nx = g->n[0], ny = g->n[1], nz = g->n[2];
    const double ix = 1.0 / g->d[0], iy = 1.0 / g->d[1], iz = 1.0 / g->d[2];
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nx; ++i)
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t k = 0; k < nz; ++k) {
                const int64_t c = mt_idx(g, i, j, k);
                const double dBz_dy = (B[2][c] - B[2][mt_idx(g, i, j - 1, k)]) * iy;
                const double dBy_dz = (B[1][c] - mt_fetch(g, B[1], i, j, k - 1)) * iz;
                const double dBx_dz = (B[0][c] - mt_fetch(g, B[0], i, j, k - 1)) * iz;
                const double dBz_dx = (B[2][c] - B[2][mt_idx(g, i - 1, j, k)]) * ix;
                const double dBy_dx = (B[1][c] - B[1][mt_idx(g, i - 1, j, k)]) * ix;
                const double dBx_dy = (B[0][c] - B[0][mt_idx(g, i, j - 1, k)]) * iy;
                E[0][c] += dt * ((dBz_dy - dBy_dz) - J[0][c]);
                E[1][c] += dt * ((dBx_dz - dBz_dx) - J[1][c]);
                E[2][c] += dt * ((dBy_dx - dBx_dy) - J[2][c]);
            }
}

/* Threads the OpenMP runtime would use (the caller's choice when > 0). */
int orc_mt_threads(int nthreads) { return nthreads > 0 ? nthreads : omp_get_max_threads(); }

/* One PIC step (Yee solver; Boris or Vay, momentum- or energy-conserving
 * gather) on `nthreads` threads, as orc_pic_step_full with solver 0.
 * scratch: nthreads * 3 * C doubles, the threads' private current arrays. */
void orc_mt_pic_step(const orc_grid* g, int p, double dt, double q, double m, int64_t np, double* x, double* y,
                     double* z, double* ux, double* uy, double* uz, const double* w, double* const fields[9],
                     double drive_amp, double drive_k, double t, int pusher, int gather, int nthreads,
                     double* scratch) {
    const int64_t C = g->n[0] * g->n[1] * g->n[2];
    double* const E[3] = {fields[0], fields[1], fields[2]};
    double* const B[3] = {fields[3], fields[4], fields[5]};
    double* const J[3] = {fields[6], fields[7], fields[8]};
    const double* const F[6] = {fields[0], fields[1], fields[2], fields[3], fields[4], fields[5]};
    const double L[3] = {g->n[0] * g->d[0], g->n[1] * g->d[1], g->n[2] * g->d[2]};
    const int T = orc_mt_threads(nthreads);
#pragma omp parallel num_threads(T)
    {
        const int tid = omp_get_thread_num();
        const int nt = omp_get_num_threads();
        double* const Jt[3] = {scratch + (3 * (int64_t)tid) * C, scratch + (3 * (int64_t)tid + 1) * C,
                               scratch + (3 * (int64_t)tid + 2) * C};
        for (int c = 0; c < 3; ++c) memset(Jt[c], 0, (size_t)C * sizeof(double));
        /* this thread's contiguous block of the particles */
        const int64_t n0 = np * tid / nt, n1 = np * (tid + 1) / nt;
        for (int64_t n = n0; n < n1; ++n) {
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
            orc_deposit_esirkepov(g, p, dt, q * w[n], x0, x1, Jt);
            x[n] = orc_wrap(x1[0], L[0]);
            y[n] = orc_wrap(x1[1], L[1]);
            z[n] = g->zopen ? x1[2] : orc_wrap(x1[2], L[2]);
            ux[n] = u[0];
            uy[n] = u[1];
            uz[n] = u[2];
        }
#pragma omp barrier
        /* J = sum of the private copies, in thread order, cells split among the threads */
#pragma omp for schedule(static)
        for (int64_t i = 0; i < C; ++i)
            for (int c = 0; c < 3; ++c) {
                double s = 0.0;
                for (int k = 0; k < nt; ++k) s += scratch[(3 * (int64_t)k + c) * C + i];
                J[c][i] = s;
            }
    }
    mt_yee_b(g, 0.5 * dt, E, B);
    mt_yee_e(g, dt, E, B, J);
    mt_yee_b(g, 0.5 * dt, E, B);
}
