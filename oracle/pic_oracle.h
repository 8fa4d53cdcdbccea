/*
 * FP64 CPU oracle for the electromagnetic PIC hot path: declarations.
 * TEST INFRASTRUCTURE ONLY (see pic_oracle.c).  Internal to oracle/; the
 * CUDA library has its own, unrelated header.
 */
#ifndef PIC_ORACLE_H
#define PIC_ORACLE_H
#include <stdint.h>

typedef struct {
    int64_t n[3]; /* cells per axis */
    double d[3];  /* cell size per axis */
    int64_t zopen; /* 0: periodic in z; 1: z open, fields beyond the ends are zero (moving-window runs) */
} orc_grid;

double orc_shape(int p, double xi);
void orc_gather(const orc_grid* g, int p, const double* const F[6], double x, double y, double z, double EB[6]);
void orc_gather_ec(const orc_grid* g, int p, const double* const F[6], double x, double y, double z, double EB[6]);
void orc_boris(double q, double m, double dt, const double E[3], const double B[3], double u[3]);
void orc_vay(double q, double m, double dt, const double E[3], const double B[3], double u[3]);
void orc_advance(double dt, const double u[3], double x[3]);
double orc_wrap(double x, double L);
void orc_deposit_esirkepov(const orc_grid* g, int p, double dt, double qw, const double x0[3], const double x1[3],
                           double* const J[3]);
void orc_deposit_rho(const orc_grid* g, int p, double qw, const double x[3], double* rho);
void orc_yee_b(const orc_grid* g, double h, const double* const E[3], double* const B[3]);
void orc_yee_e(const orc_grid* g, double dt, double* const E[3], const double* const B[3], const double* const J[3]);
void orc_yee_step(const orc_grid* g, double dt, double* const E[3], double* const B[3], const double* const J[3]);
void orc_pic_step(const orc_grid* g, int p, double dt, double q, double m, int64_t np, double* x, double* y,
                  double* z, double* ux, double* uy, double* uz, const double* w, double* const fields[9],
                  double drive_amp, double drive_k, double t);
void orc_yee_b_ckc(const orc_grid* g, double h, const double* const E[3], double* const B[3]);
void orc_yee_step_ckc(const orc_grid* g, double dt, double* const E[3], double* const B[3], const double* const J[3]);
void orc_pic_step_full(const orc_grid* g, int p, double dt, double q, double m, int64_t np, double* x, double* y,
                       double* z, double* ux, double* uy, double* uz, const double* w, double* const fields[9],
                       double drive_amp, double drive_k, double t, int pusher, int gather, int solver);
void orc_pic_step_alg(const orc_grid* g, int p, double dt, double q, double m, int64_t np, double* x, double* y,
                      double* z, double* ux, double* uy, double* uz, const double* w, double* const fields[9],
                      double drive_amp, double drive_k, double t, int pusher, int gather);
void orc_filter_z(const orc_grid* g, int npass, const double* in, double* out);
void orc_pic_step_filtered(const orc_grid* g, int p, double dt, double q, double m, int64_t np, double* x,
                           double* y, double* z, double* ux, double* uy, double* uz, const double* w,
                           double* const fields[9], double drive_amp, double drive_k, double t, int pusher,
                           int gather, int solver, int npass);
void orc_div_edge(const orc_grid* g, const double* const F[3], double* out);
void orc_div_face(const orc_grid* g, const double* const F[3], double* out);
double orc_field_energy(const orc_grid* g, const double* const F[6]);
double orc_kinetic_energy(double m, int64_t np, const double* ux, const double* uy, const double* uz,
                          const double* w);
/* adjoint (pic_oracle_adj.c) */
double orc_dshape(int p, double xi);
void orc_gather_adj(const orc_grid* g, int p, const double* const F[6], double* const lamF[6], const double x[3],
                    const double lamEB[6], double lam_x[3]);
void orc_boris_adj(double q, double m, double dt, const double E[3], const double B[3], const double u_old[3],
                   const double lam_unew[3], double lam_uold[3], double lam_E[3], double lam_B[3]);
void orc_deposit_adj(const orc_grid* g, int p, double dt, double qw, const double x0[3], const double x1[3],
                     const double* const lamJ[3], double lam_x0[3], double lam_x1[3]);
void orc_yee_step_adj(const orc_grid* g, double dt, double* const lamE[3], double* const lamB[3],
                      double* const lamJ[3]);
void orc_pic_adjoint(const orc_grid* g, int p, double dt, double q, double m, int64_t np, double* x, double* y,
                     double* z, double* ux, double* uy, double* uz, const double* w, double* const fields[9],
                     int nsteps, double A, double kd, double* dL_dA, double* dL_du, double* loss);
void orc_curlE(const orc_grid* g, const double* const E[3], double* const out[3]);
void orc_curlE_T(const orc_grid* g, const double* const lamB[3], double* const out[3]);
void orc_curlB_T(const orc_grid* g, const double* const lamE[3], double* const out[3]);
#endif
