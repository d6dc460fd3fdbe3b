/*
 * ssm_oracle.h -- declarations of the FP64 CPU oracle of the split-step method.
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the benchmark's
 * CPU-baseline leg; never by the CUDA library.  Particle arrays are
 * particle-major: x[d*i + c].
 */
#ifndef SSM_ORACLE_H
#define SSM_ORACLE_H

#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

enum { ORC_COEF_CUBIC1D_GAUSS = 0, ORC_COEF_COUPLED3D = 1, ORC_COEF_OU = 2, ORC_COEF_COUPLED1D = 3,
       ORC_COEF_GL1 = 4, ORC_COEF_GL2 = 5, ORC_COEF_POLY = 6, ORC_COEF_CS = 7, ORC_COEF_GLSTAB = 8 };

typedef struct {
    int d;            /* space dimension: 1 or 3 (OU: any) */
    int coef;         /* ORC_COEF_* */
    int64_t N;        /* particles */
    double h;         /* step size */
    double T;         /* horizon (used for the fine Brownian grid) */
    uint64_t seed;    /* Philox key */
    double p[4];      /* OU: rho, lambda, eta; GL1/GL2: sigma', c; POLY: gamma; CS: lambda, sigma';
                         GLSTAB: gamma */
    double x0_mean;   /* X_0 = x0_mean + x0_std * Z */
    double x0_std;
    int fine_log2;    /* 0: own grid; L > 0: Brownian path on the grid T 2^-L */
    int measure_y;    /* coupled sets: 0 = step 1 against mu^X (the SSM); 1 = against
                         mu^Y, the joint R^{dN} system of the earlier implicit scheme */
} orc_problem;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void orc_normals(uint64_t seed, int d, int64_t i, int64_t step, int stream, double *z);
void orc_brownian(const orc_problem *P, int64_t i, int64_t n, double *dw);
double orc_cardano_cubic(double x, double h);
double orc_cardano_gl(double x, double h);
int orc_implicit_point(const orc_problem *P, const double *x, const double *xi, double *y_out);
int orc_implicit_one(const orc_problem *P, const double *x, int64_t i, double *y_out);
void orc_explicit_one(const orc_problem *P, const double *y, int64_t i, int64_t n, double *x_out);
void orc_drift_one(const orc_problem *P, const double *y, int64_t i, double *b_out);
void orc_pair_sum_coupled(const orc_problem *P, const double *x, const double *y,
                          double *S, double *JS);
int orc_implicit_step(const orc_problem *P, const double *x, double *y, int *iters);
void orc_joint_residual_one(const orc_problem *P, const double *x, const double *y, int64_t i, double *g);
void orc_explicit_step(const orc_problem *P, const double *y, int64_t n, double *xnext);
void orc_sample_step(const orc_problem *P, const double *x, double *y, const int64_t *idx, int64_t n,
                     int64_t step, double *xout);
void orc_init_x0(const orc_problem *P, double *x);
void orc_moments(const orc_problem *P, const double *x, double *m);
int orc_run(const orc_problem *P, double *x, int64_t n0, int64_t nsteps, double *mom,
            int64_t *newton_iters_total);
int orc_num_threads(void);

#endif
