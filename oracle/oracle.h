/*
 * oracle.h -- declarations of the FP64 CPU oracle (test infrastructure only).
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg use
 * these functions.  The CUDA library neither includes this header nor links
 * the oracle.
 */
#ifndef PDMTS_ORACLE_H
#define PDMTS_ORACLE_H
#include <stdint.h>

enum { ORC_MICRO_POWER = 0, ORC_MICRO_EXP = 1 };
enum { ORC_FORCE_LINEAR = 0, ORC_FORCE_PMB = 1 };

typedef struct {
    int32_t dim;        /* 2 or 3 */
    int32_t micro_kind; /* ORC_MICRO_POWER: c/|xi|^3 ; ORC_MICRO_EXP: c exp(-|xi|/l) */
    int32_t force_kind; /* ORC_FORCE_LINEAR (Eq. 2) or ORC_FORCE_PMB */
    int32_t breaking;   /* 1: apply Eq. 4 ; 0: bond status frozen */
    int64_t n;          /* number of PD nodes */
    double c;           /* micromodulus constant (PMB c, or c0 of the exponential form) */
    double l;           /* length scale of the exponential form */
    double s0;          /* critical stretch */
    double rho;         /* mass density */
    double dt;          /* time step */
} orc_pd_params;

int orc_set_threads(int n);  /* host threads of the node loops (n <= 0: all); returns the count */
int orc_family(int dim, int64_t n, const double *X, double delta, int64_t *row_ptr, int32_t *col);
int64_t orc_precrack(int dim, int64_t n, const int64_t *P, const int64_t *row_ptr,
                     const int32_t *col, int ncut, const int64_t *cut, uint8_t *mu);
double orc_stretch_literal(int dim, const double *xi, const double *eta);
int64_t orc_pd_forces(const orc_pd_params *p, const double *X, const double *V,
                      const int64_t *row_ptr, const int32_t *col, uint8_t *mu,
                      const double *alpha, const double *u, double *f);
int64_t orc_pd_run(const orc_pd_params *p, const double *X, const double *V,
                   const int64_t *row_ptr, const int32_t *col, uint8_t *mu,
                   const double *alpha, const double *b, const double *g,
                   const double *theta, double theta_init, int init,
                   double *u, double *v, double *a, int64_t nsteps);
void orc_damage(int64_t n, const double *V, const int64_t *row_ptr, const int32_t *col,
                const uint8_t *mu, double *phi);
double orc_strain_energy(const orc_pd_params *p, const double *X, const double *V,
                         const int64_t *row_ptr, const int32_t *col, const uint8_t *mu,
                         const double *alpha, const double *u);
double orc_kinetic_energy(const orc_pd_params *p, const double *V, const double *alpha,
                          const double *v);

#endif
