/*
 * pd_oracle.c -- plain FP64 CPU oracle for bond-based peridynamics (PD).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference that the CUDA path is
 * checked against.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it.  It shares no source, header, table or
 * helper with the CUDA library, and it never calls that library.
 *
 * Everything is written for clarity, not speed: one node at a time, one bond
 * at a time, in ascending neighbour order, in IEEE double precision, compiled
 * with -ffp-contract=off so that no fused multiply-add changes a rounding.
 *
 * What it computes (arXiv 2403.03605, Section 2.1 and Section 2.4):
 *   family      H_delta(x) = { x' : |x' - x| <= delta }            (Sec. 2.1)
 *   motion      rho u'' = sum_j f(xi) V_j + b                       (Eq. 1)
 *   bond force  f = c(|xi|) (xi (x) xi) . eta  (linearised form)    (Eq. 2)
 *   stretch     s = (|xi + eta| - |xi|) / |xi|                      (Eq. 3)
 *   status      mu = 1 while s < s_crit at every step so far         (Eq. 4)
 *   damage      phi = 1 - sum mu V / sum V                          (Eq. 5)
 *   time        Newmark gamma = 1/2, beta = 0 (velocity Verlet)     (Eq. 38)
 * plus the Arlequin weighting of the PD energy by (1 - alpha)        (Eq. 17, Eq. 34)
 *
 * Readings of points the paper leaves open or garbles:
 *  - The breaking test s >= s_crit is evaluated as |xi+eta|^2 >= (1+s0)^2 |xi|^2,
 *    which is the same inequality squared (both sides are non-negative).
 *    orc_stretch_literal() evaluates Eq. 3 literally so a test can check that
 *    the two agree away from exact ties.
 *  - A bond that reaches s >= s_crit at a step carries no force at that step
 *    (Eq. 4 includes t' = t).
 *  - In the Arlequin overlap the PD mass is (1 - alpha_i) rho V_i, loads are
 *    weighted by (1 - alpha_i) and a bond is weighted by
 *    w_ij = 1 - (alpha_i + alpha_j) / 2, which keeps f_ij = -f_ji (Eq. 34).
 *  - The micromodulus of the benchmark plates is the PMB constant c; in the
 *    linearised form of Eq. 2 it becomes c(|xi|) = c / |xi|^3.  The
 *    exponential micromodulus of Sec. 3.2 / Sec. 3.3 is c0 exp(-|xi| / l).
 *  - Pre-cracks are axis-aligned cuts; a bond is cut when its end points lie
 *    strictly on opposite sides of the cut plane and the crossing point lies in
 *    the half-open range [lo, hi) along the cut.  It is evaluated exactly in
 *    integer lattice units.
 *
 * Layout: every per-node vector field is structure-of-arrays, component d of
 * node i at [d * n + i].  The family is CSR: row_ptr[n + 1], col[row_ptr[n]],
 * with each row sorted ascending.  Bond status is one byte per CSR entry.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Host threads.  The node loops below may run on several threads: node i    */
/* reads u, X, V and alpha and writes only its own row of mu and its own      */
/* force, so the result does not depend on the thread count.  The default is  */
/* one thread; the benchmark's CPU baseline asks for every core.             */
/* ------------------------------------------------------------------------ */
static int g_threads = 1;

int orc_set_threads(int n)
{
#ifdef _OPENMP
    g_threads = n > 0 ? n : omp_get_num_procs();
#else
    (void)n;
    g_threads = 1;
#endif
    return g_threads;
}

/* ------------------------------------------------------------------------ */
/* Micromodulus c(|xi|) (Eq. 2 with the readings above).                     */
/* ------------------------------------------------------------------------ */
static double micromodulus(const orc_pd_params *p, double xi2)
{
    double r = sqrt(xi2);
    if (p->micro_kind == ORC_MICRO_EXP)
        return p->c * exp(-r / p->l);
    /* power law: c(|xi|) = c_PMB / |xi|^3 */
    return p->c / (xi2 * r);
}

/* ------------------------------------------------------------------------ */
/* Family search (Sec. 2.1): all j != i with |x_j - x_i|^2 <= delta^2.        */
/* A uniform bin grid of cell size delta limits the candidates to the 3^d    */
/* surrounding cells; each row is then sorted ascending.                     */
/* If col is NULL only row_ptr is filled (pass 1).                           */
/* ------------------------------------------------------------------------ */
static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

int orc_family(int dim, int64_t n, const double *X, double delta,
               int64_t *row_ptr, int32_t *col)
{
    if (dim < 1 || dim > 3 || n < 0 || delta <= 0.0)
        return -1;
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    int64_t nb[3] = {1, 1, 1};
    for (int d = 0; d < dim; ++d) {
        lo[d] = hi[d] = n > 0 ? X[d * n] : 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double x = X[d * n + i];
            if (x < lo[d]) lo[d] = x;
            if (x > hi[d]) hi[d] = x;
        }
        nb[d] = (int64_t)floor((hi[d] - lo[d]) / delta) + 1;
    }
    int64_t ncell = nb[0] * nb[1] * nb[2];
    int64_t *head = malloc(sizeof(int64_t) * (size_t)ncell);
    int64_t *next = malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *cell = malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1) * 3);
    if (!head || !next || !cell) {
        free(head); free(next); free(cell);
        return -2;
    }
    for (int64_t c = 0; c < ncell; ++c) head[c] = -1;
    for (int64_t i = n - 1; i >= 0; --i) {
        int64_t id = 0;
        for (int d = 2; d >= 0; --d) {
            int64_t k = 0;
            if (d < dim) {
                k = (int64_t)floor((X[d * n + i] - lo[d]) / delta);
                if (k >= nb[d]) k = nb[d] - 1;
            }
            cell[3 * i + d] = k;
            id = id * nb[d] + k;
        }
        next[i] = head[id];
        head[id] = i;
    }
    double d2max = delta * delta;
    int64_t total = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (row_ptr) row_ptr[i] = total;
        int64_t start = total;
        for (int64_t c2 = -1; c2 <= 1; ++c2)
        for (int64_t c1 = -1; c1 <= 1; ++c1)
        for (int64_t c0 = -1; c0 <= 1; ++c0) {
            int64_t off[3] = {c0, c1, c2};
            int64_t k[3];
            int skip = 0;
            for (int d = 0; d < 3; ++d) {
                if (d >= dim && off[d] != 0) { skip = 1; break; }
                k[d] = cell[3 * i + d] + off[d];
                if (k[d] < 0 || k[d] >= nb[d]) { skip = 1; break; }
            }
            if (skip) continue;
            int64_t id = (k[2] * nb[1] + k[1]) * nb[0] + k[0];
            for (int64_t j = head[id]; j >= 0; j = next[j]) {
                if (j == i) continue;
                double r2 = 0.0;
                for (int d = 0; d < dim; ++d) {
                    double xi = X[d * n + j] - X[d * n + i];
                    r2 += xi * xi;
                }
                if (r2 <= d2max) {
                    if (col) col[total] = (int32_t)j;
                    ++total;
                }
            }
        }
        if (col) qsort(col + start, (size_t)(total - start), sizeof(int32_t), cmp_i32);
    }
    if (row_ptr) row_ptr[n] = total;
    free(head); free(next); free(cell);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Pre-crack (reading of the benchmark set-up, exact in integer units).      */
/* P holds integer node coordinates (dim * n, SoA) in the same unit as the   */
/* cut description cut[5 * c + {normal axis, level, along axis, lo, hi}].    */
/* Sets mu = 0 for every CSR bond that crosses a cut; returns the number of  */
/* directed bonds cut.                                                       */
/* ------------------------------------------------------------------------ */
int64_t orc_precrack(int dim, int64_t n, const int64_t *P, const int64_t *row_ptr,
                     const int32_t *col, int ncut, const int64_t *cut, uint8_t *mu)
{
    int64_t count = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            int64_t j = col[k];
            int is_cut = 0;
            for (int c = 0; c < ncut && !is_cut; ++c) {
                int na = (int)cut[5 * c + 0], pa = (int)cut[5 * c + 2];
                int64_t level = cut[5 * c + 1], lo = cut[5 * c + 3], hi = cut[5 * c + 4];
                if (na >= dim || pa >= dim) continue;
                int64_t ni = P[na * n + i], nj = P[na * n + j];
                int64_t ai = P[pa * n + i], aj = P[pa * n + j];
                /* strictly opposite sides of the cut plane */
                if (!((ni < level && nj > level) || (ni > level && nj < level)))
                    continue;
                /* crossing coordinate a_c = ai + (level - ni) (aj - ai) / (nj - ni) */
                int64_t D = nj - ni;
                int64_t num = ai * D + (level - ni) * (aj - ai); /* a_c = num / D */
                int ge_lo, lt_hi;
                if (D > 0) {
                    ge_lo = num >= lo * D;
                    lt_hi = num < hi * D;
                } else {
                    ge_lo = num <= lo * D;
                    lt_hi = num > hi * D;
                }
                if (ge_lo && lt_hi) is_cut = 1;
            }
            if (is_cut) {
                mu[k] = 0;
                ++count;
            }
        }
    }
    return count;
}

/* ------------------------------------------------------------------------ */
/* Eq. 3, literally.                                                         */
/* ------------------------------------------------------------------------ */
double orc_stretch_literal(int dim, const double *xi, const double *eta)
{
    double a = 0.0, b = 0.0;
    for (int d = 0; d < dim; ++d) {
        a += (xi[d] + eta[d]) * (xi[d] + eta[d]);
        b += xi[d] * xi[d];
    }
    return (sqrt(a) - sqrt(b)) / sqrt(b);
}

/* ------------------------------------------------------------------------ */
/* Internal force density f_i = sum_j w_ij mu_ij f(xi_ij) V_j  (Eq. 1, 2, 4). */
/* If p->breaking, bonds with s >= s0 are switched off first (Eq. 4).        */
/* Returns the number of bonds broken by this call.                          */
/* ------------------------------------------------------------------------ */
int64_t orc_pd_forces(const orc_pd_params *p, const double *X, const double *V,
                      const int64_t *row_ptr, const int32_t *col, uint8_t *mu,
                      const double *alpha, const double *u, double *f)
{
    const int dim = p->dim;
    const int64_t n = p->n;
    const double s0p2 = (1.0 + p->s0) * (1.0 + p->s0);
    int64_t newly = 0;
#pragma omp parallel for schedule(static) reduction(+ : newly) num_threads(g_threads)
    for (int64_t i = 0; i < n; ++i) {
        double fi[3] = {0.0, 0.0, 0.0};
        double ai = alpha ? alpha[i] : 0.0;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            if (!mu[k]) continue;
            int64_t j = col[k];
            double xi[3], eta[3];
            double xi2 = 0.0, y2 = 0.0, dot = 0.0;
            for (int d = 0; d < dim; ++d) {
                xi[d] = X[d * n + j] - X[d * n + i];   /* bond, Sec. 2.1 */
                eta[d] = u[d * n + j] - u[d * n + i];  /* relative displacement */
            }
            for (int d = 0; d < dim; ++d) xi2 += xi[d] * xi[d];
            for (int d = 0; d < dim; ++d) {
                double y = xi[d] + eta[d];
                y2 += y * y;
            }
            if (p->breaking && y2 >= s0p2 * xi2) {        /* s >= s0, Eq. 3-4 */
                mu[k] = 0;
                ++newly;
                continue;
            }
            double aj = alpha ? alpha[j] : 0.0;
            double w = 1.0 - 0.5 * (ai + aj);
            double c = micromodulus(p, xi2);
            if (p->force_kind == ORC_FORCE_PMB) {
                /* PMB: f = c_PMB s (xi + eta) / |xi + eta|, with c(|xi|) = c_PMB / |xi|^3 */
                double r = sqrt(xi2), ry = sqrt(y2);
                double s = (ry - r) / r;
                double cp = c * xi2 * r;
                double sc = w * cp * s / ry * V[j];
                for (int d = 0; d < dim; ++d) fi[d] += sc * (xi[d] + eta[d]);
            } else {
                for (int d = 0; d < dim; ++d) dot += xi[d] * eta[d];
                double sc = w * c * dot * V[j];
                for (int d = 0; d < dim; ++d) fi[d] += sc * xi[d];
            }
        }
        for (int d = 0; d < dim; ++d) f[d * n + i] = fi[d];
    }
    return newly;
}

/* ------------------------------------------------------------------------ */
/* Acceleration from force density, Eq. 33 (PD row) with Eq. 34 weights:      */
/*   a_i = (f_i + (1 - alpha_i) b_i + theta g_i) / ((1 - alpha_i) rho)        */
/* g is the interface force per unit volume (G^PD^T lambda / V), may be NULL. */
/* ------------------------------------------------------------------------ */
static void accel(const orc_pd_params *p, const double *alpha, const double *b,
                  const double *g, double theta, const double *f, double *a)
{
    const int dim = p->dim;
    const int64_t n = p->n;
    for (int64_t i = 0; i < n; ++i) {
        double ai = alpha ? alpha[i] : 0.0;
        double m = (1.0 - ai) * p->rho;
        for (int d = 0; d < dim; ++d) {
            double t = f[d * n + i];
            if (b) t = t + (1.0 - ai) * b[d * n + i];
            if (g) t = t + theta * g[d * n + i];
            a[d * n + i] = t / m;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Velocity-Verlet time stepping (Eq. 38 with gamma = 1/2, beta = 0):         */
/*   u_{k+1} = u_k + dt v_k + dt^2/2 a_k                                      */
/*   a_{k+1} = M^-1 (forces at u_{k+1})                                       */
/*   v_{k+1} = v_k + dt/2 (a_k + a_{k+1})                                     */
/* If init != 0, a_0 is first computed from u_0 (breaking as configured) with */
/* theta_init.  theta[k] (or 0 if theta is NULL) scales g at step k+1.        */
/* Returns the total number of bonds broken, or -1 on a bad argument.         */
/* ------------------------------------------------------------------------ */
int64_t orc_pd_run(const orc_pd_params *p, const double *X, const double *V,
                   const int64_t *row_ptr, const int32_t *col, uint8_t *mu,
                   const double *alpha, const double *b, const double *g,
                   const double *theta, double theta_init, int init,
                   double *u, double *v, double *a, int64_t nsteps)
{
    if (!p || p->dim < 1 || p->dim > 3 || p->n < 0) return -1;
    const int dim = p->dim;
    const int64_t n = p->n;
    const double dt = p->dt;
    const double hdt = 0.5 * dt;
    const double hdt2 = 0.5 * dt * dt;
    double *f = malloc(sizeof(double) * (size_t)(dim * n > 0 ? dim * n : 1));
    double *an = malloc(sizeof(double) * (size_t)(dim * n > 0 ? dim * n : 1));
    if (!f || !an) { free(f); free(an); return -1; }
    int64_t broken = 0;
    if (init) {
        broken += orc_pd_forces(p, X, V, row_ptr, col, mu, alpha, u, f);
        accel(p, alpha, b, g, theta_init, f, a);
    }
    for (int64_t k = 0; k < nsteps; ++k) {
        for (int64_t q = 0; q < dim * n; ++q)
            u[q] = u[q] + dt * v[q] + hdt2 * a[q];
        broken += orc_pd_forces(p, X, V, row_ptr, col, mu, alpha, u, f);
        accel(p, alpha, b, g, theta ? theta[k] : 0.0, f, an);
        for (int64_t q = 0; q < dim * n; ++q) {
            v[q] = v[q] + hdt * (a[q] + an[q]);
            a[q] = an[q];
        }
    }
    free(f); free(an);
    return broken;
}

/* ------------------------------------------------------------------------ */
/* Damage, Eq. 5: phi_i = 1 - sum_j mu_ij V_j / sum_j V_j.                    */
/* ------------------------------------------------------------------------ */
void orc_damage(int64_t n, const double *V, const int64_t *row_ptr, const int32_t *col,
                const uint8_t *mu, double *phi)
{
    for (int64_t i = 0; i < n; ++i) {
        double num = 0.0, den = 0.0;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            den += V[col[k]];
            if (mu[k]) num += V[col[k]];
        }
        phi[i] = den > 0.0 ? 1.0 - num / den : 0.0;
    }
}

/* ------------------------------------------------------------------------ */
/* Elastic energy of the linearised bond model (Eq. 6 in nodal quadrature):   */
/*   Pi = 1/4 sum_i sum_j w_ij mu_ij c(|xi|) (xi . eta)^2 V_i V_j             */
/* and kinetic energy 1/2 sum_i (1 - alpha_i) rho V_i |v_i|^2 (Eq. 15-16).    */
/* ------------------------------------------------------------------------ */
double orc_strain_energy(const orc_pd_params *p, const double *X, const double *V,
                         const int64_t *row_ptr, const int32_t *col, const uint8_t *mu,
                         const double *alpha, const double *u)
{
    const int dim = p->dim;
    const int64_t n = p->n;
    double e = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double ai = alpha ? alpha[i] : 0.0;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            if (!mu[k]) continue;
            int64_t j = col[k];
            double xi2 = 0.0, dot = 0.0;
            for (int d = 0; d < dim; ++d) {
                double xi = X[d * n + j] - X[d * n + i];
                double eta = u[d * n + j] - u[d * n + i];
                xi2 += xi * xi;
                dot += xi * eta;
            }
            double aj = alpha ? alpha[j] : 0.0;
            double w = 1.0 - 0.5 * (ai + aj);
            e += 0.25 * w * micromodulus(p, xi2) * dot * dot * V[i] * V[j];
        }
    }
    return e;
}

double orc_kinetic_energy(const orc_pd_params *p, const double *V, const double *alpha,
                          const double *v)
{
    const int dim = p->dim;
    const int64_t n = p->n;
    double e = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double ai = alpha ? alpha[i] : 0.0;
        double m = (1.0 - ai) * p->rho * V[i];
        for (int d = 0; d < dim; ++d) e += 0.5 * m * v[d * n + i] * v[d * n + i];
    }
    return e;
}
