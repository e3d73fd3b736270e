/*
 * Plain fp64 CPU oracle for the 25-point acoustic-isotropic wave step with
 * its PML boundary ("Accelerating High-Order Stencils on GPUs",
 * arXiv 2009.04619).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this library: only the test suite, the package's smoke check and the
 * benchmark's CPU-baseline leg use it.  It shares no code, header, table or
 * constant with the CUDA library; both sides only see the same seeded inputs.
 *
 * Layout (the oracle's own, independent of the GPU layout): every field is a
 * dense array of (Nz+2H)*(Ny+2H)*(Nx+2H) doubles, x fastest, with a halo of
 * H = 4 points on every side that holds zeros (u = 0 outside the computed
 * domain).  Nx = nx + 2 nb is the computed extent along x (inner region nx
 * plus a PML of nb points on each side, section III-B), likewise y and z.
 *
 * Parity status: the interior update, the time recurrence, the source
 * scaling and the CFL limit are pinned by closed forms (coefficients,
 * polynomial exactness, Green's function, von Neumann bound).  The PML
 * update is pinned by invariants only (eta = 0 reduction, absorption,
 * symmetry, energy decay) because the paper does not print its formulas:
 * against the paper itself the PML numbers are "parity unpinned".
 */
#ifndef SEISGB_ORACLE_H
#define SEISGB_ORACLE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORA_H 4 /* halo width = stencil radius R (section IV) */

typedef struct {
    int nx, ny, nz; /* inner-region points */
    int nb;         /* PML width per side (0 = no PML, zero walls) */
    double dx, dy, dz, dt;
    double vmax;    /* velocity that sets the PML damping strength */
    double r0;      /* target PML reflection coefficient, 0 < r0 <= 1 */
} ora_grid;

/* Central second-derivative weights of order 2M: w[0..M]. */
void ora_fd2_weights(int M, double *w);
/* 25-point Laplacian coefficients c0, cx[1..4], cy[1..4], cz[1..4] (index 0 unused). */
void ora_laplacian_coeffs(const ora_grid *g, double *c0, double *cx, double *cy, double *cz);
/* Von Neumann stability limit of the leapfrog step with this Laplacian. */
double ora_cfl_dt(double vmax, double dx, double dy, double dz);

size_t ora_field_len(const ora_grid *g);
long ora_index(const ora_grid *g, int i, int j, int k);
int ora_is_pml(const ora_grid *g, int i, int j, int k);
int ora_region(const ora_grid *g, int i, int j, int k);
double ora_eta_axis(int n_inner, int nb, double eta_max, int i);
double ora_eta_max(const ora_grid *g, double h);
void ora_eta(const ora_grid *g, double *eta);

void ora_laplacian(const ora_grid *g, const double *u, double *lap, int nthreads);
void ora_step(const ora_grid *g, const double *m, const double *eta,
              const double *u_prev, const double *u_cur, const double *phi_cur,
              double *u_next, double *phi_next, int nthreads);
void ora_step_points(const ora_grid *g, const float *m, const float *u_prev, const float *u_cur,
                     const float *phi, const int *pts, int npts, double *out_u, double *out_phi,
                     int nthreads);
int ora_run_shot(const ora_grid *g, const float *velocity, const float *wavelet, int nt,
                 const int *src_ijk, const int *rec_ijk, int nrec, double *traces,
                 double *u_final, double *u_prev_final, double *phi_final, int nthreads);

int ora_adjoint_shot(const ora_grid *g, const float *velocity, const float *wavelet, int nt,
                     const int *src_ijk, const int *rec_ijk, int nrec, const double *observed,
                     double *misfit, double *grad_v, int nthreads);

#ifdef __cplusplus
}
#endif
#endif
