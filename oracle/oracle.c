/*
 * Plain fp64 CPU oracle for the 25-point acoustic-isotropic wave step with a
 * PML boundary (arXiv 2009.04619, section III-A).
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path.  Shares no code
 * with the CUDA library.  Written for a reader checking it against the paper:
 * no blocking, fusion or reordering beyond what the equations state.
 *
 * Readings of passages the paper leaves open (each listed in the design
 * notes):
 *  - Laplacian coefficients (section III-A, Eq. 3 names them c_xyz, c_xm,
 *    c_ym, c_zm without values): the standard 8th-order central
 *    second-derivative weights, c_xm = w_m / dx^2 and
 *    c_xyz = w_0 (1/dx^2 + 1/dy^2 + 1/dz^2).
 *  - Time recurrence (Eq. 2, Algorithm 1): the step with index n maps
 *    (u^{n-1}, u^n) to u^{n+1}; u^0 = u^{-1} = 0; the source term of Eq. 2's
 *    right-hand side, dt^2 V^2 f^n, is added into u^{n+1}.
 *  - Source f = w(t) delta(x - x_s): one grid point, amplitude w / (dx dy dz).
 *  - PML (section III-A names a PML and a 7-point stencil on an eta array
 *    with halo 1, section IV; no formulas): single isotropic complex stretch
 *    s = 1 + eta / (i omega), giving
 *        u_tt + 2 eta u_t + eta^2 u = V^2 (lap u + phi),
 *        phi_t + eta phi = - grad(eta) . grad(u),
 *    discretised with centred u_t, backward-Euler damping on phi and 2nd
 *    order central differences (the 7-point star) for both gradients.
 *    eta = eta_x(i) + eta_y(j) + eta_z(k), eta_a = eta_max (d / nb)^2 with d
 *    the distance in points into the layer, eta_max = -3 vmax ln(r0)/(2 nb h).
 *    The PML update is applied at computed points outside the inner box; the
 *    inner box uses Eq. 2 unchanged.
 *  - Outside the computed domain u = 0 (zero halo, never written).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define R ORA_H

static int ext_x(const ora_grid *g) { return g->nx + 2 * g->nb; }
static int ext_y(const ora_grid *g) { return g->ny + 2 * g->nb; }
static int ext_z(const ora_grid *g) { return g->nz + 2 * g->nb; }

size_t ora_field_len(const ora_grid *g)
{
    return (size_t)(ext_x(g) + 2 * R) * (size_t)(ext_y(g) + 2 * R) * (size_t)(ext_z(g) + 2 * R);
}

/* Flat index of computed point (i, j, k); -R <= i < Nx + R etc.  x is the
 * innermost (fastest) dimension, as the paper stores the grid (section IV-A). */
long ora_index(const ora_grid *g, int i, int j, int k)
{
    long sx = ext_x(g) + 2 * R, sy = ext_y(g) + 2 * R;
    return ((long)(k + R) * sy + (j + R)) * sx + (i + R);
}

/* Central second-derivative weights of order 2M (Fornberg's closed form):
 *   w_m = 2 (-1)^{m+1} (M!)^2 / (m^2 (M-m)! (M+m)!),  w_0 = -2 sum_m w_m.
 * For M = 4 these are the coefficients of the 8th-order, radius-4 stencil of
 * section III-A. */
void ora_fd2_weights(int M, double *w)
{
    double fM = 1.0;
    for (int q = 2; q <= M; ++q) fM *= q;
    double s = 0.0;
    for (int m = 1; m <= M; ++m) {
        double a = 1.0, b = 1.0;
        for (int q = 2; q <= M - m; ++q) a *= q;
        for (int q = 2; q <= M + m; ++q) b *= q;
        double sign = (m % 2 == 1) ? 1.0 : -1.0;
        w[m] = 2.0 * sign * fM * fM / ((double)m * m * a * b);
        s += w[m];
    }
    w[0] = -2.0 * s;
}

/* Coefficients of the 25-point Laplacian, section III-A (Eq. 3). */
void ora_laplacian_coeffs(const ora_grid *g, double *c0, double *cx, double *cy, double *cz)
{
    double w[R + 1];
    ora_fd2_weights(R, w);
    double ix = 1.0 / (g->dx * g->dx), iy = 1.0 / (g->dy * g->dy), iz = 1.0 / (g->dz * g->dz);
    *c0 = w[0] * (ix + iy + iz);
    cx[0] = cy[0] = cz[0] = 0.0;
    for (int m = 1; m <= R; ++m) {
        cx[m] = w[m] * ix;
        cy[m] = w[m] * iy;
        cz[m] = w[m] * iz;
    }
}

/* Von Neumann limit of the leapfrog step of Eq. 2 with the Laplacian above:
 * the amplification stays on the unit circle while dt^2 V^2 max|symbol| <= 4.
 * The 1D symbol -(w_0 + 2 sum_m w_m cos(m theta)) peaks at theta = pi. */
double ora_cfl_dt(double vmax, double dx, double dy, double dz)
{
    double w[R + 1];
    ora_fd2_weights(R, w);
    double S = w[0];
    for (int m = 1; m <= R; ++m) S += 2.0 * w[m] * ((m % 2) ? -1.0 : 1.0);
    S = fabs(S);
    double sum = S * (1.0 / (dx * dx) + 1.0 / (dy * dy) + 1.0 / (dz * dz));
    return 2.0 / (vmax * sqrt(sum));
}

/* Distance (points) of index i into the PML along one axis: 0 inside
 * [nb, nb + n_inner), growing by one per point outward on either side. */
static int pml_depth(int n_inner, int nb, int i)
{
    int d = 0;
    if (nb - i > d) d = nb - i;
    if (i - (nb + n_inner - 1) > d) d = i - (nb + n_inner - 1);
    return d;
}

double ora_eta_max(const ora_grid *g, double h)
{
    if (g->nb <= 0) return 0.0;
    return -3.0 * g->vmax * log(g->r0) / (2.0 * g->nb * h);
}

/* Damping profile along one axis: eta_max (d / nb)^2. */
double ora_eta_axis(int n_inner, int nb, double eta_max, int i)
{
    if (nb <= 0) return 0.0;
    double d = (double)pml_depth(n_inner, nb, i);
    return eta_max * (d / nb) * (d / nb);
}

/* The eta array of section IV-A (3D blocking using shared memory for the
 * boundary regions): eta_x(i) + eta_y(j) + eta_z(k), defined on the computed
 * domain and its halo. */
void ora_eta(const ora_grid *g, double *eta)
{
    double ex = ora_eta_max(g, g->dx), ey = ora_eta_max(g, g->dy), ez = ora_eta_max(g, g->dz);
    for (int k = -R; k < ext_z(g) + R; ++k)
        for (int j = -R; j < ext_y(g) + R; ++j)
            for (int i = -R; i < ext_x(g) + R; ++i)
                eta[ora_index(g, i, j, k)] = ora_eta_axis(g->nx, g->nb, ex, i) +
                                             ora_eta_axis(g->ny, g->nb, ey, j) +
                                             ora_eta_axis(g->nz, g->nb, ez, k);
}

/* A computed point lies in the PML when it is outside the inner box
 * (section III-B). */
int ora_is_pml(const ora_grid *g, int i, int j, int k)
{
    return pml_depth(g->nx, g->nb, i) > 0 || pml_depth(g->ny, g->nb, j) > 0 ||
           pml_depth(g->nz, g->nb, k) > 0;
}

/* The seven-region decomposition of section III-B (Fig. 1): 0 inner,
 * 1 top / 2 bottom (full x and y, cut along z), 3 front / 4 back (full x,
 * inner z, cut along y), 5 left / 6 right (inner y and z, cut along x). */
int ora_region(const ora_grid *g, int i, int j, int k)
{
    int nb = g->nb;
    if (k < nb) return 1;
    if (k >= nb + g->nz) return 2;
    if (j < nb) return 3;
    if (j >= nb + g->ny) return 4;
    if (i < nb) return 5;
    if (i >= nb + g->nx) return 6;
    return 0;
}

static int pick_threads(int nthreads)
{
#ifdef _OPENMP
    return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

/* 25-point star Laplacian at every computed point (section III-A, Eq. 3). */
void ora_laplacian(const ora_grid *g, const double *u, double *lap, int nthreads)
{
    double c0, cx[R + 1], cy[R + 1], cz[R + 1];
    ora_laplacian_coeffs(g, &c0, cx, cy, cz);
    long sx = ext_x(g) + 2 * R, sxy = sx * (ext_y(g) + 2 * R);
    int Nx = ext_x(g), Ny = ext_y(g), Nz = ext_z(g);
    int nth = pick_threads(nthreads);
#pragma omp parallel for num_threads(nth) schedule(static)
    for (int k = 0; k < Nz; ++k)
        for (int j = 0; j < Ny; ++j)
            for (int i = 0; i < Nx; ++i) {
                long p = ora_index(g, i, j, k);
                double L = c0 * u[p];
                for (int m = 1; m <= R; ++m)
                    L += cx[m] * (u[p + m] + u[p - m]) + cy[m] * (u[p + m * sx] + u[p - m * sx]) +
                         cz[m] * (u[p + m * sxy] + u[p - m * sxy]);
                lap[p] = L;
            }
}

/* Values one point's update reads: the 25-point star of u^n along each axis
 * (u[a][R + o] = u^n at offset o on axis a, |o| <= R), eta at offsets -1, 0,
 * +1 on each axis, and m, u^{n-1}, phi^n at the point. */
typedef struct {
    double u[3][2 * R + 1];
    double eta[3][3];
    double m, u_prev, phi;
    int pml;
} ora_star;

/* One point of one time step: Eq. 2 in the inner region, the PML reading
 * above outside it.  m = V^2 dt^2. */
static void star_update(const ora_grid *g, double c0, const double *cx, const double *cy,
                        const double *cz, const ora_star *s, double *u_next, double *phi_next)
{
    const double *cc[3] = {cx, cy, cz};
    const double h[3] = {g->dx, g->dy, g->dz};
    double u0 = s->u[0][R];
    double L = c0 * u0;
    for (int mm = 1; mm <= R; ++mm)
        L += cc[0][mm] * (s->u[0][R + mm] + s->u[0][R - mm]) +
             cc[1][mm] * (s->u[1][R + mm] + s->u[1][R - mm]) +
             cc[2][mm] * (s->u[2][R + mm] + s->u[2][R - mm]);
    if (!s->pml) {
        /* Eq. 2: u^{n+1} = (2 + dt^2 V^2 lap) u^n - u^{n-1} */
        *u_next = 2.0 * u0 - s->u_prev + s->m * L;
        *phi_next = s->phi;
        return;
    }
    double dt = g->dt;
    double e = s->eta[0][1] * dt;
    /* grad(eta) . grad(u) with 2nd-order central differences (the 7-point star
     * on eta, halo 1) */
    double gd[3];
    for (int ax = 0; ax < 3; ++ax)
        gd[ax] = (s->eta[ax][2] - s->eta[ax][0]) / (2.0 * h[ax]) *
                 ((s->u[ax][R + 1] - s->u[ax][R - 1]) / (2.0 * h[ax]));
    double gsum = gd[0] + gd[1] + gd[2];
    *u_next = ((2.0 - e * e) * u0 - (1.0 - e) * s->u_prev + s->m * (L + s->phi)) / (1.0 + e);
    *phi_next = (s->phi - dt * gsum) / (1.0 + e);
}

/* One time step at every computed point: writes u^{n+1} and phi^{n+1}. */
void ora_step(const ora_grid *g, const double *m, const double *eta, const double *u_prev,
              const double *u_cur, const double *phi_cur, double *u_next, double *phi_next,
              int nthreads)
{
    double c0, cx[R + 1], cy[R + 1], cz[R + 1];
    ora_laplacian_coeffs(g, &c0, cx, cy, cz);
    long sx = ext_x(g) + 2 * R, sxy = sx * (ext_y(g) + 2 * R);
    const long st[3] = {1, sx, sxy};
    int Nx = ext_x(g), Ny = ext_y(g), Nz = ext_z(g);
    int nth = pick_threads(nthreads);
#pragma omp parallel for num_threads(nth) schedule(static)
    for (int k = 0; k < Nz; ++k)
        for (int j = 0; j < Ny; ++j)
            for (int i = 0; i < Nx; ++i) {
                long p = ora_index(g, i, j, k);
                ora_star s;
                for (int ax = 0; ax < 3; ++ax) {
                    for (int o = -R; o <= R; ++o) s.u[ax][R + o] = u_cur[p + o * st[ax]];
                    for (int o = -1; o <= 1; ++o) s.eta[ax][o + 1] = eta[p + o * st[ax]];
                }
                s.m = m[p];
                s.u_prev = u_prev[p];
                s.phi = phi_cur[p];
                s.pml = ora_is_pml(g, i, j, k);
                star_update(g, c0, cx, cy, cz, &s, &u_next[p], &phi_next[p]);
            }
}

/* The same step evaluated at listed points only, reading fp32 compact fields
 * (Nz*Ny*Nx, x fastest; zero outside the computed domain) and the eta profile
 * directly.  Lets a test check a full-size GPU step on sampled outputs.
 * pts: npts triples (i, j, k); out_u / out_phi: npts doubles. */
void ora_step_points(const ora_grid *g, const float *m, const float *u_prev, const float *u_cur,
                     const float *phi, const int *pts, int npts, double *out_u, double *out_phi,
                     int nthreads)
{
    double c0, cx[R + 1], cy[R + 1], cz[R + 1];
    ora_laplacian_coeffs(g, &c0, cx, cy, cz);
    int N[3] = {ext_x(g), ext_y(g), ext_z(g)};
    int nin[3] = {g->nx, g->ny, g->nz};
    double emax[3] = {ora_eta_max(g, g->dx), ora_eta_max(g, g->dy), ora_eta_max(g, g->dz)};
    int nth = pick_threads(nthreads);
#pragma omp parallel for num_threads(nth) schedule(static)
    for (int q = 0; q < npts; ++q) {
        int c[3] = {pts[3 * q], pts[3 * q + 1], pts[3 * q + 2]};
        ora_star s;
        for (int ax = 0; ax < 3; ++ax) {
            for (int o = -R; o <= R; ++o) {
                int d[3] = {c[0], c[1], c[2]};
                d[ax] += o;
                int inside = d[0] >= 0 && d[0] < N[0] && d[1] >= 0 && d[1] < N[1] && d[2] >= 0 &&
                             d[2] < N[2];
                s.u[ax][R + o] =
                    inside ? (double)u_cur[((size_t)d[2] * N[1] + d[1]) * N[0] + d[0]] : 0.0;
            }
            for (int o = -1; o <= 1; ++o) {
                double e = 0.0;
                for (int b = 0; b < 3; ++b)
                    e += ora_eta_axis(nin[b], g->nb, emax[b], c[b] + (b == ax ? o : 0));
                s.eta[ax][o + 1] = e;
            }
        }
        size_t ci = ((size_t)c[2] * N[1] + c[1]) * N[0] + c[0];
        s.m = (double)m[ci];
        s.u_prev = (double)u_prev[ci];
        s.phi = (double)phi[ci];
        s.pml = ora_is_pml(g, c[0], c[1], c[2]);
        star_update(g, c0, cx, cy, cz, &s, &out_u[q], &out_phi[q]);
    }
}

/* Algorithm 1: the time loop with source injection, plus receiver sampling
 * of u^{n+1} after injection.  Inputs are the fp32 values the GPU sees,
 * widened to double; m = v^2 dt^2 is formed in double.
 *   velocity: Nz*Ny*Nx floats (computed domain, x fastest)
 *   wavelet:  nt floats, w(n dt)
 *   traces:   nt*nrec doubles, traces[n*nrec + r] = u^{n+1}(rec_r)
 *   u_final, u_prev_final, phi_final: Nz*Ny*Nx doubles or NULL.
 * Returns 0, or -1 on bad arguments / allocation failure. */
int ora_run_shot(const ora_grid *g, const float *velocity, const float *wavelet, int nt,
                 const int *src_ijk, const int *rec_ijk, int nrec, double *traces,
                 double *u_final, double *u_prev_final, double *phi_final, int nthreads)
{
    int Nx = ext_x(g), Ny = ext_y(g), Nz = ext_z(g);
    if (Nx <= 0 || Ny <= 0 || Nz <= 0 || nt < 0) return -1;
    size_t n = ora_field_len(g);
    double *buf = (double *)calloc(6 * n, sizeof(double));
    if (!buf) return -1;
    double *m = buf, *eta = buf + n, *u0 = buf + 2 * n, *u1 = buf + 3 * n, *u2 = buf + 4 * n,
           *phi = buf + 5 * n;
    double *phi_next = (double *)calloc(n, sizeof(double));
    if (!phi_next) {
        free(buf);
        return -1;
    }
    double dt = g->dt;
    for (int k = 0; k < Nz; ++k)
        for (int j = 0; j < Ny; ++j)
            for (int i = 0; i < Nx; ++i) {
                double v = (double)velocity[((size_t)k * Ny + j) * Nx + i];
                m[ora_index(g, i, j, k)] = v * v * dt * dt;
            }
    ora_eta(g, eta);
    double inv_vol = 1.0 / (g->dx * g->dy * g->dz);
    long ps = src_ijk ? ora_index(g, src_ijk[0], src_ijk[1], src_ijk[2]) : -1;
    double *u_prev = u0, *u_cur = u1, *u_next = u2;
    for (int step = 0; step < nt; ++step) {
        ora_step(g, m, eta, u_prev, u_cur, phi, u_next, phi_next, nthreads);
        if (ps >= 0) u_next[ps] += m[ps] * (double)wavelet[step] * inv_vol; /* Eq. 2 RHS */
        for (int r = 0; r < nrec; ++r)
            traces[(size_t)step * nrec + r] =
                u_next[ora_index(g, rec_ijk[3 * r], rec_ijk[3 * r + 1], rec_ijk[3 * r + 2])];
        double *t = u_prev;
        u_prev = u_cur;
        u_cur = u_next;
        u_next = t;
        t = phi;
        phi = phi_next;
        phi_next = t;
    }
    for (int k = 0; k < Nz; ++k)
        for (int j = 0; j < Ny; ++j)
            for (int i = 0; i < Nx; ++i) {
                size_t c = ((size_t)k * Ny + j) * Nx + i;
                long p = ora_index(g, i, j, k);
                if (u_final) u_final[c] = u_cur[p];
                if (u_prev_final) u_prev_final[c] = u_prev[p];
                if (phi_final) phi_final[c] = phi[p];
            }
    /* phi and phi_next may have swapped: free whichever pointer is not in buf */
    if (phi == buf + 5 * n) free(phi_next);
    else free(phi);
    free(buf);
    return 0;
}

/* ------------------------------------------------------------------------
 * Gradient of the trace misfit with respect to the velocity model.
 *
 * The paper has no adjoint; this is the exact discrete adjoint of the step
 * above (Eq. 2 with the PML reading), written in the scaled variable
 * w = M lambda, where lambda is the Lagrange multiplier of u and M the
 * coefficient of (L u + phi + f) in the update (m inside, m / (1 + e) in the
 * PML).  Backward in time, k = nt .. 1, starting from zero:
 *   psi(x)  = sum_a [c_a nu(x + e_a) - c_a nu(x - e_a)] / (2 h_a),
 *             c_a = dt (d eta / d x_a) / (1 + e) at PML points, 0 elsewhere
 *             (the transpose of phi's grad(eta).grad(u) coupling);
 *   w^k     = 2 w^{k+1} - w^{k+2} + m (L w^{k+1} + psi + K^T r^{k-1})   inside,
 *             [(2 - e^2) w^{k+1} - (1 - e) w^{k+2} + m (...)] / (1 + e)   in the PML;
 *   nu^k    = nu^{k+1} / (1 + e) + w^{k+1} at PML points (0 elsewhere);
 *   dJ/dm  += w^k g^{k-1} / m,  g^n = L u^n + phi^n + f^n (forward);
 * with r^n = d^n - obs^n the trace residual of J = 1/2 sum (d - obs)^2.
 * Finally dJ/dv = dJ/dm * 2 v dt^2 (dt held fixed).  Plain: the forward
 * history of g is kept whole (small grids only).
 * ------------------------------------------------------------------------ */
int ora_adjoint_shot(const ora_grid *g, const float *velocity, const float *wavelet, int nt,
                     const int *src_ijk, const int *rec_ijk, int nrec, const double *observed,
                     double *misfit, double *grad_v, int nthreads)
{
    int Nx = ext_x(g), Ny = ext_y(g), Nz = ext_z(g);
    if (Nx <= 0 || Ny <= 0 || Nz <= 0 || nt < 1) return -1;
    size_t n = ora_field_len(g);
    long sx = Nx + 2 * R, sxy = sx * (Ny + 2 * R);
    const long st3[3] = {1, sx, sxy};
    const double hh[3] = {g->dx, g->dy, g->dz};
    /* every work array in one table, so that a failed allocation frees the rest */
    enum { A_M, A_ETA, A_UA, A_UB, A_UC, A_PA, A_PB, A_LAP, A_GACC, A_TR, A_W1, A_W2, A_WK,
           A_NU, A_NUN, A_PSI, A_GM, A_WL, A_COUNT };
    double *arr[A_COUNT];
    int ok = 1;
    for (int q = 0; q < A_COUNT; ++q) {
        size_t len = q == A_GACC ? n * (size_t)nt
                   : q == A_TR   ? (size_t)nt * (nrec > 0 ? nrec : 1)
                                 : n;
        arr[q] = calloc(len, sizeof(double));
        ok = ok && arr[q] != NULL;
    }
    if (!ok) {
        for (int q = 0; q < A_COUNT; ++q) free(arr[q]);
        return -1;
    }
    double *m = arr[A_M], *eta = arr[A_ETA], *ua = arr[A_UA], *ub = arr[A_UB], *uc = arr[A_UC];
    double *pa = arr[A_PA], *pb = arr[A_PB], *lap = arr[A_LAP], *gacc = arr[A_GACC];
    double *traces = arr[A_TR], *w1 = arr[A_W1], *w2 = arr[A_W2], *wk = arr[A_WK];
    double *nu = arr[A_NU], *nun = arr[A_NUN], *psi = arr[A_PSI], *gm = arr[A_GM], *wl = arr[A_WL];
    double dt = g->dt;
    for (int k = 0; k < Nz; ++k)
        for (int j = 0; j < Ny; ++j)
            for (int i = 0; i < Nx; ++i) {
                double v = (double)velocity[((size_t)k * Ny + j) * Nx + i];
                m[ora_index(g, i, j, k)] = v * v * dt * dt;
            }
    ora_eta(g, eta);
    double inv_vol = 1.0 / (g->dx * g->dy * g->dz);
    long ps = src_ijk ? ora_index(g, src_ijk[0], src_ijk[1], src_ijk[2]) : -1;
    /* forward, keeping g^n = L u^n + phi^n + f^n */
    double *u_prev = ua, *u_cur = ub, *u_next = uc, *phi = pa, *phi_next = pb;
    for (int step = 0; step < nt; ++step) {
        ora_laplacian(g, u_cur, lap, nthreads);
        double *gn = gacc + (size_t)step * n;
        for (int k = 0; k < Nz; ++k)
            for (int j = 0; j < Ny; ++j)
                for (int i = 0; i < Nx; ++i) {
                    long p = ora_index(g, i, j, k);
                    gn[p] = lap[p] + (ora_is_pml(g, i, j, k) ? phi[p] : 0.0);
                }
        if (ps >= 0) gn[ps] += (double)wavelet[step] * inv_vol;
        ora_step(g, m, eta, u_prev, u_cur, phi, u_next, phi_next, nthreads);
        if (ps >= 0) u_next[ps] += m[ps] * (double)wavelet[step] * inv_vol;
        for (int r = 0; r < nrec; ++r)
            traces[(size_t)step * nrec + r] =
                u_next[ora_index(g, rec_ijk[3 * r], rec_ijk[3 * r + 1], rec_ijk[3 * r + 2])];
        double *t = u_prev;
        u_prev = u_cur;
        u_cur = u_next;
        u_next = t;
        t = phi;
        phi = phi_next;
        phi_next = t;
    }
    double J = 0.0;
    for (size_t q = 0; q < (size_t)nt * nrec; ++q) {
        double d = traces[q] - observed[q];
        J += 0.5 * d * d;
    }
    *misfit = J;
    /* backward */
    for (int kk = nt; kk >= 1; --kk) {
        /* psi from nu^{k+1}; nu^k */
        for (int k = 0; k < Nz; ++k)
            for (int j = 0; j < Ny; ++j)
                for (int i = 0; i < Nx; ++i) {
                    long p = ora_index(g, i, j, k);
                    int c[3] = {i, j, k};
                    double s = 0.0;
                    for (int ax = 0; ax < 3; ++ax)
                        for (int sg = -1; sg <= 1; sg += 2) {
                            int d[3] = {c[0], c[1], c[2]};
                            d[ax] += sg;
                            if (d[0] < 0 || d[0] >= Nx || d[1] < 0 || d[1] >= Ny || d[2] < 0 ||
                                d[2] >= Nz || !ora_is_pml(g, d[0], d[1], d[2]))
                                continue;
                            long q = p + sg * st3[ax];
                            double e = eta[q] * dt;
                            double ca = dt * (eta[q + st3[ax]] - eta[q - st3[ax]]) / (2.0 * hh[ax]) /
                                        (1.0 + e);
                            s += sg * ca * nu[q] / (2.0 * hh[ax]);
                        }
                    psi[p] = s;
                    if (ora_is_pml(g, i, j, k)) {
                        double e = eta[p] * dt;
                        nun[p] = nu[p] / (1.0 + e) + w1[p];
                    } else {
                        nun[p] = 0.0;
                    }
                }
        ora_laplacian(g, w1, wl, nthreads);
        for (int k = 0; k < Nz; ++k)
            for (int j = 0; j < Ny; ++j)
                for (int i = 0; i < Nx; ++i) {
                    long p = ora_index(g, i, j, k);
                    double a = wl[p] + psi[p];
                    if (!ora_is_pml(g, i, j, k)) {
                        wk[p] = 2.0 * w1[p] - w2[p] + m[p] * a;
                    } else {
                        double e = eta[p] * dt;
                        wk[p] = ((2.0 - e * e) * w1[p] - (1.0 - e) * w2[p] + m[p] * a) / (1.0 + e);
                    }
                }
        /* K^T r^{k-1}: the residual enters at the receivers, scaled by M = m there */
        for (int r = 0; r < nrec; ++r) {
            long p = ora_index(g, rec_ijk[3 * r], rec_ijk[3 * r + 1], rec_ijk[3 * r + 2]);
            double res = traces[(size_t)(kk - 1) * nrec + r] - observed[(size_t)(kk - 1) * nrec + r];
            wk[p] += m[p] * res;
        }
        const double *gk = gacc + (size_t)(kk - 1) * n;
        for (size_t q = 0; q < n; ++q)
            if (m[q] > 0.0) gm[q] += wk[q] * gk[q] / m[q];
        double *t = w2;
        w2 = w1;
        w1 = wk;
        wk = t;
        t = nu;
        nu = nun;
        nun = t;
    }
    for (int k = 0; k < Nz; ++k)
        for (int j = 0; j < Ny; ++j)
            for (int i = 0; i < Nx; ++i) {
                long p = ora_index(g, i, j, k);
                double v = (double)velocity[((size_t)k * Ny + j) * Nx + i];
                grad_v[((size_t)k * Ny + j) * Nx + i] = gm[p] * 2.0 * v * dt * dt;
            }
    for (int q = 0; q < A_COUNT; ++q) free(arr[q]);
    return 0;
}
