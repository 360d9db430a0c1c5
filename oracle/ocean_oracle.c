/*
 * ocean_oracle.c -- plain, slow FP64 CPU oracle of one baroclinic time step of the
 * hydrostatic free-surface ocean model (arXiv 2309.06662, Sec. "New numerical methods
 * for finite volume fluid dynamics on the sphere" and Sec. "Optimization of ocean free
 * surface dynamics").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load this file's library.  It shares no code, header or table
 * with the CUDA path: every index, metric and formula below is written out again from
 * the discrete equations.
 *
 * The paper names the ingredients but prints no formula, constant or stencil; every
 * reading taken here is stated in the comment of the function that uses it: full-cell
 * bathymetry (a cell is wet when its centre lies above the sea floor), product-form
 * spherical metrics, Coriolis 2 Omega sin(phi) at the row (u) and face (v) latitudes,
 * free-slip corner vorticity, WENO-Z weights with eps = 1e-30, zero advective flux at the
 * sea floor and the surface, the Pacanowski-Philander constants, chi = 0.1 with a
 * forward-Euler first step, and equal averaging weights over the sub-cycle (or the
 * power-law shape, see ora_filter_weights).  Summary of the step n -> n+1:
 *   1. buoyancy b = g[alpha(T-T0) - beta_s(S-S0)] (linear equation of state);
 *      hydrostatic pressure p, summed top -> bottom (the "hydrostatic pressure"
 *      intermediate of Sec. "Starting from scratch with Julia");
 *   2. w from continuity, summed bottom -> top, w = 0 at the sea floor;
 *   3. Richardson-number mixing (Pacanowski & Philander 1981 form) -> kappa, nu at
 *      w-faces (the "vertical diffusivity" intermediate; Sec. "How performance was
 *      measured" names the Ri-based closure);
 *   4. tendencies: flux-form tracer advection and vector-invariant momentum, both
 *      with WENO-Z reconstructions (Jiang & Shu 1996 stencils, Borges et al. 2008
 *      weights) that drop to third and first order next to land;
 *   5. quasi-second-order Adams-Bashforth predictor (the IMEX AB2 scheme);
 *   6. backward-Euler vertical diffusion, one tridiagonal (Thomas) solve per column;
 *   7. split-explicit barotropic sub-cycle: N_s forward-backward substeps of length
 *      2 dt/(N_s+1), averaged with equal weights 1/N_s;
 *   8. barotropic correction of u, v.
 * Plain loops, no blocking or fusion; OpenMP only splits independent rows.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads of the OpenMP row loops (the benchmark times the oracle on all host cores and
 * on one). */
void ora_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
int ora_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

typedef struct {
    /* grid */
    int kind, nx, ny, nz, px, py;
    double x0, x1, y0, y1;
    double *zf, *zc, *dz;
    /* parameters */
    double dt, chi, g, rho0, alpha, beta_s, T0, S0, f0, betap, omega, radius;
    double nu0, ri_a, nu_b, kappa_b, kappa_conv, weno_eps, min_depth;
    int ns, weno_linear, filter;
    int vweno;                       /* vertical WENO: 0 index-space, 1 from the level thicknesses */
    int mom_vadv;                    /* vertical momentum advection: 0 centred, 1 WENO flux form */
    double* fw;                      /* averaging weights a_m of the sub-cycle, m = 1..ns */
    /* column data */
    double *depth, *taux, *tauy;
    int *kb;                         /* lowest wet level, nz for land */
    /* prognostic state */
    double *u, *v, *T, *S, *eta;
    double *Gu0, *Gv0, *GT0, *GS0;   /* tendencies of the previous step */
    long nstep;
    /* work arrays (diagnostics of the current state) */
    double *b, *p, *w, *kap, *nu;
    double *Gu, *Gv, *GT, *GS;
    double *GU, *GV, *U, *V, *Hu, *Hv;
    /* learned closure: diffusivity on interior wet faces and tracer tendency corrections
     * supplied for the next steps (NULL = Richardson-number closure only) */
    double *ext_kap, *ext_dGT, *ext_dGS;
} ora_t;

#define PI 3.14159265358979323846

/* ------------------------------------------------------------------ grid metrics */

static double deg2rad(double d) { return d * (PI / 180.0); }

/* latitude (radians) of cell centres of row j, and of the south face of row j */
static double phi_c(const ora_t* m, int j) {
    return deg2rad(m->y0 + (j + 0.5) * ((m->y1 - m->y0) / m->ny));
}
static double phi_f(const ora_t* m, int j) {
    return deg2rad(m->y0 + j * ((m->y1 - m->y0) / m->ny));
}
/* zonal width of a cell (and of a u-face) in row j */
static double dx_c(const ora_t* m, int j) {
    if (m->kind == 0) return (m->x1 - m->x0) / m->nx;
    return m->radius * cos(phi_c(m, j)) * deg2rad((m->x1 - m->x0) / m->nx);
}
/* zonal width along the south face of row j (v-face, vorticity corner) */
static double dx_v(const ora_t* m, int j) {
    if (m->kind == 0) return (m->x1 - m->x0) / m->nx;
    return m->radius * cos(phi_f(m, j)) * deg2rad((m->x1 - m->x0) / m->nx);
}
static double dy_(const ora_t* m) {
    if (m->kind == 0) return (m->y1 - m->y0) / m->ny;
    return m->radius * deg2rad((m->y1 - m->y0) / m->ny);
}
static double area_c(const ora_t* m, int j) { return dx_c(m, j) * dy_(m); }
static double area_z(const ora_t* m, int j) { return dx_v(m, j) * dy_(m); }
/* Coriolis parameter at u-points (row centre latitude) and v-points (south face) */
static double f_u(const ora_t* m, int j) {
    if (m->kind == 0) {
        double y = m->y0 + (j + 0.5) * ((m->y1 - m->y0) / m->ny);
        return m->f0 + m->betap * (y - 0.5 * (m->y0 + m->y1));
    }
    return 2.0 * m->omega * sin(phi_c(m, j));
}
static double f_v(const ora_t* m, int j) {
    if (m->kind == 0) {
        double y = m->y0 + j * ((m->y1 - m->y0) / m->ny);
        return m->f0 + m->betap * (y - 0.5 * (m->y0 + m->y1));
    }
    return 2.0 * m->omega * sin(phi_f(m, j));
}
/* vertical spacing between the centres of cells k-1 and k (w-face k) */
static double dz_f(const ora_t* m, int k) { return m->zc[k] - m->zc[k - 1]; }

/* ------------------------------------------------------------------ indexing */

/* Wrap a column index; returns 0 when the column lies outside a walled domain. */
static int col(const ora_t* m, int i, int j, int* ic, int* jc) {
    if (m->px) { i %= m->nx; if (i < 0) i += m->nx; }
    else if (i < 0 || i >= m->nx) return 0;
    if (m->py) { j %= m->ny; if (j < 0) j += m->ny; }
    else if (j < 0 || j >= m->ny) return 0;
    *ic = i; *jc = j;
    return 1;
}
static long at3(const ora_t* m, int i, int j, int k) {
    return ((long)k * m->ny + j) * m->nx + i;
}
static int wet(const ora_t* m, int i, int j, int k) {
    int ic, jc;
    if (k < 0 || k >= m->nz) return 0;
    if (!col(m, i, j, &ic, &jc)) return 0;
    return k >= m->kb[jc * m->nx + ic];
}
static int kbot(const ora_t* m, int i, int j) {
    int ic, jc;
    if (!col(m, i, j, &ic, &jc)) return m->nz;
    return m->kb[jc * m->nx + ic];
}
/* u-face i sits between cells i-1 and i; v-face j between rows j-1 and j */
static int uwet(const ora_t* m, int i, int j, int k) { return wet(m, i - 1, j, k) && wet(m, i, j, k); }
static int vwet(const ora_t* m, int i, int j, int k) { return wet(m, i, j - 1, k) && wet(m, i, j, k); }

/* value of a cell-centred field (0 outside the domain) */
static double cval(const ora_t* m, const double* F, int i, int j, int k) {
    int ic, jc;
    if (k < 0 || k >= m->nz || !col(m, i, j, &ic, &jc)) return 0.0;
    return F[at3(m, ic, jc, k)];
}
/* value of a u-face field: 0 on dry faces and walls */
static double uval(const ora_t* m, const double* F, int i, int j, int k) {
    int ic, jc;
    if (!uwet(m, i, j, k)) return 0.0;
    col(m, i, j, &ic, &jc);
    return F[at3(m, ic, jc, k)];
}
static double vval(const ora_t* m, const double* F, int i, int j, int k) {
    int ic, jc;
    if (!vwet(m, i, j, k)) return 0.0;
    col(m, i, j, &ic, &jc);
    return F[at3(m, ic, jc, k)];
}
static double col2(const ora_t* m, const double* F, int i, int j) {
    int ic, jc;
    if (!col(m, i, j, &ic, &jc)) return 0.0;
    return F[jc * m->nx + ic];
}

/* ------------------------------------------------------------------ WENO */

/*
 * Fifth-order WENO-Z reconstruction at the face downstream of q[2] (q[0..4] ordered
 * from upwind to downwind).  Candidate polynomials and smoothness indicators of
 * Jiang & Shu (1996); weights alpha_r = d_r (1 + (tau5/(beta_r + eps))^2) with
 * tau5 = |beta_0 - beta_2| (Borges et al. 2008, exponent 2); ideal weights
 * d = (1/10, 6/10, 3/10).  linear != 0 uses the ideal weights (the linear
 * fifth-order upwind scheme).
 */
double ora_weno5(const double* q, double eps, int linear) {
    double p0 = (2.0 * q[0] - 7.0 * q[1] + 11.0 * q[2]) / 6.0;
    double p1 = (-q[1] + 5.0 * q[2] + 2.0 * q[3]) / 6.0;
    double p2 = (2.0 * q[2] + 5.0 * q[3] - q[4]) / 6.0;
    double d0 = 0.1, d1 = 0.6, d2 = 0.3;
    if (linear) return d0 * p0 + d1 * p1 + d2 * p2;
    double a = q[0] - 2.0 * q[1] + q[2], bb = q[0] - 4.0 * q[1] + 3.0 * q[2];
    double b0 = 13.0 / 12.0 * a * a + 0.25 * bb * bb;
    a = q[1] - 2.0 * q[2] + q[3]; bb = q[1] - q[3];
    double b1 = 13.0 / 12.0 * a * a + 0.25 * bb * bb;
    a = q[2] - 2.0 * q[3] + q[4]; bb = 3.0 * q[2] - 4.0 * q[3] + q[4];
    double b2 = 13.0 / 12.0 * a * a + 0.25 * bb * bb;
    double tau = fabs(b0 - b2);
    double r0 = tau / (b0 + eps), r1 = tau / (b1 + eps), r2 = tau / (b2 + eps);
    double a0 = d0 * (1.0 + r0 * r0), a1 = d1 * (1.0 + r1 * r1), a2 = d2 * (1.0 + r2 * r2);
    return (a0 * p0 + a1 * p1 + a2 * p2) / (a0 + a1 + a2);
}

/*
 * Third-order WENO-Z at the face downstream of q[1] (q[0..2] upwind to downwind):
 * candidates (-q0 + 3 q1)/2 and (q1 + q2)/2, indicators (q1-q0)^2 and (q2-q1)^2,
 * ideal weights (1/3, 2/3), tau3 = |beta_0 - beta_1|.
 */
double ora_weno3(const double* q, double eps, int linear) {
    double p0 = (-q[0] + 3.0 * q[1]) / 2.0;
    double p1 = (q[1] + q[2]) / 2.0;
    double d0 = 1.0 / 3.0, d1 = 2.0 / 3.0;
    if (linear) return d0 * p0 + d1 * p1;
    double b0 = (q[1] - q[0]) * (q[1] - q[0]);
    double b1 = (q[2] - q[1]) * (q[2] - q[1]);
    double tau = fabs(b0 - b1);
    double r0 = tau / (b0 + eps), r1 = tau / (b1 + eps);
    double a0 = d0 * (1.0 + r0 * r0), a1 = d1 * (1.0 + r1 * r1);
    return (a0 * p0 + a1 * p1) / (a0 + a1);
}

/*
 * Adaptive order next to land (the "adaptive-order" reading): the fifth-order
 * reconstruction when all five stencil points lie in the fluid, else the third-order
 * one when its three central points do, else the upwind value (first order).
 */
double ora_recon(const double* q, const int* in, double eps, int linear) {
    if (in[0] && in[1] && in[2] && in[3] && in[4]) return ora_weno5(q, eps, linear);
    if (in[1] && in[2] && in[3]) return ora_weno3(q + 1, eps, linear);
    return q[2];
}

/* ------------------------------------------------------------------ WENO on stretched levels */

/*
 * Reconstruction weights on a non-uniform stencil (the "stretched" reading of the
 * adaptive WENO of Sec. "New numerical methods for finite volume fluid dynamics on the
 * sphere").  The n cells of the stencil span the edges e[0..n], monotone in either
 * direction.  c[0..n-1] are the weights for which sum_j c_j qbar_j is the value at x = xf
 * of the polynomial of degree n-1 whose means over the n cells are qbar_j.  With
 * p(x) = sum_m a_m ((x - xf)/h)^m the cell means are M a with
 *   M[j][m] = mean over cell j of ((x - xf)/h)^m
 *           = (s_{j+1}^{m+1} - s_j^{m+1}) / ((m+1)(s_{j+1} - s_j)),  s = (e - xf)/h,
 * and the value at xf is a_0, the first entry of M^{-1} qbar; so c is the first row of
 * M^{-1}, the solution of M^T c = (1, 0, ..., 0).  Gaussian elimination with partial
 * pivoting; h is the mean cell width (the weights do not depend on it).
 */
static void recon_weights(int n, const double* e, double xf, double* c) {
    double A[5][6];
    double h = fabs(e[n] - e[0]) / n;
    for (int j = 0; j < n; j++) {
        double s0 = (e[j] - xf) / h, s1 = (e[j + 1] - xf) / h;
        double p0 = s0, p1 = s1;   /* s^{m+1} */
        for (int m = 0; m < n; m++) {
            A[m][j] = (p1 - p0) / ((m + 1) * (s1 - s0));   /* row m of M^T */
            p0 *= s0;
            p1 *= s1;
        }
    }
    for (int m = 0; m < n; m++) A[m][n] = (m == 0) ? 1.0 : 0.0;
    for (int col = 0; col < n; col++) {
        int piv = col;
        for (int r = col + 1; r < n; r++)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        for (int t = 0; t <= n; t++) { double x = A[col][t]; A[col][t] = A[piv][t]; A[piv][t] = x; }
        for (int r = col + 1; r < n; r++) {
            double f = A[r][col] / A[col][col];
            for (int t = col; t <= n; t++) A[r][t] -= f * A[col][t];
        }
    }
    for (int r = n - 1; r >= 0; r--) {
        double s = A[r][n];
        for (int t = r + 1; t < n; t++) s -= A[r][t] * c[t];
        c[r] = s / A[r][r];
    }
}

/*
 * Coefficients of the reconstruction at the face xf downstream of cell 2 of an ordered
 * five-cell stencil with edges e[0..5] (upwind to downwind): the three third-order
 * candidates on cells {0,1,2}, {1,2,3}, {2,3,4}; the ideal weights d_r for which
 * sum_r d_r (candidate r) is the fifth-order reconstruction on all five cells (d_0 and d_2
 * from its outermost weights, d_1 = 1 - d_0 - d_2); and the same for the third-order
 * scheme on cells 1..3 (candidates on {1,2} and {2,3}).  Only the parts whose edges lie
 * inside [0, nz] are computed: five = 0 skips the fifth-order part.
 */
typedef struct { double c[3][3], d[3], c3[2][2], d3[2]; } wcoef_t;

void ora_weno_coeffs(const double* e, double xf, int five, double* out /* 18 values */) {
    wcoef_t w;
    memset(&w, 0, sizeof(w));
    if (five) {
        double c5[5];
        for (int r = 0; r < 3; r++) recon_weights(3, e + r, xf, w.c[r]);
        recon_weights(5, e, xf, c5);
        w.d[0] = c5[0] / w.c[0][0];
        w.d[2] = c5[4] / w.c[2][2];
        w.d[1] = 1.0 - w.d[0] - w.d[2];
    }
    double c3[3];
    recon_weights(2, e + 1, xf, w.c3[0]);
    recon_weights(2, e + 2, xf, w.c3[1]);
    recon_weights(3, e + 1, xf, c3);
    w.d3[0] = c3[0] / w.c3[0][0];
    w.d3[1] = 1.0 - w.d3[0];
    memcpy(out, &w, sizeof(w));
}

/* WENO-Z of an ordered stencil with the coefficients of ora_weno_coeffs: candidates and
 * ideal weights from the level thicknesses, smoothness indicators and tau5 in index space
 * (the Jiang-Shu forms of ora_weno5).  The reading: the indicators only rank the
 * candidates, so they keep their uniform form while the candidates and weights carry the
 * grid. */
static double weno5_coef(const double* q, const wcoef_t* w, double eps, int linear) {
    double p[3];
    for (int r = 0; r < 3; r++) p[r] = w->c[r][0] * q[r] + w->c[r][1] * q[r + 1] + w->c[r][2] * q[r + 2];
    if (linear) return w->d[0] * p[0] + w->d[1] * p[1] + w->d[2] * p[2];
    double a = q[0] - 2.0 * q[1] + q[2], bb = q[0] - 4.0 * q[1] + 3.0 * q[2];
    double b0 = 13.0 / 12.0 * a * a + 0.25 * bb * bb;
    a = q[1] - 2.0 * q[2] + q[3]; bb = q[1] - q[3];
    double b1 = 13.0 / 12.0 * a * a + 0.25 * bb * bb;
    a = q[2] - 2.0 * q[3] + q[4]; bb = 3.0 * q[2] - 4.0 * q[3] + q[4];
    double b2 = 13.0 / 12.0 * a * a + 0.25 * bb * bb;
    double tau = fabs(b0 - b2);
    double r0 = tau / (b0 + eps), r1 = tau / (b1 + eps), r2 = tau / (b2 + eps);
    double a0 = w->d[0] * (1.0 + r0 * r0), a1 = w->d[1] * (1.0 + r1 * r1), a2 = w->d[2] * (1.0 + r2 * r2);
    return (a0 * p[0] + a1 * p[1] + a2 * p[2]) / (a0 + a1 + a2);
}
/* third order on q[1..3] with the stretched candidates and weights */
static double weno3_coef(const double* q, const wcoef_t* w, double eps, int linear) {
    double p0 = w->c3[0][0] * q[1] + w->c3[0][1] * q[2];
    double p1 = w->c3[1][0] * q[2] + w->c3[1][1] * q[3];
    if (linear) return w->d3[0] * p0 + w->d3[1] * p1;
    double b0 = (q[2] - q[1]) * (q[2] - q[1]);
    double b1 = (q[3] - q[2]) * (q[3] - q[2]);
    double tau = fabs(b0 - b1);
    double r0 = tau / (b0 + eps), r1 = tau / (b1 + eps);
    double a0 = w->d3[0] * (1.0 + r0 * r0), a1 = w->d3[1] * (1.0 + r1 * r1);
    return (a0 * p0 + a1 * p1) / (a0 + a1);
}

/* Adaptive order with stretched coefficients (same order selection as ora_recon). */
double ora_recon_coef(const double* q, const int* in, const double* e, double xf, double eps,
                      int linear) {
    double wc[18];
    if (in[0] && in[1] && in[2] && in[3] && in[4]) {
        ora_weno_coeffs(e, xf, 1, wc);
        return weno5_coef(q, (const wcoef_t*)wc, eps, linear);
    }
    if (in[1] && in[2] && in[3]) {
        ora_weno_coeffs(e, xf, 0, wc);
        return weno3_coef(q, (const wcoef_t*)wc, eps, linear);
    }
    return q[2];
}

/*
 * Reconstruction at the level face zf[kf] (bottom face of level kf) of one column of a
 * field, F[base + k s] for k in [k0, nz) (levels outside that range are not in the
 * fluid), upwind by the sign of the face velocity wt (wt >= 0 takes the levels below).
 * vweno = 0: index-space coefficients (ora_recon); 1: coefficients of the level
 * thicknesses (ora_recon_coef).
 */
static double recon_vertical(const ora_t* m, const double* F, long base, long s, int kf, int k0,
                             double wt) {
    double q[5], e[6];
    int in[5];
    int pos = wt >= 0.0;
    for (int n = 0; n < 5; n++) {
        int kk = pos ? kf - 3 + n : kf + 2 - n;
        in[n] = kk >= k0 && kk < m->nz;
        q[n] = in[n] ? F[base + (long)kk * s] : 0.0;
    }
    if (!m->vweno) return ora_recon(q, in, m->weno_eps, m->weno_linear);
    for (int n = 0; n < 6; n++) {
        int ke = pos ? kf - 3 + n : kf + 3 - n;   /* edge n of the ordered stencil */
        e[n] = (ke >= 0 && ke <= m->nz) ? m->zf[ke] : 0.0;   /* unused when outside */
    }
    return ora_recon_coef(q, in, e, m->zf[kf], m->weno_eps, m->weno_linear);
}

/* ------------------------------------------------------------------ diagnostics */

static double buoy(const ora_t* m, double T, double S) {
    return m->g * (m->alpha * (T - m->T0) - m->beta_s * (S - m->S0));
}

/* buoyancy, hydrostatic pressure, vertical velocity, diffusivities of the state */
static void diagnose(ora_t* m) {
    int nx = m->nx, ny = m->ny, nz = m->nz;
    long n3 = (long)nx * ny * nz;
    memset(m->b, 0, n3 * sizeof(double));
    memset(m->p, 0, n3 * sizeof(double));
    memset(m->w, 0, n3 * sizeof(double));
    memset(m->kap, 0, n3 * sizeof(double));
    memset(m->nu, 0, n3 * sizeof(double));
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; j++) {
        double dy = dy_(m), ac = area_c(m, j);
        for (int i = 0; i < nx; i++) {
            int kb = m->kb[j * nx + i];
            if (kb >= nz) continue;
            for (int k = kb; k < nz; k++) {
                long c = at3(m, i, j, k);
                m->b[c] = buoy(m, m->T[c], m->S[c]);
            }
            /* pressure: top cell centre sits half a layer below the surface */
            m->p[at3(m, i, j, nz - 1)] = -m->b[at3(m, i, j, nz - 1)] * (m->zf[nz] - m->zc[nz - 1]);
            for (int k = nz - 2; k >= kb; k--)
                m->p[at3(m, i, j, k)] = m->p[at3(m, i, j, k + 1)]
                    - 0.5 * (m->b[at3(m, i, j, k)] + m->b[at3(m, i, j, k + 1)]) * dz_f(m, k + 1);
            /* w at the bottom face of each cell, integrated upward from the sea floor */
            m->w[at3(m, i, j, kb)] = 0.0;
            for (int k = kb; k < nz - 1; k++) {
                double div = dy * m->dz[k] * (uval(m, m->u, i + 1, j, k) - uval(m, m->u, i, j, k))
                           + m->dz[k] * (dx_v(m, j + 1) * vval(m, m->v, i, j + 1, k)
                                         - dx_v(m, j) * vval(m, m->v, i, j, k));
                m->w[at3(m, i, j, k + 1)] = m->w[at3(m, i, j, k)] - div / ac;
            }
            /* Richardson-number closure on the interior w-faces of the column */
            for (int k = kb + 1; k < nz; k++) {
                double dzf = dz_f(m, k);
                double n2 = (m->b[at3(m, i, j, k)] - m->b[at3(m, i, j, k - 1)]) / dzf;
                double ua = 0.5 * (uval(m, m->u, i, j, k) + uval(m, m->u, i + 1, j, k));
                double ub = 0.5 * (uval(m, m->u, i, j, k - 1) + uval(m, m->u, i + 1, j, k - 1));
                double va = 0.5 * (vval(m, m->v, i, j, k) + vval(m, m->v, i, j + 1, k));
                double vb = 0.5 * (vval(m, m->v, i, j, k - 1) + vval(m, m->v, i, j + 1, k - 1));
                double s2 = ((ua - ub) * (ua - ub) + (va - vb) * (va - vb)) / (dzf * dzf);
                double kap, nu;
                if (n2 < 0.0) {
                    kap = m->kappa_conv; nu = m->kappa_conv;
                } else {
                    double ri = n2 / (s2 > 1e-14 ? s2 : 1e-14);
                    double q = 1.0 + m->ri_a * ri;
                    nu = m->nu0 / (q * q) + m->nu_b;
                    kap = nu / q + m->kappa_b;
                }
                m->kap[at3(m, i, j, k)] = kap;
                m->nu[at3(m, i, j, k)] = nu;
            }
            /* a learned diffusivity replaces kappa on the interior wet faces */
            if (m->ext_kap)
                for (int k = kb + 1; k < nz; k++) m->kap[at3(m, i, j, k)] = m->ext_kap[at3(m, i, j, k)];
        }
    }
}

/* ------------------------------------------------------------------ tracer tendency */

/* advective flux of tracer C through u-face i of cell row j, level k */
static double flux_x(const ora_t* m, const double* C, int i, int j, int k) {
    if (!uwet(m, i, j, k)) return 0.0;
    double ut = uval(m, m->u, i, j, k);
    double q[5]; int in[5];
    for (int n = 0; n < 5; n++) {
        int ii = ut >= 0.0 ? i - 3 + n : i + 2 - n;
        q[n] = cval(m, C, ii, j, k);
        in[n] = wet(m, ii, j, k);
    }
    return ut * dy_(m) * m->dz[k] * ora_recon(q, in, m->weno_eps, m->weno_linear);
}
static double flux_y(const ora_t* m, const double* C, int i, int j, int k) {
    if (!vwet(m, i, j, k)) return 0.0;
    double vt = vval(m, m->v, i, j, k);
    double q[5]; int in[5];
    for (int n = 0; n < 5; n++) {
        int jj = vt >= 0.0 ? j - 3 + n : j + 2 - n;
        q[n] = cval(m, C, i, jj, k);
        in[n] = wet(m, i, jj, k);
    }
    return vt * dx_v(m, j) * m->dz[k] * ora_recon(q, in, m->weno_eps, m->weno_linear);
}
/* flux through the bottom face of cell k: zero at the sea floor and at the surface */
static double flux_z(const ora_t* m, const double* C, int i, int j, int k) {
    int kb = kbot(m, i, j);
    if (k >= m->nz || k <= kb) return 0.0;
    double wt = cval(m, m->w, i, j, k);
    long s = (long)m->nx * m->ny;
    return wt * area_c(m, j) * recon_vertical(m, C, at3(m, i, j, 0), s, k, kb, wt);
}

static void tracer_tendency(ora_t* m, const double* C, double* G) {
    int nx = m->nx, ny = m->ny, nz = m->nz;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; j++)
        for (int k = 0; k < nz; k++)
            for (int i = 0; i < nx; i++) {
                long c = at3(m, i, j, k);
                if (!wet(m, i, j, k)) { G[c] = 0.0; continue; }
                double div = flux_x(m, C, i + 1, j, k) - flux_x(m, C, i, j, k)
                           + flux_y(m, C, i, j + 1, k) - flux_y(m, C, i, j, k)
                           + flux_z(m, C, i, j, k + 1) - flux_z(m, C, i, j, k);
                G[c] = -div / (area_c(m, j) * m->dz[k]);
            }
}

/* ------------------------------------------------------------------ momentum tendency */

/* relative vorticity at corner (i, j) (south-west corner of cell (i, j)); zero unless
 * all four surrounding cells are wet (free slip at the coast) */
static double zeta(const ora_t* m, int i, int j, int k) {
    if (!(wet(m, i - 1, j - 1, k) && wet(m, i, j - 1, k) && wet(m, i - 1, j, k) && wet(m, i, j, k)))
        return 0.0;
    double circ = dy_(m) * (vval(m, m->v, i, j, k) - vval(m, m->v, i - 1, j, k))
                - (dx_c(m, j) * uval(m, m->u, i, j, k) - dx_c(m, j - 1) * uval(m, m->u, i, j - 1, k));
    return circ / area_z(m, j);
}
static int corner_in(const ora_t* m, int i, int j, int k) {
    return wet(m, i - 1, j - 1, k) || wet(m, i, j - 1, k) || wet(m, i - 1, j, k) || wet(m, i, j, k);
}
/* kinetic energy at the centre of cell (i, j, k) */
static double kin(const ora_t* m, int i, int j, int k) {
    double ua = uval(m, m->u, i, j, k), ub = uval(m, m->u, i + 1, j, k);
    double va = vval(m, m->v, i, j, k), vb = vval(m, m->v, i, j + 1, k);
    return 0.25 * (ua * ua + ub * ub) + 0.25 * (va * va + vb * vb);
}

/*
 * Vertical advection term of the vector-invariant momentum equation, w du/dz, at level k
 * of a velocity column F[base + k s] whose wet levels are [k0, nz), with the column's
 * face velocities wbot (bottom face of level k) and wtop (top face).
 * mom_vadv = 0, centred:  1/2 [wtop (F_{k+1} - F_k)/dzf_{k+1} + wbot (F_k - F_{k-1})/dzf_k].
 * mom_vadv = 1, WENO flux form (the vertical part of the WENO vector-invariant scheme):
 *   [wtop F~_{k+1/2} - wbot F~_{k-1/2} - F_k (wtop - wbot)] / dz_k,
 * F~ the upwind reconstruction at the face (recon_vertical, same order reduction and
 * coefficients as the tracers).  Faces at the top of the column and below its lowest wet
 * level carry no flux (wtop, wbot = 0 there).  Both forms equal w dF/dz for a linear
 * profile and constant w on uniform levels; the flux form vanishes for a uniform
 * profile whatever w does.
 */
static double vertical_advection(const ora_t* m, const double* F, long base, long s, int k, int k0,
                                 double wbot, double wtop) {
    int nz = m->nz;
    double fk = F[base + (long)k * s];
    if (k + 1 >= nz) wtop = 0.0;
    if (k <= k0) wbot = 0.0;
    if (!m->mom_vadv) {
        double up = 0.0, dn = 0.0;
        if (k + 1 < nz) up = wtop * (F[base + (long)(k + 1) * s] - fk) / dz_f(m, k + 1);
        if (k > k0) dn = wbot * (fk - F[base + (long)(k - 1) * s]) / dz_f(m, k);
        return 0.5 * (up + dn);
    }
    double ft = (k + 1 < nz) ? wtop * recon_vertical(m, F, base, s, k + 1, k0, wtop) : 0.0;
    double fb = (k > k0) ? wbot * recon_vertical(m, F, base, s, k, k0, wbot) : 0.0;
    return (ft - fb - fk * (wtop - wbot)) / m->dz[k];
}

/*
 * The vertical advection term of one velocity column alone (the tests' handle on
 * vertical_advection): levels zf[0..nz] bottom to top, F[0..nz-1], wet levels [k0, nz),
 * wf[k] the velocity on the bottom face of level k (wf[nz] on the surface), scheme
 * switches as in ora_create; out[k] for k in [k0, nz).
 */
void ora_vertical_advection_column(int nz, const double* zf, const double* F, int k0,
                                   const double* wf, int vweno, int mom_vadv, double eps,
                                   double* out) {
    ora_t m;
    memset(&m, 0, sizeof(m));
    m.nz = nz;
    m.zf = (double*)zf;
    m.zc = malloc(nz * sizeof(double));
    m.dz = malloc(nz * sizeof(double));
    for (int k = 0; k < nz; k++) {
        m.zc[k] = 0.5 * (zf[k] + zf[k + 1]);
        m.dz[k] = zf[k + 1] - zf[k];
    }
    m.vweno = vweno;
    m.mom_vadv = mom_vadv;
    m.weno_eps = eps;
    for (int k = k0; k < nz; k++)
        out[k] = vertical_advection(&m, F, 0, 1, k, k0, wf[k], wf[k + 1]);
    free(m.zc);
    free(m.dz);
}

static void momentum_tendency(ora_t* m) {
    int nx = m->nx, ny = m->ny, nz = m->nz;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; j++)
        for (int k = 0; k < nz; k++)
            for (int i = 0; i < nx; i++) {
                long c = at3(m, i, j, k);
                double q[5]; int in[5];
                /* ---- u at the west face of cell (i, j) */
                m->Gu[c] = 0.0;
                if (uwet(m, i, j, k)) {
                    double vh = 0.25 * (vval(m, m->v, i - 1, j, k) + vval(m, m->v, i, j, k)
                                      + vval(m, m->v, i - 1, j + 1, k) + vval(m, m->v, i, j + 1, k));
                    for (int n = 0; n < 5; n++) {
                        int jj = vh >= 0.0 ? j - 2 + n : j + 3 - n;
                        q[n] = zeta(m, i, jj, k);
                        in[n] = corner_in(m, i, jj, k);
                    }
                    double zt = ora_recon(q, in, m->weno_eps, m->weno_linear);
                    double dxc = dx_c(m, j);
                    double dK = (kin(m, i, j, k) - kin(m, i - 1, j, k)) / dxc;
                    double dP = (cval(m, m->p, i, j, k) - cval(m, m->p, i - 1, j, k)) / dxc;
                    int k0 = kbot(m, i - 1, j) > kbot(m, i, j) ? kbot(m, i - 1, j) : kbot(m, i, j);
                    double wt = k + 1 < nz ? 0.5 * (cval(m, m->w, i - 1, j, k + 1) + cval(m, m->w, i, j, k + 1)) : 0.0;
                    double wb = 0.5 * (cval(m, m->w, i - 1, j, k) + cval(m, m->w, i, j, k));
                    double va = vertical_advection(m, m->u, at3(m, i, j, 0), (long)nx * ny, k, k0, wb, wt);
                    double wind = (k == nz - 1) ? m->taux[j * nx + i] / (m->rho0 * m->dz[nz - 1]) : 0.0;
                    m->Gu[c] = (zt + f_u(m, j)) * vh - dK - va - dP + wind;
                }
                /* ---- v at the south face of cell (i, j) */
                m->Gv[c] = 0.0;
                if (vwet(m, i, j, k)) {
                    double uh = 0.25 * (uval(m, m->u, i, j - 1, k) + uval(m, m->u, i + 1, j - 1, k)
                                      + uval(m, m->u, i, j, k) + uval(m, m->u, i + 1, j, k));
                    for (int n = 0; n < 5; n++) {
                        int ii = uh >= 0.0 ? i - 2 + n : i + 3 - n;
                        q[n] = zeta(m, ii, j, k);
                        in[n] = corner_in(m, ii, j, k);
                    }
                    double zt = ora_recon(q, in, m->weno_eps, m->weno_linear);
                    double dy = dy_(m);
                    double dK = (kin(m, i, j, k) - kin(m, i, j - 1, k)) / dy;
                    double dP = (cval(m, m->p, i, j, k) - cval(m, m->p, i, j - 1, k)) / dy;
                    int k0 = kbot(m, i, j - 1) > kbot(m, i, j) ? kbot(m, i, j - 1) : kbot(m, i, j);
                    double wt = k + 1 < nz ? 0.5 * (cval(m, m->w, i, j - 1, k + 1) + cval(m, m->w, i, j, k + 1)) : 0.0;
                    double wb = 0.5 * (cval(m, m->w, i, j - 1, k) + cval(m, m->w, i, j, k));
                    double va = vertical_advection(m, m->v, at3(m, i, j, 0), (long)nx * ny, k, k0, wb, wt);
                    double wind = (k == nz - 1) ? m->tauy[j * nx + i] / (m->rho0 * m->dz[nz - 1]) : 0.0;
                    m->Gv[c] = -(zt + f_v(m, j)) * uh - dK - va - dP + wind;
                }
            }
}

/* all tendencies of the current state (diagnostics first) */
void ora_tendencies(ora_t* m) {
    diagnose(m);
    tracer_tendency(m, m->T, m->GT);
    tracer_tendency(m, m->S, m->GS);
    if (m->ext_dGT) {   /* learned tracer tendency corrections on wet cells */
        long n3 = (long)m->nx * m->ny * m->nz;
        for (long c = 0; c < n3; c++) {
            m->GT[c] += m->ext_dGT[c];
            m->GS[c] += m->ext_dGS[c];
        }
    }
    momentum_tendency(m);
}

/* Supply (or, with NULL, remove) the learned closure's fields for the following steps:
 * kappa on bottom faces and dG_T, dG_S on cells, [nz][ny][nx]; copied.  Values outside
 * interior wet faces (kappa) or wet cells (dG) are ignored. */
void ora_set_closure_fields(ora_t* m, const double* kap, const double* dgt, const double* dgs) {
    long n3 = (long)m->nx * m->ny * m->nz;
    free(m->ext_kap); free(m->ext_dGT); free(m->ext_dGS);
    m->ext_kap = m->ext_dGT = m->ext_dGS = 0;
    if (!kap) return;
    m->ext_kap = malloc(n3 * sizeof(double));
    m->ext_dGT = malloc(n3 * sizeof(double));
    m->ext_dGS = malloc(n3 * sizeof(double));
    memcpy(m->ext_kap, kap, n3 * sizeof(double));
    for (long c = 0; c < n3; c++) {
        int k = (int)(c / ((long)m->nx * m->ny));
        long c2 = c % ((long)m->nx * m->ny);
        int w = k >= m->kb[c2];
        m->ext_dGT[c] = w ? dgt[c] : 0.0;
        m->ext_dGS[c] = w ? dgs[c] : 0.0;
    }
}

/* ------------------------------------------------------------------ implicit solve */

/*
 * Thomas algorithm for a[k] x[k-1] + b[k] x[k] + c[k] x[k+1] = d[k], k = 0..n-1
 * (a[0] and c[n-1] unused), without pivoting.  Forward elimination from k = 0,
 * back substitution from k = n-1.
 */
void ora_thomas(int n, const double* a, const double* b, const double* c, const double* d,
                double* x) {
    double cp[512], dp[512];
    if (n <= 0) return;
    cp[0] = c[0] / b[0];
    dp[0] = d[0] / b[0];
    for (int k = 1; k < n; k++) {
        double den = b[k] - a[k] * cp[k - 1];
        cp[k] = c[k] / den;
        dp[k] = (d[k] - a[k] * dp[k - 1]) / den;
    }
    x[n - 1] = dp[n - 1];
    for (int k = n - 2; k >= 0; k--) x[k] = dp[k] - cp[k] * x[k + 1];
}

/*
 * Backward-Euler vertical diffusion of one column slice phi[k0..nz-1] (stride s in the
 * 3-D array), diffusivity K[k] on the bottom face of level k, zero flux through the
 * bottom of level k0 and the top of level nz-1:
 *   phi_k - phi*_k = dt/dz_k [K_{k+1}(phi_{k+1}-phi_k)/dzf_{k+1} - K_k(phi_k-phi_{k-1})/dzf_k].
 */
static void diffuse_column(const ora_t* m, double* phi, long base, long s, int k0, const double* K) {
    int n = m->nz - k0;
    double a[512], bd[512], c[512], d[512], x[512];
    if (n <= 0) return;
    for (int r = 0; r < n; r++) {
        int k = k0 + r;
        double lo = (k > k0) ? m->dt * K[k] / (m->dz[k] * dz_f(m, k)) : 0.0;
        double hi = (k < m->nz - 1) ? m->dt * K[k + 1] / (m->dz[k] * dz_f(m, k + 1)) : 0.0;
        a[r] = -lo; c[r] = -hi; bd[r] = 1.0 + lo + hi;
        d[r] = phi[base + (long)k * s];
    }
    ora_thomas(n, a, bd, c, d, x);
    for (int r = 0; r < n; r++) phi[base + (long)(k0 + r) * s] = x[r];
}

static void implicit_solves(ora_t* m) {
    int nx = m->nx, ny = m->ny, nz = m->nz;
    long s = (long)nx * ny;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; j++) {
        double K[512];
        for (int i = 0; i < nx; i++) {
            long base = (long)j * nx + i;
            int kb = m->kb[base];
            if (kb < nz) {
                for (int k = 0; k < nz; k++) K[k] = m->kap[base + k * s];
                diffuse_column(m, m->T, base, s, kb, K);
                diffuse_column(m, m->S, base, s, kb, K);
            }
            /* u-column at face i: both neighbouring columns wet from max(kb) upward */
            int kbu = kbot(m, i - 1, j) > kb ? kbot(m, i - 1, j) : kb;
            if (!m->px && i == 0) kbu = nz;
            if (kbu < nz) {
                for (int k = 0; k < nz; k++)
                    K[k] = 0.5 * (cval(m, m->nu, i - 1, j, k) + m->nu[base + k * s]);
                diffuse_column(m, m->u, base, s, kbu, K);
            }
            int kbv = kbot(m, i, j - 1) > kb ? kbot(m, i, j - 1) : kb;
            if (!m->py && j == 0) kbv = nz;
            if (kbv < nz) {
                for (int k = 0; k < nz; k++)
                    K[k] = 0.5 * (cval(m, m->nu, i, j - 1, k) + m->nu[base + k * s]);
                diffuse_column(m, m->v, base, s, kbv, K);
            }
        }
    }
}

/* ------------------------------------------------------------------ averaging filter */

/*
 * Weights a_1..a_ns of the time average that closes the barotropic sub-cycle.
 *
 * filter 0: equal weights a_m = 1/ns (a boxcar over the ns substeps).
 * filter 1: the power-law shape of Shchepetkin & McWilliams (2005, Ocean Modelling 9),
 *   s(x) = x^p (1 - x^q) - r x with p = 2, q = 4, r = 0.284.  The shape is negative near
 *   x = 0, positive over its main lobe and returns to zero at x*, the root of
 *   x - x^5 = r above the maximum of x - x^5 (x = 5^(-1/4)).  It is sampled at the ns
 *   interior points x_m = m x* / (ns + 1) and normalised so that the weights sum to one.
 * Either way the substep length follows from the first moment: dtau = dt / sum_m m a_m,
 * which puts the centroid of the average exactly at t + dt (for the boxcar this is
 * dtau = 2 dt / (ns + 1)).  Returns sum_m m a_m.
 */
double ora_filter_weights(int ns, int filter, double* a) {
    if (filter == 0) {
        for (int m = 0; m < ns; m++) a[m] = 1.0 / ns;
    } else {
        const double r = 0.284;
        double lo = pow(5.0, -0.25), hi = 1.0;   /* x - x^5 - r: > 0 at lo, < 0 at hi */
        for (int it = 0; it < 200; it++) {
            double mid = 0.5 * (lo + hi);
            if (mid - pow(mid, 5.0) - r > 0.0) lo = mid; else hi = mid;
        }
        double xs = 0.5 * (lo + hi), sum = 0.0;
        for (int m = 1; m <= ns; m++) {
            double x = m * xs / (ns + 1.0);
            a[m - 1] = x * x * (1.0 - pow(x, 4.0)) - r * x;
            sum += a[m - 1];
        }
        for (int m = 0; m < ns; m++) a[m] /= sum;
    }
    double mom = 0.0;
    for (int m = 1; m <= ns; m++) mom += m * a[m - 1];
    return mom;
}

/* ------------------------------------------------------------------ barotropic mode */

/*
 * Split-explicit sub-cycle.  From eta^0 = eta (in place), U^0, V^0 (transports, m^2/s)
 * and the slow forcing GU, GV, take N_s forward-backward substeps of length
 * dtau = dt / sum_m m a_m (2 dt/(N_s + 1) for equal weights):
 *   eta^m = eta^{m-1} - dtau/A_c [dy (U_{i+1} - U_i) + dxv_{j+1} V_{j+1} - dxv_j V_j]^{m-1}
 *   U^m   = U^{m-1} + dtau [-g H_u (eta^m_i - eta^m_{i-1})/dx_c + GU]
 *   V^m   = V^{m-1} + dtau [-g H_v (eta^m_j - eta^m_{j-1})/dy + GV]
 * and return the averages sum_m a_m (eta, U, V)^m over m = 1..N_s with the filter's
 * weights (ora_filter_weights; their first moment sum_m a_m m dtau is exactly dt) in
 * eta, Ubar, Vbar.
 */
void ora_barotropic(ora_t* m, double* eta, const double* U0, const double* V0, const double* GU,
                    const double* GV, double* Ubar, double* Vbar) {
    int nx = m->nx, ny = m->ny, ns = m->ns;
    long n2 = (long)nx * ny;
    double dtau = m->filter == 0 ? 2.0 * m->dt / (ns + 1.0) : m->dt / ora_filter_weights(ns, m->filter, m->fw);
    double *U = malloc(n2 * sizeof(double)), *V = malloc(n2 * sizeof(double));
    double *E = malloc(n2 * sizeof(double)), *Ea = calloc(n2, sizeof(double));
    double dy = dy_(m);
    memcpy(U, U0, n2 * sizeof(double));
    memcpy(V, V0, n2 * sizeof(double));
    memcpy(E, eta, n2 * sizeof(double));
    for (long c = 0; c < n2; c++) { Ubar[c] = 0.0; Vbar[c] = 0.0; }
    for (int step = 1; step <= ns; step++) {
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                long c = (long)j * nx + i;
                if (m->kb[c] >= m->nz) { E[c] = 0.0; continue; }
                double div = dy * (col2(m, U, i + 1, j) - U[c])
                           + dx_v(m, j + 1) * col2(m, V, i, j + 1) - dx_v(m, j) * V[c];
                E[c] = E[c] - dtau / area_c(m, j) * div;
            }
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                long c = (long)j * nx + i;
                if (m->Hu[c] > 0.0)
                    U[c] = U[c] + dtau * (-m->g * m->Hu[c] * (E[c] - col2(m, E, i - 1, j)) / dx_c(m, j) + GU[c]);
                else U[c] = 0.0;
                if (m->Hv[c] > 0.0)
                    V[c] = V[c] + dtau * (-m->g * m->Hv[c] * (E[c] - col2(m, E, i, j - 1)) / dy + GV[c]);
                else V[c] = 0.0;
            }
        for (long c = 0; c < n2; c++) {
            if (m->filter == 0) {
                Ea[c] += E[c] / ns;
                Ubar[c] += U[c] / ns;
                Vbar[c] += V[c] / ns;
            } else {
                double a = m->fw[step - 1];
                Ea[c] += a * E[c];
                Ubar[c] += a * U[c];
                Vbar[c] += a * V[c];
            }
        }
    }
    memcpy(eta, Ea, n2 * sizeof(double));
    free(U); free(V); free(E); free(Ea);
}

/* ------------------------------------------------------------------ the step */

static void column_sums(const ora_t* m, const double* F, int which, double* out) {
    /* sum over wet levels of dz_k F_k on u-faces (which = 0) or v-faces (which = 1) */
    int nx = m->nx, ny = m->ny, nz = m->nz;
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            double s = 0.0;
            for (int k = 0; k < nz; k++) {
                int ok = which == 0 ? uwet(m, i, j, k) : vwet(m, i, j, k);
                if (ok) s += m->dz[k] * F[at3(m, i, j, k)];
            }
            out[(long)j * nx + i] = s;
        }
}

void ora_step(ora_t* m, int nsteps) {
    int nx = m->nx, ny = m->ny, nz = m->nz;
    long n3 = (long)nx * ny * nz, n2 = (long)nx * ny;
    for (int it = 0; it < nsteps; it++) {
        ora_tendencies(m);
        if (m->nstep == 0) {   /* first step: forward Euler (G^{n-1} := G^n) */
            memcpy(m->Gu0, m->Gu, n3 * sizeof(double));
            memcpy(m->Gv0, m->Gv, n3 * sizeof(double));
            memcpy(m->GT0, m->GT, n3 * sizeof(double));
            memcpy(m->GS0, m->GS, n3 * sizeof(double));
        }
        double ca = 1.5 + m->chi, cb = 0.5 + m->chi;
        /* barotropic transports of the state at time n */
        column_sums(m, m->u, 0, m->U);
        column_sums(m, m->v, 1, m->V);
        /* quasi-AB2 predictor; the combined momentum tendencies are kept in Gu0/Gv0
         * only until the slow forcing is formed, then replaced by G^n */
        for (long c = 0; c < n3; c++) {
            double gu = ca * m->Gu[c] - cb * m->Gu0[c];
            double gv = ca * m->Gv[c] - cb * m->Gv0[c];
            double gt = ca * m->GT[c] - cb * m->GT0[c];
            double gs = ca * m->GS[c] - cb * m->GS0[c];
            m->u[c] += m->dt * gu;
            m->v[c] += m->dt * gv;
            m->T[c] += m->dt * gt;
            m->S[c] += m->dt * gs;
            m->Gu0[c] = gu;
            m->Gv0[c] = gv;
        }
        column_sums(m, m->Gu0, 0, m->GU);
        column_sums(m, m->Gv0, 1, m->GV);
        memcpy(m->Gu0, m->Gu, n3 * sizeof(double));
        memcpy(m->Gv0, m->Gv, n3 * sizeof(double));
        memcpy(m->GT0, m->GT, n3 * sizeof(double));
        memcpy(m->GS0, m->GS, n3 * sizeof(double));
        /* backward-Euler vertical diffusion */
        implicit_solves(m);
        /* barotropic sub-cycle from (eta^n, U^n, V^n) */
        double *Ub = malloc(n2 * sizeof(double)), *Vb = malloc(n2 * sizeof(double));
        ora_barotropic(m, m->eta, m->U, m->V, m->GU, m->GV, Ub, Vb);
        /* correction: depth-integrated u, v take the averaged transports */
        double *su = malloc(n2 * sizeof(double)), *sv = malloc(n2 * sizeof(double));
        column_sums(m, m->u, 0, su);
        column_sums(m, m->v, 1, sv);
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                long c2 = (long)j * nx + i;
                for (int k = 0; k < nz; k++) {
                    long c = at3(m, i, j, k);
                    if (uwet(m, i, j, k)) m->u[c] += (Ub[c2] - su[c2]) / m->Hu[c2];
                    else m->u[c] = 0.0;
                    if (vwet(m, i, j, k)) m->v[c] += (Vb[c2] - sv[c2]) / m->Hv[c2];
                    else m->v[c] = 0.0;
                }
            }
        free(Ub); free(Vb); free(su); free(sv);
        m->nstep++;
    }
}

/* ------------------------------------------------------------------ reductions */

/* Neumaier-compensated running sum */
typedef struct { double s, c; } csum_t;
static void cadd(csum_t* a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}

/*
 * out[0] = sum T V over wet cells, out[1] = sum S V, out[2] = sum eta A over wet
 * columns (compensated), out[3] = kinetic energy 1/2 sum u^2 V_u + 1/2 sum v^2 V_v,
 * out[4] = max advective CFL number (w of the current state), out[5] = 1 if any state
 * value is not finite,
 * out[6] = wet volume, out[7] = step counter.
 */
void ora_diagnostics(ora_t* m, double* out) {
    int nx = m->nx, ny = m->ny, nz = m->nz;
    diagnose(m);   /* w of the state being reported, for the vertical CFL number */
    csum_t st = {0, 0}, ss = {0, 0}, se = {0, 0}, ke = {0, 0}, vol = {0, 0};
    double cfl = 0.0;
    int bad = 0;
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                long c = at3(m, i, j, k);
                double vc = area_c(m, j) * m->dz[k];
                if (wet(m, i, j, k)) {
                    cadd(&st, m->T[c] * vc);
                    cadd(&ss, m->S[c] * vc);
                    cadd(&vol, vc);
                    double wc = fabs(m->w[c]) * m->dt / m->dz[k];
                    if (wc > cfl) cfl = wc;
                }
                if (uwet(m, i, j, k)) {
                    cadd(&ke, 0.5 * m->u[c] * m->u[c] * vc);
                    double uc = fabs(m->u[c]) * m->dt / dx_c(m, j);
                    if (uc > cfl) cfl = uc;
                }
                if (vwet(m, i, j, k)) {
                    cadd(&ke, 0.5 * m->v[c] * m->v[c] * dx_v(m, j) * dy_(m) * m->dz[k]);
                    double vcf = fabs(m->v[c]) * m->dt / dy_(m);
                    if (vcf > cfl) cfl = vcf;
                }
                if (!isfinite(m->u[c]) || !isfinite(m->v[c]) || !isfinite(m->T[c]) || !isfinite(m->S[c]))
                    bad = 1;
            }
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            long c = (long)j * nx + i;
            if (m->kb[c] < nz) cadd(&se, m->eta[c] * area_c(m, j));
            if (!isfinite(m->eta[c])) bad = 1;
        }
    out[0] = st.s + st.c; out[1] = ss.s + ss.c; out[2] = se.s + se.c;
    out[3] = ke.s + ke.c; out[4] = cfl; out[5] = bad; out[6] = vol.s + vol.c;
    out[7] = (double)m->nstep;
}

/* ------------------------------------------------------------------ create / fields */

/*
 * igrid = {kind, nx, ny, nz, periodic_x, periodic_y}; dgrid = {x0, x1, y0, y1};
 * zf[nz+1] bottom to top; depth, taux, tauy [ny][nx];
 * prm = {dt, chi, g, rho0, alpha, beta_s, T0, S0, f0, beta_plane, omega, radius,
 *        nu0, ri_a, nu_b, kappa_b, kappa_conv, weno_eps, min_depth};
 * iprm = {n_substeps, weno_linear, averaging filter (0 equal weights, 1 power-law shape),
 *         vertical WENO coefficients (0 index space, 1 from the level thicknesses),
 *         vertical momentum advection (0 centred, 1 WENO flux form)}.
 */
ora_t* ora_create(const int* igrid, const double* dgrid, const double* zf, const double* depth,
                  const double* taux, const double* tauy, const double* prm, const int* iprm) {
    ora_t* m = calloc(1, sizeof(ora_t));
    m->kind = igrid[0]; m->nx = igrid[1]; m->ny = igrid[2]; m->nz = igrid[3];
    m->px = igrid[4]; m->py = igrid[5];
    m->x0 = dgrid[0]; m->x1 = dgrid[1]; m->y0 = dgrid[2]; m->y1 = dgrid[3];
    m->dt = prm[0]; m->chi = prm[1]; m->g = prm[2]; m->rho0 = prm[3]; m->alpha = prm[4];
    m->beta_s = prm[5]; m->T0 = prm[6]; m->S0 = prm[7]; m->f0 = prm[8]; m->betap = prm[9];
    m->omega = prm[10]; m->radius = prm[11]; m->nu0 = prm[12]; m->ri_a = prm[13];
    m->nu_b = prm[14]; m->kappa_b = prm[15]; m->kappa_conv = prm[16]; m->weno_eps = prm[17];
    m->min_depth = prm[18];
    m->ns = iprm[0]; m->weno_linear = iprm[1]; m->filter = iprm[2];
    m->vweno = iprm[3]; m->mom_vadv = iprm[4];
    m->fw = malloc((m->ns > 0 ? m->ns : 1) * sizeof(double));
    if (m->ns > 0) ora_filter_weights(m->ns, m->filter, m->fw);
    int nx = m->nx, ny = m->ny, nz = m->nz;
    long n2 = (long)nx * ny, n3 = n2 * nz;
    m->zf = malloc((nz + 1) * sizeof(double));
    m->zc = malloc(nz * sizeof(double));
    m->dz = malloc(nz * sizeof(double));
    for (int k = 0; k <= nz; k++) m->zf[k] = zf[k];
    for (int k = 0; k < nz; k++) {
        m->zc[k] = 0.5 * (zf[k] + zf[k + 1]);
        m->dz[k] = zf[k + 1] - zf[k];
    }
    m->depth = malloc(n2 * sizeof(double));
    m->taux = malloc(n2 * sizeof(double));
    m->tauy = malloc(n2 * sizeof(double));
    m->kb = malloc(n2 * sizeof(int));
    memcpy(m->depth, depth, n2 * sizeof(double));
    memcpy(m->taux, taux, n2 * sizeof(double));
    memcpy(m->tauy, tauy, n2 * sizeof(double));
    /* full-cell bathymetry: cell k is wet when its centre lies above the sea floor;
     * columns shallower than min_depth are land */
    for (long c = 0; c < n2; c++) {
        int kb = nz;
        if (depth[c] >= m->min_depth)
            for (int k = nz - 1; k >= 0 && m->zc[k] > -depth[c]; k--) kb = k;
        m->kb[c] = kb;
    }
    double** arrs3[] = {&m->u, &m->v, &m->T, &m->S, &m->Gu0, &m->Gv0, &m->GT0, &m->GS0,
                        &m->b, &m->p, &m->w, &m->kap, &m->nu, &m->Gu, &m->Gv, &m->GT, &m->GS};
    for (unsigned a = 0; a < sizeof(arrs3) / sizeof(arrs3[0]); a++) *arrs3[a] = calloc(n3, sizeof(double));
    double** arrs2[] = {&m->eta, &m->GU, &m->GV, &m->U, &m->V, &m->Hu, &m->Hv};
    for (unsigned a = 0; a < sizeof(arrs2) / sizeof(arrs2[0]); a++) *arrs2[a] = calloc(n2, sizeof(double));
    /* depths of the u- and v-columns */
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            double hu = 0.0, hv = 0.0;
            for (int k = 0; k < nz; k++) {
                if (uwet(m, i, j, k)) hu += m->dz[k];
                if (vwet(m, i, j, k)) hv += m->dz[k];
            }
            m->Hu[(long)j * nx + i] = hu;
            m->Hv[(long)j * nx + i] = hv;
        }
    return m;
}

void ora_destroy(ora_t* m) {
    if (!m) return;
    double* arrs[] = {m->zf, m->zc, m->dz, m->depth, m->taux, m->tauy, m->u, m->v, m->T, m->S,
                      m->eta, m->Gu0, m->Gv0, m->GT0, m->GS0, m->b, m->p, m->w, m->kap, m->nu,
                      m->Gu, m->Gv, m->GT, m->GS, m->GU, m->GV, m->U, m->V, m->Hu, m->Hv};
    for (unsigned a = 0; a < sizeof(arrs) / sizeof(arrs[0]); a++) free(arrs[a]);
    free(m->kb);
    free(m->fw);
    free(m->ext_kap); free(m->ext_dGT); free(m->ext_dGS);
    free(m);
}

/* field ids: 0 u, 1 v, 2 T, 3 S, 4 eta, 5 Gu_prev, 6 Gv_prev, 7 GT_prev, 8 GS_prev,
 * 9 w, 10 p, 11 kappa, 12 nu, 13 Gu, 14 Gv, 15 GT, 16 GS, 17 Hu, 18 Hv, 19 b (2-D ids:
 * 4, 17, 18) */
static double* field_ptr(ora_t* m, int id, int* is2d) {
    *is2d = 0;
    switch (id) {
        case 0: return m->u;   case 1: return m->v;   case 2: return m->T;   case 3: return m->S;
        case 4: *is2d = 1; return m->eta;
        case 5: return m->Gu0; case 6: return m->Gv0; case 7: return m->GT0; case 8: return m->GS0;
        case 9: return m->w;   case 10: return m->p;  case 11: return m->kap; case 12: return m->nu;
        case 13: return m->Gu; case 14: return m->Gv; case 15: return m->GT; case 16: return m->GS;
        case 17: *is2d = 1; return m->Hu;
        case 18: *is2d = 1; return m->Hv;
        case 19: return m->b;
        default: return 0;
    }
}

/* Set a field; values on dry cells/faces (and on land columns for eta) become 0. */
int ora_set_field(ora_t* m, int id, const double* src) {
    int is2d;
    double* F = field_ptr(m, id, &is2d);
    if (!F) return -1;
    int nx = m->nx, ny = m->ny, nz = m->nz;
    if (is2d) {
        for (long c = 0; c < (long)nx * ny; c++) F[c] = (m->kb[c] < nz) ? src[c] : 0.0;
        return 0;
    }
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                long c = at3(m, i, j, k);
                int ok = (id == 0 || id == 5 || id == 13) ? uwet(m, i, j, k)
                       : (id == 1 || id == 6 || id == 14) ? vwet(m, i, j, k) : wet(m, i, j, k);
                F[c] = ok ? src[c] : 0.0;
            }
    return 0;
}

int ora_get_field(ora_t* m, int id, double* dst) {
    int is2d;
    double* F = field_ptr(m, id, &is2d);
    if (!F) return -1;
    long n = (long)m->nx * m->ny * (is2d ? 1 : m->nz);
    memcpy(dst, F, n * sizeof(double));
    return 0;
}

long ora_get_step(const ora_t* m) { return m->nstep; }
void ora_set_step(ora_t* m, long n) { m->nstep = n; }
int ora_kbot(const ora_t* m, int i, int j) { return kbot(m, i, j); }
