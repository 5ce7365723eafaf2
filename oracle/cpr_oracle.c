/*
 * cpr_oracle.c -- FP64 CPU oracle of the CPR hot path (arXiv 1709.01619).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg.  It is written from the paper's equations,
 * step by step, with no blocking or fusion, so that it can be read against
 * the paper.  It shares no code with the CUDA path.
 *
 * Map to the paper:
 *   Euler flux and equation of state ........ Sec. 2, Eqs. 3-5
 *   CPR differential form, per point ......... Sec. 2.2, Eqs. 16-17
 *   flux divergence Pi[div F] ................ Sec. 2.2 (chain rule variant,
 *                                              and the Lagrange-polynomial
 *                                              variant, which differentiates
 *                                              the interpolated flux)
 *   correction delta via Radau polynomials ... Sec. 2.2 (g_DG of Huynh)
 *   Rusanov common flux ...................... Sec. 2.2 Eq. 12, Sec. 4
 *   SSP-RK3, CFL time step ................... Sec. 4, Eq. 36
 *   element average .......................... Algorithm 9
 *   troubled-cell limiter .................... Sec. 2.6 Eq. 35, Algorithms 10-11
 *   averaged-solution error norm ............. Sec. 4
 * Readings where the paper is silent or garbled are listed next to the code
 * that takes them.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Threads                                                                  */
/* ------------------------------------------------------------------------ */
int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* Legendre polynomials                                                     */
/* ------------------------------------------------------------------------ */

/* P_k(x): Bonnet's recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}. */
double oracle_legendre(int k, double x)
{
    if (k == 0) return 1.0;
    double pm1 = 1.0, pk = x;
    for (int m = 1; m < k; ++m) {
        double pn = ((2.0 * m + 1.0) * x * pk - m * pm1) / (m + 1.0);
        pm1 = pk;
        pk = pn;
    }
    return pk;
}

/* P_k'(x): P'_{m+1} = P'_{m-1} + (2m+1) P_m, valid on the closed interval. */
double oracle_legendre_d(int k, double x)
{
    if (k == 0) return 0.0;
    double dm1 = 0.0;      /* P'_0 */
    double dk = 1.0;       /* P'_1 */
    for (int m = 1; m < k; ++m) {
        double dn = dm1 + (2.0 * m + 1.0) * oracle_legendre(m, x);
        dm1 = dk;
        dk = dn;
    }
    return dk;
}

/* P_k''(x) on the open interval from Legendre's equation
 * (1 - x^2) P'' - 2 x P' + k (k+1) P = 0. */
static double legendre_dd(int k, double x)
{
    return (2.0 * x * oracle_legendre_d(k, x) - k * (k + 1.0) * oracle_legendre(k, x)) /
           (1.0 - x * x);
}

static void sort_ascending(double* v, double* w, int n)
{
    for (int i = 1; i < n; ++i)
        for (int j = i; j > 0 && v[j - 1] > v[j]; --j) {
            double t = v[j]; v[j] = v[j - 1]; v[j - 1] = t;
            t = w[j]; w[j] = w[j - 1]; w[j - 1] = t;
        }
}

/* Gauss-Legendre: the n roots of P_n by Newton iteration,
 * w = 2 / ((1 - x^2) P_n'(x)^2). */
static void gauss_nodes(int n, double* x, double* w)
{
    for (int i = 0; i < n; ++i) {
        double z = cos(PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double dz = oracle_legendre(n, z) / oracle_legendre_d(n, z);
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        double d = oracle_legendre_d(n, z);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * d * d);
    }
    sort_ascending(x, w, n);
}

/* Gauss-Lobatto with n = p + 1 points: +-1 and the roots of P_p',
 * w = 2 / (p (p+1) P_p(x)^2).  The paper's CPR solution points (Sec. 2.2,
 * Fig. 1b). */
static void lobatto_nodes(int n, double* x, double* w)
{
    int p = n - 1;
    x[0] = -1.0;
    x[n - 1] = 1.0;
    for (int i = 1; i < n - 1; ++i) {
        double z = -cos(PI * i / p); /* Chebyshev-Lobatto starting guess */
        for (int it = 0; it < 100; ++it) {
            double dz = oracle_legendre_d(p, z) / legendre_dd(p, z);
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = z;
    }
    for (int i = 0; i < n; ++i) {
        double pp = oracle_legendre(p, x[i]);
        w[i] = 2.0 / (p * (p + 1.0) * pp * pp);
    }
    sort_ascending(x, w, n);
}

/* Lagrange basis l_l(x) through the nodes xi. */
static double lagrange(int n, const double* xi, int l, double x)
{
    double r = 1.0;
    for (int m = 0; m < n; ++m)
        if (m != l) r *= (x - xi[m]) / (xi[l] - xi[m]);
    return r;
}

/* l_l'(x) = sum_{k != l} 1/(xi_l - xi_k) prod_{m != l, k} (x - xi_m)/(xi_l - xi_m) */
static double lagrange_d(int n, const double* xi, int l, double x)
{
    double s = 0.0;
    for (int k = 0; k < n; ++k) {
        if (k == l) continue;
        double t = 1.0 / (xi[l] - xi[k]);
        for (int m = 0; m < n; ++m)
            if (m != l && m != k) t *= (x - xi[m]) / (xi[l] - xi[m]);
        s += t;
    }
    return s;
}

int oracle_tables(int p, int pts, oracle_tab* T)
{
    if (p < 1 || p > ORACLE_PMAX || !T) return -1;
    if (pts != OR_GAUSS && pts != OR_LOBATTO) return -1;
    memset(T, 0, sizeof(*T));
    int n = p + 1;
    T->n = n;
    if (pts == OR_GAUSS) gauss_nodes(n, T->xi, T->w);
    else lobatto_nodes(n, T->xi, T->w);
    for (int a = 0; a < n; ++a)
        for (int l = 0; l < n; ++l) T->D[a][l] = lagrange_d(n, T->xi, l, T->xi[a]);
    for (int l = 0; l < n; ++l) {
        T->lm[l] = lagrange(n, T->xi, l, -1.0);
        T->lp[l] = lagrange(n, T->xi, l, 1.0);
    }
    /* Correction functions g_DG (Sec. 2.2: Radau polynomials, Huynh):
     *   g_L = ((-1)^(p+1) / 2) (P_{p+1} - P_p),  g_L(-1) = 1, g_L(1) = 0
     *   g_R = (1/2) (P_{p+1} + P_p),             g_R(-1) = 0, g_R(1) = 1 */
    double sgn = (p % 2 == 0) ? -1.0 : 1.0; /* (-1)^(p+1) */
    for (int a = 0; a < n; ++a) {
        double d1 = oracle_legendre_d(p + 1, T->xi[a]);
        double d0 = oracle_legendre_d(p, T->xi[a]);
        T->dgl[a] = 0.5 * sgn * (d1 - d0);
        T->dgr[a] = 0.5 * (d1 + d0);
    }
    return 0;
}

/* Solve the n x n system A x = b by Gaussian elimination with partial
 * pivoting (A and b are overwritten); returns -1 if A is singular. */
static int solve_dense(int n, double A[ORACLE_NMAX][ORACLE_NMAX], double* b, double* x)
{
    for (int k = 0; k < n; ++k) {
        int piv = k;
        for (int r = k + 1; r < n; ++r)
            if (fabs(A[r][k]) > fabs(A[piv][k])) piv = r;
        if (A[piv][k] == 0.0) return -1;
        if (piv != k) {
            for (int m = 0; m < n; ++m) {
                double t = A[k][m]; A[k][m] = A[piv][m]; A[piv][m] = t;
            }
            double t = b[k]; b[k] = b[piv]; b[piv] = t;
        }
        for (int r = k + 1; r < n; ++r) {
            double f = A[r][k] / A[k][k];
            for (int m = k; m < n; ++m) A[r][m] -= f * A[k][m];
            b[r] -= f * b[k];
        }
    }
    for (int k = n - 1; k >= 0; --k) {
        double s = b[k];
        for (int m = k + 1; m < n; ++m) s -= A[k][m] * x[m];
        x[k] = s / A[k][k];
    }
    return 0;
}

int oracle_tables_corr(int p, int pts, int corr, oracle_tab* T)
{
    if (oracle_tables(p, pts, T)) return -1;
    if (corr == OR_CORR_GDG) return 0;
    if (corr != OR_CORR_NDG && corr != OR_CORR_NDG_LUMPED) return -1;
    int n = T->n;
    /* Nodal DG, Sec. 2.3: dq/dt + D f - L [f.n - F_com] = 0 with the lifting
     * matrix L = M^-1 M^A.  For the face xi = +1 of a tensor-product element
     * M^A = l(+1) (x) M_1d, and M_2d = M_1d (x) M_1d, so L reduces to
     * M_1d^-1 l(+1) along every line.  With n = +1 on the right face and -1
     * on the left one this is the CPR form with g_R' = M^-1 l(+1) and
     * g_L' = -M^-1 l(-1). */
    double M[ORACLE_NMAX][ORACLE_NMAX];
    if (corr == OR_CORR_NDG) {
        double gx[ORACLE_NMAX + 1], gw[ORACLE_NMAX + 1];
        gauss_nodes(n + 1, gx, gw); /* exact for the degree-2p integrands */
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                double s = 0.0;
                for (int q = 0; q < n + 1; ++q)
                    s += gw[q] * lagrange(n, T->xi, i, gx[q]) * lagrange(n, T->xi, j, gx[q]);
                M[i][j] = s;
            }
    } else {
        /* the integrals by the solution points' own quadrature */
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) M[i][j] = i == j ? T->w[i] : 0.0;
    }
    for (int side = 0; side < 2; ++side) {
        double A[ORACLE_NMAX][ORACLE_NMAX], b[ORACLE_NMAX], x[ORACLE_NMAX];
        for (int i = 0; i < n; ++i) {
            for (int j = 0; j < n; ++j) A[i][j] = M[i][j];
            b[i] = side ? T->lp[i] : T->lm[i];
        }
        if (solve_dense(n, A, b, x)) return -1;
        for (int a = 0; a < n; ++a) {
            if (side) T->dgr[a] = x[a];
            else T->dgl[a] = -x[a];
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sizes and coordinates                                                    */
/* ------------------------------------------------------------------------ */
int oracle_nvars(const oracle_cfg* c) { return c->eqn == OR_EULER ? 4 : 1; }

long oracle_state_size(const oracle_cfg* c)
{
    long n = c->p + 1;
    return (long)oracle_nvars(c) * c->nx * c->ny * n * n;
}

static int check_cfg(const oracle_cfg* c)
{
    if (!c) return -1;
    if (c->eqn != OR_ADVECTION && c->eqn != OR_EULER) return -1;
    if (c->scheme != OR_CPR && c->scheme != OR_FV_MUSCL && c->scheme != OR_FV_MUSCL3) return -1;
    if (c->scheme != OR_CPR) {
        /* one average per element; the MUSCL limiter is part of the
         * reconstruction */
        if (c->nx < 1 || c->ny < 1 || c->p != 0 || c->limiter) return -1;
        if (!(c->x1 > c->x0) || !(c->y1 > c->y0)) return -1;
        if (c->flux == OR_UPWIND && c->eqn != OR_ADVECTION) return -1;
        return 0;
    }
    if (c->nx < 1 || c->ny < 1 || c->p < 1 || c->p > ORACLE_PMAX) return -1;
    if (!(c->x1 > c->x0) || !(c->y1 > c->y0)) return -1;
    if (c->corr != OR_CORR_GDG && c->corr != OR_CORR_NDG && c->corr != OR_CORR_NDG_LUMPED) return -1;
    if (c->div == OR_DIV_CHAIN && c->eqn != OR_EULER && c->eqn != OR_ADVECTION) return -1;
    if (c->flux == OR_UPWIND && c->eqn != OR_ADVECTION) return -1;
    return 0;
}

int oracle_point_coords(const oracle_cfg* c, double* x, double* y)
{
    if (check_cfg(c)) return -1;
    if (c->scheme != OR_CPR) {
        /* FV: the element centre stands for the element */
        double hx = (c->x1 - c->x0) / c->nx, hy = (c->y1 - c->y0) / c->ny;
        for (int j = 0; j < c->ny; ++j)
            for (int i = 0; i < c->nx; ++i) {
                x[(long)j * c->nx + i] = c->x0 + hx * (i + 0.5);
                y[(long)j * c->nx + i] = c->y0 + hy * (j + 0.5);
            }
        return 0;
    }
    oracle_tab T;
    oracle_tables_corr(c->p, c->pts, c->corr, &T);
    int n = T.n;
    double hx = (c->x1 - c->x0) / c->nx, hy = (c->y1 - c->y0) / c->ny;
    for (int j = 0; j < c->ny; ++j)
        for (int i = 0; i < c->nx; ++i) {
            long e = (long)j * c->nx + i;
            for (int b = 0; b < n; ++b)
                for (int a = 0; a < n; ++a) {
                    /* affine map of Sec. 2: xi in [-1, 1] -> element */
                    x[e * n * n + b * n + a] = c->x0 + hx * (i + 0.5 * (T.xi[a] + 1.0));
                    y[e * n * n + b * n + a] = c->y0 + hy * (j + 0.5 * (T.xi[b] + 1.0));
                }
        }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Physics: Sec. 2, Eqs. 3-5                                                */
/* ------------------------------------------------------------------------ */

/* p = (gamma - 1)(e - rho (u^2 + v^2) / 2), Eq. 5 */
static double pressure(double gam, const double* q)
{
    double u = q[1] / q[0], v = q[2] / q[0];
    return (gam - 1.0) * (q[3] - 0.5 * (q[1] * u + q[2] * v));
}

/* Normal flux F_n = nx f + ny g of Eq. 4, written with the normal velocity
 * Vn = nx u + ny v: (rho Vn, rho u Vn + nx p, rho v Vn + ny p, (e + p) Vn). */
static void normal_flux(const oracle_cfg* c, const double* q, double nx, double ny,
                        double* F)
{
    if (c->eqn == OR_ADVECTION) {
        F[0] = (c->ax * nx + c->ay * ny) * q[0];
        return;
    }
    double u = q[1] / q[0], v = q[2] / q[0];
    double p = pressure(c->gamma, q);
    double vn = nx * u + ny * v;
    F[0] = q[0] * vn;
    F[1] = q[1] * vn + nx * p;
    F[2] = q[2] * vn + ny * p;
    F[3] = (q[3] + p) * vn;
}

/* Largest signal speed along the normal: |Vn| + c, c = sqrt(gamma p / rho). */
static double normal_speed(const oracle_cfg* c, const double* q, double nx, double ny)
{
    if (c->eqn == OR_ADVECTION) return fabs(c->ax * nx + c->ay * ny);
    double u = q[1] / q[0], v = q[2] / q[0];
    double cs = sqrt(c->gamma * pressure(c->gamma, q) / q[0]);
    return fabs(nx * u + ny * v) + cs;
}

/* Directional derivative of the normal flux: dF = (dF_n/dq) dq (the
 * "analytical flux derivative" used by the chain-rule divergence, Sec. 2.2). */
static void normal_flux_jvp(const oracle_cfg* c, const double* q, const double* dq,
                            double nx, double ny, double* dF)
{
    if (c->eqn == OR_ADVECTION) {
        dF[0] = (c->ax * nx + c->ay * ny) * dq[0];
        return;
    }
    double g1 = c->gamma - 1.0;
    double r = q[0], u = q[1] / r, v = q[2] / r;
    double p = pressure(c->gamma, q);
    double vn = nx * u + ny * v;
    double dvn = (nx * dq[1] + ny * dq[2] - vn * dq[0]) / r;
    double dp = g1 * (dq[3] - (u * dq[1] + v * dq[2]) + 0.5 * (u * u + v * v) * dq[0]);
    dF[0] = nx * dq[1] + ny * dq[2];
    dF[1] = dq[1] * vn + q[1] * dvn + nx * dp;
    dF[2] = dq[2] * vn + q[2] * dvn + ny * dp;
    dF[3] = (dq[3] + dp) * vn + (q[3] + p) * dvn;
}

/* qbar += (dF_n/dq)^T w */
static void normal_flux_vjp(const oracle_cfg* c, const double* q, const double* w,
                            double nx, double ny, double* qbar)
{
    if (c->eqn == OR_ADVECTION) {
        qbar[0] += (c->ax * nx + c->ay * ny) * w[0];
        return;
    }
    double g1 = c->gamma - 1.0;
    double r = q[0], u = q[1] / r, v = q[2] / r;
    double p = pressure(c->gamma, q);
    double vn = nx * u + ny * v;
    double dvn[4] = {-vn / r, nx / r, ny / r, 0.0};
    double dpq[4] = {g1 * 0.5 * (u * u + v * v), -g1 * u, -g1 * v, g1};
    double C = w[1] * q[1] + w[2] * q[2] + w[3] * (q[3] + p);
    double P = w[1] * nx + w[2] * ny + w[3] * vn;
    qbar[0] += C * dvn[0] + P * dpq[0];
    qbar[1] += w[0] * nx + vn * w[1] + C * dvn[1] + P * dpq[1];
    qbar[2] += w[0] * ny + vn * w[2] + C * dvn[2] + P * dpq[2];
    qbar[3] += vn * w[3] + C * dvn[3] + P * dpq[3];
}

/* Gradient of the signal speed |Vn| + c with respect to q (Euler). */
static void normal_speed_grad(const oracle_cfg* c, const double* q, double nx, double ny,
                              double* gs)
{
    if (c->eqn == OR_ADVECTION) {
        gs[0] = 0.0;
        return;
    }
    double g1 = c->gamma - 1.0;
    double r = q[0], u = q[1] / r, v = q[2] / r;
    double p = pressure(c->gamma, q);
    double cs = sqrt(c->gamma * p / r);
    double vn = nx * u + ny * v;
    double sg = vn >= 0.0 ? 1.0 : -1.0;
    double dvn[4] = {-vn / r, nx / r, ny / r, 0.0};
    double dpq[4] = {g1 * 0.5 * (u * u + v * v), -g1 * u, -g1 * v, g1};
    double k = c->gamma / (2.0 * cs * r);
    for (int m = 0; m < 4; ++m) {
        double dcs = k * (dpq[m] - (m == 0 ? p / r : 0.0));
        gs[m] = sg * dvn[m] + dcs;
    }
}

/* ------------------------------------------------------------------------ */
/* Common flux (Sec. 2.2 Eq. 12 replaces the normal flux by a Riemann flux;  */
/* Sec. 4 names the Rusanov solver)                                          */
/* ------------------------------------------------------------------------ */

/* Rusanov: F = (F_n(qm) + F_n(qp)) / 2 - lambda (qp - qm) / 2, with
 * lambda = max(|Vn(qm)| + c(qm), |Vn(qp)| + c(qp))  (reading: the paper does
 * not state lambda; the larger of the two one-sided speeds is taken).
 * Upwind (linear advection only): F = a_n qm if a_n >= 0, else a_n qp. */
/* Roe's flux for the Euler equations along the unit normal (nx, ny):
 *   F = (F_n(qm) + F_n(qp)) / 2 - (1/2) sum_k |lambda_k| alpha_k r_k
 * over the characteristic fields of the Roe-averaged state (density
 * sqrt(rho_m rho_p), velocity and total enthalpy averaged with weights
 * sqrt(rho)): acoustic waves lambda = Vn -+ c with strengths
 * (dp -+ rho c dVn) / (2 c^2), the entropy wave lambda = Vn with dRho -
 * dp / c^2, the shear wave lambda = Vn with rho dVt (t = (-ny, nx)).
 * Entropy fix of Harten and Hyman on the acoustic fields: with lambda_m,
 * lambda_p the field's speed at the two states and delta = max(0, lambda -
 * lambda_m, lambda_p - lambda) (positive only across a transonic
 * rarefaction), |lambda| < delta is replaced by (lambda^2 + delta^2) /
 * (2 delta); shocks and contacts keep the plain Roe flux. */
/* |lambda| with the Harten-Hyman fix (lambda_m, lambda_p: the field's speed
 * at the minus and plus states). */
static double roe_fix(double lam, double lam_m, double lam_p)
{
    double d = 0.0;
    if (lam - lam_m > d) d = lam - lam_m;
    if (lam_p - lam > d) d = lam_p - lam;
    double a = fabs(lam);
    return a < d ? (lam * lam + d * d) / (2.0 * d) : a;
}

static void roe_flux(const oracle_cfg* c, const double* qm, const double* qp, double nx, double ny,
                     double* F)
{
    double g = c->gamma;
    double Fm[4], Fp[4];
    normal_flux(c, qm, nx, ny, Fm);
    normal_flux(c, qp, nx, ny, Fp);
    double um = qm[1] / qm[0], vm = qm[2] / qm[0], up = qp[1] / qp[0], vp = qp[2] / qp[0];
    double pm = pressure(g, qm), pp = pressure(g, qp);
    double Hm = (qm[3] + pm) / qm[0], Hp = (qp[3] + pp) / qp[0];
    double wm = sqrt(qm[0]), wp = sqrt(qp[0]);
    double rho = wm * wp;
    double u = (wm * um + wp * up) / (wm + wp);
    double v = (wm * vm + wp * vp) / (wm + wp);
    double H = (wm * Hm + wp * Hp) / (wm + wp);
    double cs = sqrt((g - 1.0) * (H - 0.5 * (u * u + v * v)));
    double vn = nx * u + ny * v, vt = -ny * u + nx * v;
    double dr = qp[0] - qm[0], dp = pp - pm;
    double dvn = (nx * up + ny * vp) - (nx * um + ny * vm);
    double dvt = (-ny * up + nx * vp) - (-ny * um + nx * vm);
    double a1 = (dp - rho * cs * dvn) / (2.0 * cs * cs);
    double a2 = dr - dp / (cs * cs);
    double a3 = rho * dvt;
    double a4 = (dp + rho * cs * dvn) / (2.0 * cs * cs);
    double cm = sqrt(g * pm / qm[0]), cp = sqrt(g * pp / qp[0]);
    double vnm = nx * um + ny * vm, vnp = nx * up + ny * vp;
    double l1 = roe_fix(vn - cs, vnm - cm, vnp - cp);
    double l2 = fabs(vn);
    double l4 = roe_fix(vn + cs, vnm + cm, vnp + cp);
    double r1[4] = {1.0, u - cs * nx, v - cs * ny, H - vn * cs};
    double r2[4] = {1.0, u, v, 0.5 * (u * u + v * v)};
    double r3[4] = {0.0, -ny, nx, vt};
    double r4[4] = {1.0, u + cs * nx, v + cs * ny, H + vn * cs};
    for (int k = 0; k < 4; ++k)
        F[k] = 0.5 * (Fm[k] + Fp[k]) -
               0.5 * (l1 * a1 * r1[k] + l2 * a2 * r2[k] + l2 * a3 * r3[k] + l4 * a4 * r4[k]);
}

void oracle_common_flux(const oracle_cfg* c, const double* qm, const double* qp,
                        double nx, double ny, double* F)
{
    int V = oracle_nvars(c);
    if (c->eqn == OR_EULER && c->flux == OR_ROE) {
        roe_flux(c, qm, qp, nx, ny, F);
        return;
    }
    if (c->eqn == OR_ADVECTION && (c->flux == OR_UPWIND || c->flux == OR_ROE)) {
        double an = c->ax * nx + c->ay * ny;
        F[0] = an >= 0.0 ? an * qm[0] : an * qp[0];
        return;
    }
    double Fm[4], Fp[4];
    normal_flux(c, qm, nx, ny, Fm);
    normal_flux(c, qp, nx, ny, Fp);
    double sm = normal_speed(c, qm, nx, ny), sp = normal_speed(c, qp, nx, ny);
    double lam = sm >= sp ? sm : sp;
    for (int v = 0; v < V; ++v) F[v] = 0.5 * (Fm[v] + Fp[v]) - 0.5 * lam * (qp[v] - qm[v]);
}

static void common_flux_jvp(const oracle_cfg* c, const double* qm, const double* qp,
                            const double* dqm, const double* dqp, double nx, double ny,
                            double* dF)
{
    int V = oracle_nvars(c);
    if (c->eqn == OR_ADVECTION && c->flux == OR_UPWIND) {
        double an = c->ax * nx + c->ay * ny;
        dF[0] = an >= 0.0 ? an * dqm[0] : an * dqp[0];
        return;
    }
    double dFm[4], dFp[4];
    normal_flux_jvp(c, qm, dqm, nx, ny, dFm);
    normal_flux_jvp(c, qp, dqp, nx, ny, dFp);
    double sm = normal_speed(c, qm, nx, ny), sp = normal_speed(c, qp, nx, ny);
    double lam = sm >= sp ? sm : sp;
    double gs[4] = {0, 0, 0, 0};
    double dlam = 0.0;
    if (sm >= sp) {
        normal_speed_grad(c, qm, nx, ny, gs);
        for (int m = 0; m < V; ++m) dlam += gs[m] * dqm[m];
    } else {
        normal_speed_grad(c, qp, nx, ny, gs);
        for (int m = 0; m < V; ++m) dlam += gs[m] * dqp[m];
    }
    for (int v = 0; v < V; ++v)
        dF[v] = 0.5 * (dFm[v] + dFp[v]) - 0.5 * dlam * (qp[v] - qm[v]) -
                0.5 * lam * (dqp[v] - dqm[v]);
}

static void common_flux_vjp(const oracle_cfg* c, const double* qm, const double* qp,
                            const double* w, double nx, double ny, double* qbm,
                            double* qbp)
{
    int V = oracle_nvars(c);
    if (c->eqn == OR_ADVECTION && c->flux == OR_UPWIND) {
        double an = c->ax * nx + c->ay * ny;
        if (an >= 0.0) qbm[0] += an * w[0];
        else qbp[0] += an * w[0];
        return;
    }
    double hw[4];
    for (int v = 0; v < V; ++v) hw[v] = 0.5 * w[v];
    normal_flux_vjp(c, qm, hw, nx, ny, qbm);
    normal_flux_vjp(c, qp, hw, nx, ny, qbp);
    double sm = normal_speed(c, qm, nx, ny), sp = normal_speed(c, qp, nx, ny);
    double lam = sm >= sp ? sm : sp;
    double jump = 0.0;
    for (int v = 0; v < V; ++v) {
        qbm[v] += 0.5 * lam * w[v];
        qbp[v] -= 0.5 * lam * w[v];
        jump += w[v] * (qp[v] - qm[v]);
    }
    double gs[4] = {0, 0, 0, 0};
    if (sm >= sp) {
        normal_speed_grad(c, qm, nx, ny, gs);
        for (int m = 0; m < V; ++m) qbm[m] -= 0.5 * jump * gs[m];
    } else {
        normal_speed_grad(c, qp, nx, ny, gs);
        for (int m = 0; m < V; ++m) qbp[m] -= 0.5 * jump * gs[m];
    }
}

/* ------------------------------------------------------------------------ */
/* CPR residual, Sec. 2.2 Eq. 16-17                                          */
/* ------------------------------------------------------------------------ */

/* Value of variable v at point (a, b) of element e. */
#define QAT(q, v, e, b, a) (q)[(((long)(v) * ne + (e)) * n + (b)) * n + (a)]

typedef struct {
    /* edge states of one element: left/right edges indexed by row b,
     * bottom/top edges indexed by column a */
    double qL[4][ORACLE_NMAX], qR[4][ORACLE_NMAX], qB[4][ORACLE_NMAX], qT[4][ORACLE_NMAX];
} edge_states;

/* Interpolate the solution to the four edges: q(-1, eta_b) = sum_l l_l(-1)
 * q_{l,b} etc. (Fig. 1; for Lobatto points these are copies of edge points). */
static void element_edge_states(const oracle_cfg* c, const oracle_tab* T, const double* q,
                                long e, edge_states* E)
{
    int n = T->n, V = oracle_nvars(c);
    long ne = (long)c->nx * c->ny;
    for (int v = 0; v < V; ++v)
        for (int k = 0; k < n; ++k) {
            double sL = 0, sR = 0, sB = 0, sT = 0;
            for (int l = 0; l < n; ++l) {
                sL += T->lm[l] * QAT(q, v, e, k, l);
                sR += T->lp[l] * QAT(q, v, e, k, l);
                sB += T->lm[l] * QAT(q, v, e, l, k);
                sT += T->lp[l] * QAT(q, v, e, l, k);
            }
            E->qL[v][k] = sL;
            E->qR[v][k] = sR;
            E->qB[v][k] = sB;
            E->qT[v][k] = sT;
        }
}

/* Neighbour indices; -1 marks a transmissive boundary (reading: the ghost
 * state equals the interior edge state, so the common flux is f(q-)). */
static void neighbours(const oracle_cfg* c, int i, int j, long* eL, long* eR, long* eB,
                       long* eT)
{
    int nx = c->nx, ny = c->ny;
    int il = i - 1, ir = i + 1, jb = j - 1, jt = j + 1;
    if (c->bc_x == OR_PERIODIC) {
        il = (il + nx) % nx;
        ir = ir % nx;
    }
    if (c->bc_y == OR_PERIODIC) {
        jb = (jb + ny) % ny;
        jt = jt % ny;
    }
    *eL = (il >= 0) ? (long)j * nx + il : -1;
    *eR = (ir < nx) ? (long)j * nx + ir : -1;
    *eB = (jb >= 0) ? (long)jb * nx + i : -1;
    *eT = (jt < ny) ? (long)jt * nx + i : -1;
}

/* Common fluxes on the four edges of element (i, j): FL/FR in +x through the
 * left/right edge for each row b, GB/GT in +y through the bottom/top edge for
 * each column a. */
typedef struct {
    double FL[4][ORACLE_NMAX], FR[4][ORACLE_NMAX], GB[4][ORACLE_NMAX], GT[4][ORACLE_NMAX];
} edge_fluxes;

static void element_common_fluxes(const oracle_cfg* c, const oracle_tab* T, const double* q,
                                  int i, int j, const edge_states* own, edge_fluxes* F)
{
    int n = T->n, V = oracle_nvars(c);
    long eL, eR, eB, eT;
    neighbours(c, i, j, &eL, &eR, &eB, &eT);
    edge_states NL, NR, NB, NT;
    if (eL >= 0) element_edge_states(c, T, q, eL, &NL);
    if (eR >= 0) element_edge_states(c, T, q, eR, &NR);
    if (eB >= 0) element_edge_states(c, T, q, eB, &NB);
    if (eT >= 0) element_edge_states(c, T, q, eT, &NT);
    for (int k = 0; k < n; ++k) {
        double qm[4], qp[4], out[4];
        /* left edge: minus = right edge of the left neighbour */
        for (int v = 0; v < V; ++v) {
            qp[v] = own->qL[v][k];
            qm[v] = eL >= 0 ? NL.qR[v][k] : own->qL[v][k];
        }
        oracle_common_flux(c, qm, qp, 1.0, 0.0, out);
        for (int v = 0; v < V; ++v) F->FL[v][k] = out[v];
        /* right edge: plus = left edge of the right neighbour */
        for (int v = 0; v < V; ++v) {
            qm[v] = own->qR[v][k];
            qp[v] = eR >= 0 ? NR.qL[v][k] : own->qR[v][k];
        }
        oracle_common_flux(c, qm, qp, 1.0, 0.0, out);
        for (int v = 0; v < V; ++v) F->FR[v][k] = out[v];
        /* bottom edge */
        for (int v = 0; v < V; ++v) {
            qp[v] = own->qB[v][k];
            qm[v] = eB >= 0 ? NB.qT[v][k] : own->qB[v][k];
        }
        oracle_common_flux(c, qm, qp, 0.0, 1.0, out);
        for (int v = 0; v < V; ++v) F->GB[v][k] = out[v];
        /* top edge */
        for (int v = 0; v < V; ++v) {
            qm[v] = own->qT[v][k];
            qp[v] = eT >= 0 ? NT.qB[v][k] : own->qT[v][k];
        }
        oracle_common_flux(c, qm, qp, 0.0, 1.0, out);
        for (int v = 0; v < V; ++v) F->GT[v][k] = out[v];
    }
}

/* Residual of one element.  With f_ab = f(q_ab), g_ab = g(q_ab):
 *   Pi[div F]_ab (LP) = (2/hx) sum_l D_al f_lb + (2/hy) sum_l D_bl g_al
 *   Pi[div F]_ab (CR) = (2/hx) A(q_ab) sum_l D_al q_lb
 *                       + (2/hy) B(q_ab) sum_l D_bl q_al       (chain rule)
 *   delta_ab = (2/hx) [(F*_L,b - f_L,b) g_L'(xi_a) + (F*_R,b - f_R,b) g_R'(xi_a)]
 *            + (2/hy) [(G*_B,a - g_B,a) g_L'(eta_b) + (G*_T,a - g_T,a) g_R'(eta_b)]
 *   R_ab = -(Pi[div F]_ab + delta_ab)                           (Eq. 16-17)
 * The discontinuous edge flux f_L,b is the edge value of the flux polynomial:
 * sum_l l_l(-1) f_lb for LP; f(q_L,b) for CR (reading, the paper is silent). */
static void element_residual(const oracle_cfg* c, const oracle_tab* T, const double* q,
                             int i, int j, double* R)
{
    int n = T->n, V = oracle_nvars(c);
    long ne = (long)c->nx * c->ny;
    long e = (long)j * c->nx + i;
    double hx = (c->x1 - c->x0) / c->nx, hy = (c->y1 - c->y0) / c->ny;

    double fpt[4][ORACLE_NMAX][ORACLE_NMAX], gpt[4][ORACLE_NMAX][ORACLE_NMAX];
    for (int b = 0; b < n; ++b)
        for (int a = 0; a < n; ++a) {
            double qa[4], f[4], g[4];
            for (int v = 0; v < V; ++v) qa[v] = QAT(q, v, e, b, a);
            normal_flux(c, qa, 1.0, 0.0, f);
            normal_flux(c, qa, 0.0, 1.0, g);
            for (int v = 0; v < V; ++v) {
                fpt[v][b][a] = f[v];
                gpt[v][b][a] = g[v];
            }
        }

    edge_states own;
    element_edge_states(c, T, q, e, &own);

    /* discontinuous flux at the edges */
    double fL[4][ORACLE_NMAX], fR[4][ORACLE_NMAX], gB[4][ORACLE_NMAX], gT[4][ORACLE_NMAX];
    for (int k = 0; k < n; ++k) {
        if (c->div == OR_DIV_LP) {
            for (int v = 0; v < V; ++v) {
                double sL = 0, sR = 0, sB = 0, sT = 0;
                for (int l = 0; l < n; ++l) {
                    sL += T->lm[l] * fpt[v][k][l];
                    sR += T->lp[l] * fpt[v][k][l];
                    sB += T->lm[l] * gpt[v][l][k];
                    sT += T->lp[l] * gpt[v][l][k];
                }
                fL[v][k] = sL; fR[v][k] = sR; gB[v][k] = sB; gT[v][k] = sT;
            }
        } else {
            double qe[4], out[4];
            for (int v = 0; v < V; ++v) qe[v] = own.qL[v][k];
            normal_flux(c, qe, 1.0, 0.0, out);
            for (int v = 0; v < V; ++v) fL[v][k] = out[v];
            for (int v = 0; v < V; ++v) qe[v] = own.qR[v][k];
            normal_flux(c, qe, 1.0, 0.0, out);
            for (int v = 0; v < V; ++v) fR[v][k] = out[v];
            for (int v = 0; v < V; ++v) qe[v] = own.qB[v][k];
            normal_flux(c, qe, 0.0, 1.0, out);
            for (int v = 0; v < V; ++v) gB[v][k] = out[v];
            for (int v = 0; v < V; ++v) qe[v] = own.qT[v][k];
            normal_flux(c, qe, 0.0, 1.0, out);
            for (int v = 0; v < V; ++v) gT[v][k] = out[v];
        }
    }

    edge_fluxes F;
    element_common_fluxes(c, T, q, i, j, &own, &F);

    for (int b = 0; b < n; ++b)
        for (int a = 0; a < n; ++a) {
            double dfx[4], dgy[4];
            if (c->div == OR_DIV_LP) {
                for (int v = 0; v < V; ++v) {
                    double sx = 0, sy = 0;
                    for (int l = 0; l < n; ++l) {
                        sx += T->D[a][l] * fpt[v][b][l];
                        sy += T->D[b][l] * gpt[v][l][a];
                    }
                    dfx[v] = sx;
                    dgy[v] = sy;
                }
            } else {
                double dqx[4], dqy[4], qa[4];
                for (int v = 0; v < V; ++v) {
                    double sx = 0, sy = 0;
                    for (int l = 0; l < n; ++l) {
                        sx += T->D[a][l] * QAT(q, v, e, b, l);
                        sy += T->D[b][l] * QAT(q, v, e, l, a);
                    }
                    dqx[v] = sx;
                    dqy[v] = sy;
                    qa[v] = QAT(q, v, e, b, a);
                }
                normal_flux_jvp(c, qa, dqx, 1.0, 0.0, dfx);
                normal_flux_jvp(c, qa, dqy, 0.0, 1.0, dgy);
            }
            for (int v = 0; v < V; ++v) {
                double xs = dfx[v] + (F.FL[v][b] - fL[v][b]) * T->dgl[a] +
                            (F.FR[v][b] - fR[v][b]) * T->dgr[a];
                double ys = dgy[v] + (F.GB[v][a] - gB[v][a]) * T->dgl[b] +
                            (F.GT[v][a] - gT[v][a]) * T->dgr[b];
                QAT(R, v, e, b, a) = -(2.0 / hx) * xs - (2.0 / hy) * ys;
            }
        }
}

/* ------------------------------------------------------------------------ */
/* FV with second-order MUSCL reconstruction (Sec. 2.1; Sec. 2.6; the        */
/* reconstruct-then-Riemann-flux steps of Algorithm 1)                       */
/* ------------------------------------------------------------------------ */

/* Average of variable v in element (i, j), ghosts included: periodic
 * directions wrap, transmissive ones repeat the boundary element (zero
 * gradient, so the boundary face sees the boundary state on both sides). */
static double fv_cell(const oracle_cfg* c, const double* q, int v, int i, int j)
{
    int nx = c->nx, ny = c->ny;
    if (i < 0 || i >= nx) {
        if (c->bc_x == OR_PERIODIC) i = ((i % nx) + nx) % nx;
        else i = i < 0 ? 0 : nx - 1;
    }
    if (j < 0 || j >= ny) {
        if (c->bc_y == OR_PERIODIC) j = ((j % ny) + ny) % ny;
        else j = j < 0 ? 0 : ny - 1;
    }
    return q[(long)v * nx * ny + (long)j * nx + i];
}

static double minmod2(double a, double b);

/* Limited change of variable v across element (i, j) in direction d (0: x,
 * 1: y): minmod of the forward and backward differences of the averages. */
static double fv_slope(const oracle_cfg* c, const double* q, int v, int i, int j, int d)
{
    int di = d == 0, dj = d == 1;
    double qc = fv_cell(c, q, v, i, j);
    double fwd = fv_cell(c, q, v, i + di, j + dj) - qc;
    double bwd = qc - fv_cell(c, q, v, i - di, j - dj);
    return minmod2(fwd, bwd);
}

/* Third-order MUSCL (Sec. 2.6; the paper gives no formula): van Leer's
 * kappa-scheme with kappa = 1/3, the reconstruction that is exact for the
 * averages of a parabola,
 *   q_{i+1/2}^- = q_i + (1 - kappa)/4 D- + (1 + kappa)/4 D+,
 * with each one-sided difference limited by minmod against b times the
 * other, b = (3 - kappa)/(1 - kappa) = 4 (the largest b for which the face
 * value stays between the neighbouring averages):
 *   q_{i+1/2}^- = q_i + (1/6) mm(D-, 4 D+) + (1/3) mm(D+, 4 D-),
 *   q_{i-1/2}^+ = q_i - (1/6) mm(D+, 4 D-) - (1/3) mm(D-, 4 D+),
 * D+ = q_{i+1} - q_i, D- = q_i - q_{i-1} along direction d. */
static void fv3_sides(const oracle_cfg* c, const double* q, int v, int i, int j, int d, double* up,
                      double* down)
{
    int di = d == 0, dj = d == 1;
    double qc = fv_cell(c, q, v, i, j);
    double dp = fv_cell(c, q, v, i + di, j + dj) - qc;
    double dm = qc - fv_cell(c, q, v, i - di, j - dj);
    *up = qc + (minmod2(dm, 4.0 * dp) / 6.0 + minmod2(dp, 4.0 * dm) / 3.0);
    *down = qc - (minmod2(dp, 4.0 * dm) / 6.0 + minmod2(dm, 4.0 * dp) / 3.0);
}

/* States on both sides of the face between element (i, j) and its +d
 * neighbour.  Second order: each element's average moved half its limited
 * change towards the face; third order: fv3_sides. */
static void fv_face_states(const oracle_cfg* c, const double* q, int i, int j, int d,
                           double* qm, double* qp)
{
    int V = oracle_nvars(c), di = d == 0, dj = d == 1;
    for (int v = 0; v < V; ++v) {
        if (c->scheme == OR_FV_MUSCL3) {
            double up, down;
            fv3_sides(c, q, v, i, j, d, &up, &down);
            qm[v] = up;
            fv3_sides(c, q, v, i + di, j + dj, d, &up, &down);
            qp[v] = down;
        } else {
            qm[v] = fv_cell(c, q, v, i, j) + 0.5 * fv_slope(c, q, v, i, j, d);
            qp[v] = fv_cell(c, q, v, i + di, j + dj) - 0.5 * fv_slope(c, q, v, i + di, j + dj, d);
        }
    }
}

static void fv_element_residual(const oracle_cfg* c, const double* q, int i, int j, double* R)
{
    int V = oracle_nvars(c);
    long ne = (long)c->nx * c->ny, e = (long)j * c->nx + i;
    double hx = (c->x1 - c->x0) / c->nx, hy = (c->y1 - c->y0) / c->ny;
    double qm[4], qp[4], fw[4], fe[4], gs[4], gn[4];
    fv_face_states(c, q, i - 1, j, 0, qm, qp);
    oracle_common_flux(c, qm, qp, 1.0, 0.0, fw);   /* f_{i-1/2,j} */
    fv_face_states(c, q, i, j, 0, qm, qp);
    oracle_common_flux(c, qm, qp, 1.0, 0.0, fe);   /* f_{i+1/2,j} */
    fv_face_states(c, q, i, j - 1, 1, qm, qp);
    oracle_common_flux(c, qm, qp, 0.0, 1.0, gs);   /* g_{i,j-1/2} */
    fv_face_states(c, q, i, j, 1, qm, qp);
    oracle_common_flux(c, qm, qp, 0.0, 1.0, gn);   /* g_{i,j+1/2} */
    for (int v = 0; v < V; ++v) R[(long)v * ne + e] = -(fe[v] - fw[v]) / hx - (gn[v] - gs[v]) / hy;
}

int oracle_residual(const oracle_cfg* c, const double* q, double* R)
{
    if (check_cfg(c) || !q || !R) return -1;
    if (c->scheme != OR_CPR) {
        long ne = (long)c->nx * c->ny;
#pragma omp parallel for schedule(static)
        for (long e = 0; e < ne; ++e) fv_element_residual(c, q, (int)(e % c->nx), (int)(e / c->nx), R);
        return 0;
    }
    oracle_tab T;
    oracle_tables_corr(c->p, c->pts, c->corr, &T);
    long ne = (long)c->nx * c->ny;
#pragma omp parallel for schedule(static)
    for (long e = 0; e < ne; ++e) element_residual(c, &T, q, (int)(e % c->nx), (int)(e / c->nx), R);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Linearised residual and its transpose (LP divergence only)               */
/* ------------------------------------------------------------------------ */

/* dR = (dR/dq) dq, the same steps as element_residual differentiated. */
static void element_residual_jvp(const oracle_cfg* c, const oracle_tab* T, const double* q,
                                 const double* dq, int i, int j, double* dR)
{
    int n = T->n, V = oracle_nvars(c);
    long ne = (long)c->nx * c->ny;
    long e = (long)j * c->nx + i;
    double hx = (c->x1 - c->x0) / c->nx, hy = (c->y1 - c->y0) / c->ny;

    double dfpt[4][ORACLE_NMAX][ORACLE_NMAX], dgpt[4][ORACLE_NMAX][ORACLE_NMAX];
    for (int b = 0; b < n; ++b)
        for (int a = 0; a < n; ++a) {
            double qa[4], da[4], df[4], dg[4];
            for (int v = 0; v < V; ++v) {
                qa[v] = QAT(q, v, e, b, a);
                da[v] = QAT(dq, v, e, b, a);
            }
            normal_flux_jvp(c, qa, da, 1.0, 0.0, df);
            normal_flux_jvp(c, qa, da, 0.0, 1.0, dg);
            for (int v = 0; v < V; ++v) {
                dfpt[v][b][a] = df[v];
                dgpt[v][b][a] = dg[v];
            }
        }
    long eL, eR, eB, eT;
    neighbours(c, i, j, &eL, &eR, &eB, &eT);
    edge_states own, down, NL, NR, NB, NT, dNL, dNR, dNB, dNT;
    element_edge_states(c, T, q, e, &own);
    element_edge_states(c, T, dq, e, &down);
    if (eL >= 0) { element_edge_states(c, T, q, eL, &NL); element_edge_states(c, T, dq, eL, &dNL); }
    if (eR >= 0) { element_edge_states(c, T, q, eR, &NR); element_edge_states(c, T, dq, eR, &dNR); }
    if (eB >= 0) { element_edge_states(c, T, q, eB, &NB); element_edge_states(c, T, dq, eB, &dNB); }
    if (eT >= 0) { element_edge_states(c, T, q, eT, &NT); element_edge_states(c, T, dq, eT, &dNT); }

    double dFL[4][ORACLE_NMAX], dFR[4][ORACLE_NMAX], dGB[4][ORACLE_NMAX], dGT[4][ORACLE_NMAX];
    for (int k = 0; k < n; ++k) {
        double qm[4], qp[4], dqm[4], dqp[4], out[4];
        for (int v = 0; v < V; ++v) {
            qp[v] = own.qL[v][k]; dqp[v] = down.qL[v][k];
            qm[v] = eL >= 0 ? NL.qR[v][k] : own.qL[v][k];
            dqm[v] = eL >= 0 ? dNL.qR[v][k] : down.qL[v][k];
        }
        common_flux_jvp(c, qm, qp, dqm, dqp, 1.0, 0.0, out);
        for (int v = 0; v < V; ++v) dFL[v][k] = out[v];
        for (int v = 0; v < V; ++v) {
            qm[v] = own.qR[v][k]; dqm[v] = down.qR[v][k];
            qp[v] = eR >= 0 ? NR.qL[v][k] : own.qR[v][k];
            dqp[v] = eR >= 0 ? dNR.qL[v][k] : down.qR[v][k];
        }
        common_flux_jvp(c, qm, qp, dqm, dqp, 1.0, 0.0, out);
        for (int v = 0; v < V; ++v) dFR[v][k] = out[v];
        for (int v = 0; v < V; ++v) {
            qp[v] = own.qB[v][k]; dqp[v] = down.qB[v][k];
            qm[v] = eB >= 0 ? NB.qT[v][k] : own.qB[v][k];
            dqm[v] = eB >= 0 ? dNB.qT[v][k] : down.qB[v][k];
        }
        common_flux_jvp(c, qm, qp, dqm, dqp, 0.0, 1.0, out);
        for (int v = 0; v < V; ++v) dGB[v][k] = out[v];
        for (int v = 0; v < V; ++v) {
            qm[v] = own.qT[v][k]; dqm[v] = down.qT[v][k];
            qp[v] = eT >= 0 ? NT.qB[v][k] : own.qT[v][k];
            dqp[v] = eT >= 0 ? dNT.qB[v][k] : down.qT[v][k];
        }
        common_flux_jvp(c, qm, qp, dqm, dqp, 0.0, 1.0, out);
        for (int v = 0; v < V; ++v) dGT[v][k] = out[v];
    }
    for (int b = 0; b < n; ++b)
        for (int a = 0; a < n; ++a)
            for (int v = 0; v < V; ++v) {
                double sx = 0, sy = 0, fL = 0, fR = 0, gB = 0, gT = 0;
                for (int l = 0; l < n; ++l) {
                    sx += T->D[a][l] * dfpt[v][b][l];
                    sy += T->D[b][l] * dgpt[v][l][a];
                    fL += T->lm[l] * dfpt[v][b][l];
                    fR += T->lp[l] * dfpt[v][b][l];
                    gB += T->lm[l] * dgpt[v][l][a];
                    gT += T->lp[l] * dgpt[v][l][a];
                }
                double xs = sx + (dFL[v][b] - fL) * T->dgl[a] + (dFR[v][b] - fR) * T->dgr[a];
                double ys = sy + (dGB[v][a] - gB) * T->dgl[b] + (dGT[v][a] - gT) * T->dgr[b];
                QAT(dR, v, e, b, a) = -(2.0 / hx) * xs - (2.0 / hy) * ys;
            }
}

int oracle_residual_jvp(const oracle_cfg* c, const double* q, const double* dq, double* dR)
{
    if (check_cfg(c) || c->scheme != OR_CPR || c->div != OR_DIV_LP || c->flux == OR_ROE || !q || !dq || !dR) return -1;
    oracle_tab T;
    oracle_tables_corr(c->p, c->pts, c->corr, &T);
    long ne = (long)c->nx * c->ny;
#pragma omp parallel for schedule(static)
    for (long e = 0; e < ne; ++e)
        element_residual_jvp(c, &T, q, dq, (int)(e % c->nx), (int)(e / c->nx), dR);
    return 0;
}

/* qbar += (dR_e/dq)^T rbar_e for one element (serial: it scatters into the
 * neighbours' entries).  Each forward step above is transposed in reverse. */
static void element_residual_vjp(const oracle_cfg* c, const oracle_tab* T, const double* q,
                                 const double* rbar, int i, int j, double* qbar)
{
    int n = T->n, V = oracle_nvars(c);
    long ne = (long)c->nx * c->ny;
    long e = (long)j * c->nx + i;
    double hx = (c->x1 - c->x0) / c->nx, hy = (c->y1 - c->y0) / c->ny;
    long eL, eR, eB, eT;
    neighbours(c, i, j, &eL, &eR, &eB, &eT);
    edge_states own, NL, NR, NB, NT;
    element_edge_states(c, T, q, e, &own);
    if (eL >= 0) element_edge_states(c, T, q, eL, &NL);
    if (eR >= 0) element_edge_states(c, T, q, eR, &NR);
    if (eB >= 0) element_edge_states(c, T, q, eB, &NB);
    if (eT >= 0) element_edge_states(c, T, q, eT, &NT);

    /* R_ab = -(2/hx) xs_ab - (2/hy) ys_ab */
    double xsb[4][ORACLE_NMAX][ORACLE_NMAX], ysb[4][ORACLE_NMAX][ORACLE_NMAX];
    for (int v = 0; v < V; ++v)
        for (int b = 0; b < n; ++b)
            for (int a = 0; a < n; ++a) {
                xsb[v][b][a] = -(2.0 / hx) * QAT(rbar, v, e, b, a);
                ysb[v][b][a] = -(2.0 / hy) * QAT(rbar, v, e, b, a);
            }
    /* adjoints of the point fluxes, the edge fluxes and the common fluxes */
    double fb[4][ORACLE_NMAX][ORACLE_NMAX], gb[4][ORACLE_NMAX][ORACLE_NMAX];
    double FLb[4][ORACLE_NMAX], FRb[4][ORACLE_NMAX], GBb[4][ORACLE_NMAX], GTb[4][ORACLE_NMAX];
    memset(fb, 0, sizeof fb); memset(gb, 0, sizeof gb);
    memset(FLb, 0, sizeof FLb); memset(FRb, 0, sizeof FRb);
    memset(GBb, 0, sizeof GBb); memset(GTb, 0, sizeof GTb);
    for (int v = 0; v < V; ++v)
        for (int b = 0; b < n; ++b)
            for (int a = 0; a < n; ++a) {
                double xb = xsb[v][b][a], yb = ysb[v][b][a];
                /* xs = sum_l D_al f_lb + (FL_b - sum_l lm_l f_lb) gl_a + (FR_b - sum_l lp_l f_lb) gr_a */
                FLb[v][b] += xb * T->dgl[a];
                FRb[v][b] += xb * T->dgr[a];
                GBb[v][a] += yb * T->dgl[b];
                GTb[v][a] += yb * T->dgr[b];
                for (int l = 0; l < n; ++l) {
                    fb[v][b][l] += xb * (T->D[a][l] - T->lm[l] * T->dgl[a] - T->lp[l] * T->dgr[a]);
                    gb[v][l][a] += yb * (T->D[b][l] - T->lm[l] * T->dgl[b] - T->lp[l] * T->dgr[b]);
                }
            }
    /* point fluxes -> own q */
    for (int b = 0; b < n; ++b)
        for (int a = 0; a < n; ++a) {
            double qa[4], w[4], acc[4] = {0, 0, 0, 0};
            for (int v = 0; v < V; ++v) qa[v] = QAT(q, v, e, b, a);
            for (int v = 0; v < V; ++v) w[v] = fb[v][b][a];
            normal_flux_vjp(c, qa, w, 1.0, 0.0, acc);
            for (int v = 0; v < V; ++v) w[v] = gb[v][b][a];
            normal_flux_vjp(c, qa, w, 0.0, 1.0, acc);
            for (int v = 0; v < V; ++v) QAT(qbar, v, e, b, a) += acc[v];
        }
    /* common fluxes -> edge states of own element and neighbours; edge states
     * are linear in the point values: q_L,k = sum_l lm_l q_{l,k} etc. */
    for (int k = 0; k < n; ++k) {
        double qm[4], qp[4], w[4], bm[4], bp[4];
        /* left edge: qm = NL.qR (or own.qL), qp = own.qL */
        for (int v = 0; v < V; ++v) {
            qp[v] = own.qL[v][k];
            qm[v] = eL >= 0 ? NL.qR[v][k] : own.qL[v][k];
            w[v] = FLb[v][k]; bm[v] = 0; bp[v] = 0;
        }
        common_flux_vjp(c, qm, qp, w, 1.0, 0.0, bm, bp);
        for (int v = 0; v < V; ++v)
            for (int l = 0; l < n; ++l) {
                QAT(qbar, v, e, k, l) += T->lm[l] * bp[v];
                if (eL >= 0) QAT(qbar, v, eL, k, l) += T->lp[l] * bm[v];
                else QAT(qbar, v, e, k, l) += T->lm[l] * bm[v];
            }
        /* right edge: qm = own.qR, qp = NR.qL (or own.qR) */
        for (int v = 0; v < V; ++v) {
            qm[v] = own.qR[v][k];
            qp[v] = eR >= 0 ? NR.qL[v][k] : own.qR[v][k];
            w[v] = FRb[v][k]; bm[v] = 0; bp[v] = 0;
        }
        common_flux_vjp(c, qm, qp, w, 1.0, 0.0, bm, bp);
        for (int v = 0; v < V; ++v)
            for (int l = 0; l < n; ++l) {
                QAT(qbar, v, e, k, l) += T->lp[l] * bm[v];
                if (eR >= 0) QAT(qbar, v, eR, k, l) += T->lm[l] * bp[v];
                else QAT(qbar, v, e, k, l) += T->lp[l] * bp[v];
            }
        /* bottom edge: qm = NB.qT (or own.qB), qp = own.qB; column k */
        for (int v = 0; v < V; ++v) {
            qp[v] = own.qB[v][k];
            qm[v] = eB >= 0 ? NB.qT[v][k] : own.qB[v][k];
            w[v] = GBb[v][k]; bm[v] = 0; bp[v] = 0;
        }
        common_flux_vjp(c, qm, qp, w, 0.0, 1.0, bm, bp);
        for (int v = 0; v < V; ++v)
            for (int l = 0; l < n; ++l) {
                QAT(qbar, v, e, l, k) += T->lm[l] * bp[v];
                if (eB >= 0) QAT(qbar, v, eB, l, k) += T->lp[l] * bm[v];
                else QAT(qbar, v, e, l, k) += T->lm[l] * bm[v];
            }
        /* top edge: qm = own.qT, qp = NT.qB (or own.qT) */
        for (int v = 0; v < V; ++v) {
            qm[v] = own.qT[v][k];
            qp[v] = eT >= 0 ? NT.qB[v][k] : own.qT[v][k];
            w[v] = GTb[v][k]; bm[v] = 0; bp[v] = 0;
        }
        common_flux_vjp(c, qm, qp, w, 0.0, 1.0, bm, bp);
        for (int v = 0; v < V; ++v)
            for (int l = 0; l < n; ++l) {
                QAT(qbar, v, e, l, k) += T->lp[l] * bm[v];
                if (eT >= 0) QAT(qbar, v, eT, l, k) += T->lm[l] * bp[v];
                else QAT(qbar, v, e, l, k) += T->lp[l] * bp[v];
            }
    }
}

int oracle_residual_vjp(const oracle_cfg* c, const double* q, const double* rbar, double* qbar)
{
    if (check_cfg(c) || c->scheme != OR_CPR || c->div != OR_DIV_LP || c->flux == OR_ROE || !q || !rbar || !qbar) return -1;
    oracle_tab T;
    oracle_tables_corr(c->p, c->pts, c->corr, &T);
    long N = oracle_state_size(c);
    memset(qbar, 0, sizeof(double) * N);
    long ne = (long)c->nx * c->ny;
    for (long e = 0; e < ne; ++e)
        element_residual_vjp(c, &T, q, rbar, (int)(e % c->nx), (int)(e / c->nx), qbar);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Averages (Algorithm 9) and limiter (Sec. 2.6, Algorithms 10-11)          */
/* ------------------------------------------------------------------------ */

int oracle_averages(const oracle_cfg* c, const double* q, double* avg)
{
    if (check_cfg(c) || !q || !avg) return -1;
    if (c->scheme != OR_CPR) {
        /* FV stores the averages themselves */
        memcpy(avg, q, sizeof(double) * oracle_nvars(c) * c->nx * c->ny);
        return 0;
    }
    oracle_tab T;
    oracle_tables_corr(c->p, c->pts, c->corr, &T);
    int n = T.n, V = oracle_nvars(c);
    long ne = (long)c->nx * c->ny;
    for (int v = 0; v < V; ++v)
        for (long e = 0; e < ne; ++e) {
            /* Algorithm 9 reads as a running sum over the points (its "+=" is
             * lost in the text); c_m = w_a w_b / 4 is the quadrature weight of
             * the reference square, area 4. */
            double s = 0.0;
            for (int b = 0; b < n; ++b)
                for (int a = 0; a < n; ++a) s += (T.w[a] * T.w[b] * 0.25) * QAT(q, v, e, b, a);
            avg[(long)v * ne + e] = s;
        }
    return 0;
}

static double minmod3(double a, double b, double c)
{
    if (a > 0 && b > 0 && c > 0) return fmin(a, fmin(b, c));
    if (a < 0 && b < 0 && c < 0) return fmax(a, fmax(b, c));
    return 0.0;
}

static double minmod2(double a, double b)
{
    if (a > 0 && b > 0) return fmin(a, b);
    if (a < 0 && b < 0) return fmax(a, b);
    return 0.0;
}

/* TVB-modified minmod (Cockburn-Shu): keep the first argument when it is
 * already small, |a| <= M h^2. */
static double minmod_tvb(double a, double b, double c, double M, double h)
{
    if (fabs(a) <= M * h * h) return a;
    return minmod3(a, b, c);
}

long oracle_limit(const oracle_cfg* c, double* q, int* marks, double* margin)
{
    if (check_cfg(c) || c->scheme != OR_CPR || !q) return -1;
    oracle_tab T;
    oracle_tables_corr(c->p, c->pts, c->corr, &T);
    int n = T.n, V = oracle_nvars(c);
    long ne = (long)c->nx * c->ny;
    double hx = (c->x1 - c->x0) / c->nx, hy = (c->y1 - c->y0) / c->ny;
    double* avg = (double*)malloc(sizeof(double) * V * ne);
    int* mk = (int*)malloc(sizeof(int) * ne);
    if (!avg || !mk) { free(avg); free(mk); return -1; }
    oracle_averages(c, q, avg);

    /* Part 1: marking (Algorithm 10).  Reading of the garbled minmod line:
     * on an edge with outward sign s (+1 right/top, -1 left/bottom) the edge
     * deviation delta = s (q_edge - qbar_k) is compared with the forward and
     * backward differences of the averages in that direction; the element is
     * marked when |delta - mt(delta, D+, D-)| > eps for any variable and any
     * edge point.  Ghost averages at a transmissive edge equal the element's
     * own average (reading; the paper is silent on boundaries). */
    for (long e = 0; e < ne; ++e) {
        int i = (int)(e % c->nx), j = (int)(e / c->nx);
        long eL, eR, eB, eT;
        neighbours(c, i, j, &eL, &eR, &eB, &eT);
        edge_states E;
        element_edge_states(c, &T, q, e, &E);
        double worst = -INFINITY;
        for (int v = 0; v < V; ++v) {
            double qk = avg[(long)v * ne + e];
            double aL = eL >= 0 ? avg[(long)v * ne + eL] : qk;
            double aR = eR >= 0 ? avg[(long)v * ne + eR] : qk;
            double aB = eB >= 0 ? avg[(long)v * ne + eB] : qk;
            double aT = eT >= 0 ? avg[(long)v * ne + eT] : qk;
            double dxp = aR - qk, dxm = qk - aL, dyp = aT - qk, dym = qk - aB;
            for (int k = 0; k < n; ++k) {
                double d, dev;
                d = qk - E.qL[v][k];
                dev = fabs(d - minmod_tvb(d, dxp, dxm, c->tvb_M, hx)) - c->lim_eps;
                if (dev > worst) worst = dev;
                d = E.qR[v][k] - qk;
                dev = fabs(d - minmod_tvb(d, dxp, dxm, c->tvb_M, hx)) - c->lim_eps;
                if (dev > worst) worst = dev;
                d = qk - E.qB[v][k];
                dev = fabs(d - minmod_tvb(d, dyp, dym, c->tvb_M, hy)) - c->lim_eps;
                if (dev > worst) worst = dev;
                d = E.qT[v][k] - qk;
                dev = fabs(d - minmod_tvb(d, dyp, dym, c->tvb_M, hy)) - c->lim_eps;
                if (dev > worst) worst = dev;
            }
        }
        mk[e] = worst > 0.0;
        if (margin) margin[e] = worst;
        if (marks) marks[e] = mk[e];
    }

    /* Part 2: limiting of marked elements, Eq. 35 applied per direction:
     * q_ab = qbar + (x_a - x0) mm(D+x/hx, D-x/hx) + (y_b - y0) mm(D+y/hy, D-y/hy)
     * with x_a - x0 = xi_a hx / 2 (reading: the 1D formula extended to the
     * tensor-product element with independent x and y slopes). */
    long count = 0;
    for (long e = 0; e < ne; ++e) {
        if (!mk[e]) continue;
        ++count;
        int i = (int)(e % c->nx), j = (int)(e / c->nx);
        long eL, eR, eB, eT;
        neighbours(c, i, j, &eL, &eR, &eB, &eT);
        for (int v = 0; v < V; ++v) {
            double qk = avg[(long)v * ne + e];
            double aL = eL >= 0 ? avg[(long)v * ne + eL] : qk;
            double aR = eR >= 0 ? avg[(long)v * ne + eR] : qk;
            double aB = eB >= 0 ? avg[(long)v * ne + eB] : qk;
            double aT = eT >= 0 ? avg[(long)v * ne + eT] : qk;
            double sx = minmod2((aR - qk) / hx, (qk - aL) / hx);
            double sy = minmod2((aT - qk) / hy, (qk - aB) / hy);
            for (int b = 0; b < n; ++b)
                for (int a = 0; a < n; ++a)
                    QAT(q, v, e, b, a) = qk + (0.5 * hx * T.xi[a]) * sx + (0.5 * hy * T.xi[b]) * sy;
        }
    }
    free(avg);
    free(mk);
    return count;
}

/* ------------------------------------------------------------------------ */
/* Time integration, Sec. 4                                                 */
/* ------------------------------------------------------------------------ */

double oracle_max_wave(const oracle_cfg* c, const double* q)
{
    if (check_cfg(c) || !q) return -1.0;
    long npts = (long)c->nx * c->ny * (c->p + 1) * (c->p + 1);
    if (c->eqn == OR_ADVECTION) return sqrt(c->ax * c->ax + c->ay * c->ay);
    double m = 0.0;
    for (long k = 0; k < npts; ++k) {
        double qa[4] = {q[k], q[npts + k], q[2 * npts + k], q[3 * npts + k]};
        double u = qa[1] / qa[0], v = qa[2] / qa[0];
        double s = sqrt(u * u + v * v) + sqrt(c->gamma * pressure(c->gamma, qa) / qa[0]);
        if (s > m) m = s;
    }
    return m;
}

/* Eq. 36: dt <= CFL dx / (|u| + c); dx is the element size (reading), |u| the
 * speed, the maximum taken over all solution points. */
double oracle_dt(const oracle_cfg* c, const double* q)
{
    double hx = (c->x1 - c->x0) / c->nx, hy = (c->y1 - c->y0) / c->ny;
    double h = hx < hy ? hx : hy;
    return c->cfl * h / oracle_max_wave(c, q);
}

/* Three-stage SSP Runge-Kutta of Shu and Osher (the "three state" scheme of
 * Sec. 4):
 *   q1 = q + dt R(q)
 *   q2 = 3/4 q + 1/4 (q1 + dt R(q1))
 *   q  = 1/3 q + 2/3 (q2 + dt R(q2))
 * with the limiter applied to every stage result when enabled. */
int oracle_rk3_step(const oracle_cfg* c, double* q, double dt)
{
    if (check_cfg(c) || !q) return -1;
    long N = oracle_state_size(c);
    double* R = (double*)malloc(sizeof(double) * N);
    double* q1 = (double*)malloc(sizeof(double) * N);
    double* q2 = (double*)malloc(sizeof(double) * N);
    if (!R || !q1 || !q2) { free(R); free(q1); free(q2); return -1; }
    oracle_residual(c, q, R);
    for (long k = 0; k < N; ++k) q1[k] = q[k] + dt * R[k];
    if (c->limiter) oracle_limit(c, q1, NULL, NULL);
    oracle_residual(c, q1, R);
    for (long k = 0; k < N; ++k) q2[k] = 0.75 * q[k] + 0.25 * (q1[k] + dt * R[k]);
    if (c->limiter) oracle_limit(c, q2, NULL, NULL);
    oracle_residual(c, q2, R);
    for (long k = 0; k < N; ++k) q[k] = (1.0 / 3.0) * q[k] + (2.0 / 3.0) * (q2[k] + dt * R[k]);
    if (c->limiter) oracle_limit(c, q, NULL, NULL);
    free(R); free(q1); free(q2);
    return 0;
}

long oracle_run(const oracle_cfg* c, double* q, long nsteps, double dt, double t_end,
                double* t)
{
    long taken = 0;
    double tt = t ? *t : 0.0;
    for (long s = 0; s < nsteps; ++s) {
        /* Reading: with an end time, the step that would pass t_end is
         * shortened to t_end - t and the time is then set to t_end exactly;
         * no step is taken once t_end is reached (fixed or CFL steps). */
        if (t_end > 0.0 && tt >= t_end) break;
        double h = dt > 0.0 ? dt : oracle_dt(c, q);
        int last = 0;
        if (t_end > 0.0 && tt + h >= t_end) {
            h = t_end - tt;
            last = 1;
        }
        if (oracle_rk3_step(c, q, h)) return -1;
        tt = last ? t_end : tt + h;
        ++taken;
    }
    if (t) *t = tt;
    return taken;
}

/* Transpose of one SSP-RK3 step (no limiter), by recomputing the stages:
 *   qbar2  = 2/3 (qbar_out + dt J(q2)^T qbar_out)
 *   qbar1  = 1/4 (qbar2 + dt J(q1)^T qbar2)
 *   qbar_in = 1/3 qbar_out + 3/4 qbar2 + qbar1 + dt J(q)^T qbar1 */
int oracle_rk3_vjp(const oracle_cfg* c, const double* q, double dt, const double* qbar_out,
                   double* qbar_in)
{
    if (check_cfg(c) || c->scheme != OR_CPR || c->div != OR_DIV_LP || c->flux == OR_ROE || !q || !qbar_out || !qbar_in) return -1;
    long N = oracle_state_size(c);
    double* R = (double*)malloc(sizeof(double) * N);
    double* q1 = (double*)malloc(sizeof(double) * N);
    double* q2 = (double*)malloc(sizeof(double) * N);
    double* b1 = (double*)malloc(sizeof(double) * N);
    double* b2 = (double*)malloc(sizeof(double) * N);
    double* t = (double*)malloc(sizeof(double) * N);
    if (!R || !q1 || !q2 || !b1 || !b2 || !t) {
        free(R); free(q1); free(q2); free(b1); free(b2); free(t);
        return -1;
    }
    oracle_residual(c, q, R);
    for (long k = 0; k < N; ++k) q1[k] = q[k] + dt * R[k];
    oracle_residual(c, q1, R);
    for (long k = 0; k < N; ++k) q2[k] = 0.75 * q[k] + 0.25 * (q1[k] + dt * R[k]);

    oracle_residual_vjp(c, q2, qbar_out, t);
    for (long k = 0; k < N; ++k) b2[k] = (2.0 / 3.0) * (qbar_out[k] + dt * t[k]);
    oracle_residual_vjp(c, q1, b2, t);
    for (long k = 0; k < N; ++k) b1[k] = 0.25 * (b2[k] + dt * t[k]);
    oracle_residual_vjp(c, q, b1, t);
    for (long k = 0; k < N; ++k)
        qbar_in[k] = (1.0 / 3.0) * qbar_out[k] + 0.75 * b2[k] + b1[k] + dt * t[k];
    free(R); free(q1); free(q2); free(b1); free(b2); free(t);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Norms and errors                                                          */
/* ------------------------------------------------------------------------ */

int oracle_norms(const oracle_cfg* c, const double* q, const double* ref, oracle_norms_out* out)
{
    if (check_cfg(c) || !q || !out) return -1;
    memset(out, 0, sizeof(*out));
    int V = oracle_nvars(c);
    long ne = (long)c->nx * c->ny;
    long npts = ne * (c->p + 1) * (c->p + 1);
    double* avg = (double*)malloc(sizeof(double) * V * ne);
    if (!avg) return -1;
    oracle_averages(c, q, avg);
    for (int v = 0; v < V; ++v) {
        double s = 0.0;
        for (long e = 0; e < ne; ++e) s += avg[(long)v * ne + e];
        out->sum_avg[v] = s;
    }
    free(avg);
    if (ref) {
        double d2 = 0.0, r2 = 0.0;
        for (long k = 0; k < (long)V * npts; ++k) {
            double d = q[k] - ref[k];
            d2 += d * d;
            r2 += ref[k] * ref[k];
        }
        out->l2_abs = sqrt(d2);
        out->l2_rel = r2 > 0.0 ? sqrt(d2 / r2) : sqrt(d2);
    }
    long long bad = 0;
    for (long k = 0; k < npts; ++k) {
        int ok = 1;
        for (int v = 0; v < V; ++v)
            if (!isfinite(q[(long)v * npts + k])) ok = 0;
        if (ok && c->eqn == OR_EULER) {
            double qa[4] = {q[k], q[npts + k], q[2 * npts + k], q[3 * npts + k]};
            if (!(qa[0] > 0.0) || !(pressure(c->gamma, qa) > 0.0)) ok = 0;
        }
        if (!ok) ++bad;
    }
    out->n_nonphys = bad;
    out->max_wave = bad ? -1.0 : oracle_max_wave(c, q);
    return 0;
}

/* Isentropic vortex of Sec. 4.1 (Shu): mean (rho, u, v, p) = (1, uinf, vinf, 1),
 *   (du, dv) = eps/(2 pi) exp((1 - r^2)/2) (-ybar, xbar)
 *   dT = -(gamma - 1) eps^2 / (8 gamma pi^2) exp(1 - r^2),  dS = 0,
 * so T = 1 + dT, rho = T^(1/(gamma-1)), p = rho T = rho^gamma.  The exact
 * solution at time t is the initial field moved by (uinf t, vinf t); on the
 * periodic box the nearest image of the centre is used. */
static void vortex_exact(const oracle_cfg* c, const double* par, double t, double x,
                         double y, double* qv)
{
    double eps = par[0], xc = par[1], yc = par[2], ui = par[3], vi = par[4];
    double Lx = c->x1 - c->x0, Ly = c->y1 - c->y0;
    double xb = x - xc - ui * t, yb = y - yc - vi * t;
    xb -= Lx * floor(xb / Lx + 0.5);
    yb -= Ly * floor(yb / Ly + 0.5);
    double r2 = xb * xb + yb * yb;
    double g = c->gamma;
    double du = eps / (2.0 * PI) * exp(0.5 * (1.0 - r2)) * (-yb);
    double dv = eps / (2.0 * PI) * exp(0.5 * (1.0 - r2)) * xb;
    double T = 1.0 - (g - 1.0) * eps * eps / (8.0 * g * PI * PI) * exp(1.0 - r2);
    double rho = pow(T, 1.0 / (g - 1.0));
    double p = rho * T;
    double u = ui + du, v = vi + dv;
    qv[0] = rho;
    qv[1] = rho * u;
    qv[2] = rho * v;
    qv[3] = p / (g - 1.0) + 0.5 * rho * (u * u + v * v);
}

int oracle_exact_averages(const oracle_cfg* c, int kind, const double* par, double t,
                          double* avg)
{
    if (check_cfg(c) || !avg) return -1;
    double gx[10], gw[10];
    gauss_nodes(10, gx, gw);
    long ne = (long)c->nx * c->ny;
    double hx = (c->x1 - c->x0) / c->nx, hy = (c->y1 - c->y0) / c->ny;
    for (long e = 0; e < ne; ++e) {
        int i = (int)(e % c->nx), j = (int)(e / c->nx);
        double s[4] = {0, 0, 0, 0};
        for (int b = 0; b < 10; ++b)
            for (int a = 0; a < 10; ++a) {
                double x = c->x0 + hx * (i + 0.5 * (gx[a] + 1.0));
                double y = c->y0 + hy * (j + 0.5 * (gx[b] + 1.0));
                double wt = 0.25 * gw[a] * gw[b];
                if (kind == 0) {
                    s[0] += wt * sin(2.0 * PI * (x - c->ax * t)) * sin(2.0 * PI * (y - c->ay * t));
                } else {
                    double qv[4];
                    vortex_exact(c, par, t, x, y, qv);
                    for (int v = 0; v < 4; ++v) s[v] += wt * qv[v];
                }
            }
        int V = kind == 0 ? 1 : 4;
        for (int v = 0; v < V; ++v) avg[(long)v * ne + e] = s[v];
    }
    return 0;
}

double oracle_rho_avg_error(const oracle_cfg* c, const double* q, const double* exact_avg)
{
    int V = oracle_nvars(c);
    long ne = (long)c->nx * c->ny;
    double* avg = (double*)malloc(sizeof(double) * V * ne);
    if (!avg) return -1.0;
    oracle_averages(c, q, avg);
    double s = 0.0;
    for (long e = 0; e < ne; ++e) {
        double d = avg[e] - exact_avg[e];
        s += d * d;
    }
    free(avg);
    return sqrt(s / ne);
}
