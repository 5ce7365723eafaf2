// cpr_tables.cpp -- FP64 operator tables of the CPR scheme, built on the host.
//
//   nodes     Gauss-Legendre: roots of P_n; Gauss-Lobatto (the paper's CPR
//             points, Sec. 2.2 / Fig. 1b): roots of P_n - P_{n-2}, which are
//             +-1 and the roots of P'_{n-1}.
//   weights   Gauss: 2 (1 - x^2) / (n P_{n-1}(x))^2; Lobatto: 2 / (n (n-1) P_{n-1}(x)^2).
//   D         derivative of the Lagrange basis at the nodes, barycentric form
//             D_al = (lambda_l / lambda_a) / (xi_a - xi_l), D_aa = -sum_{l != a} D_al.
//   lm, lp    Lagrange basis at -1 and +1 (barycentric formula).
//   dgl, dgr  derivatives of the g_DG correction functions (Radau polynomials,
//             Sec. 2.2): g_L = (-1)^(p+1)/2 (P_{p+1} - P_p), g_R = (P_{p+1} + P_p)/2;
//             or the nodal-DG lift of Sec. 2.3 along a line, dgr = M^-1 l(+1),
//             dgl = -M^-1 l(-1), with the 1D mass matrix M_ij = int l_i l_j
//             (exact, by an (n+1)-point Gauss rule) or lumped (diag(w)).
#include <cmath>

#include "cpr_launch.h"

namespace cpr {
namespace {

// P_n(x) and P_{n-1}(x) by the three-term recurrence.
void legendre_pair(int n, double x, double* pn, double* pn1)
{
    double a = 1.0, b = x;  // P_0, P_1
    if (n == 0) {
        *pn = 1.0;
        *pn1 = 0.0;
        return;
    }
    for (int k = 2; k <= n; ++k) {
        const double c = ((2 * k - 1) * x * b - (k - 1) * a) / k;
        a = b;
        b = c;
    }
    *pn = b;
    *pn1 = a;
}

double legendre(int n, double x)
{
    double pn, pn1;
    legendre_pair(n, x, &pn, &pn1);
    return pn;
}

// P_n'(x): n (x P_n - P_{n-1}) / (x^2 - 1) inside, n (n+1)/2 (+-1)^(n+1) at the ends.
double legendre_deriv(int n, double x)
{
    if (n == 0) return 0.0;
    if (x == 1.0) return 0.5 * n * (n + 1);
    if (x == -1.0) return ((n % 2) ? 1.0 : -1.0) * 0.5 * n * (n + 1);
    double pn, pn1;
    legendre_pair(n, x, &pn, &pn1);
    return n * (x * pn - pn1) / (x * x - 1.0);
}

void gauss(int n, double* x, double* w)
{
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < n; ++i) {
        // ascending order: x_i ~ -cos(pi (4i + 3) / (4n + 2))
        double z = -std::cos(pi * (4.0 * i + 3.0) / (4.0 * n + 2.0));
        for (int it = 0; it < 60; ++it) {
            double pn, pn1;
            legendre_pair(n, z, &pn, &pn1);
            const double dp = n * (z * pn - pn1) / (z * z - 1.0);
            const double dz = pn / dp;
            z -= dz;
            if (std::fabs(dz) <= 1e-17) break;
        }
        double pn, pn1;
        legendre_pair(n, z, &pn, &pn1);
        x[i] = z;
        w[i] = 2.0 * (1.0 - z * z) / ((n * pn1) * (n * pn1));
    }
}

void lobatto(int n, double* x, double* w)
{
    const double pi = 3.14159265358979323846;
    const int p = n - 1;
    x[0] = -1.0;
    x[n - 1] = 1.0;
    for (int i = 1; i < n - 1; ++i) {
        double z = -std::cos(pi * i / p);
        for (int it = 0; it < 60; ++it) {
            // r = P_n - P_{n-2} = P_{p+1} - P_{p-1}; r' = (2p + 1) P_p
            const double r = legendre(p + 1, z) - legendre(p - 1, z);
            const double dr = (2.0 * p + 1.0) * legendre(p, z);
            const double dz = r / dr;
            z -= dz;
            if (std::fabs(dz) <= 1e-17) break;
        }
        x[i] = z;
    }
    for (int i = 0; i < n; ++i) {
        const double pp = legendre(p, x[i]);
        w[i] = 2.0 / (n * (n - 1.0) * pp * pp);
    }
}

// Lagrange basis polynomial l through the nodes xi, at x (product form).
double lagrange_at(int n, const double* xi, int l, double x)
{
    double r = 1.0;
    for (int m = 0; m < n; ++m)
        if (m != l) r *= (x - xi[m]) / (xi[l] - xi[m]);
    return r;
}

// x = M^-1 b for a small symmetric positive definite M (Cholesky).
bool spd_solve(int n, const double (*M)[kMaxN], const double* b, double* x)
{
    double L[kMaxN][kMaxN] = {};
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = M[i][j];
            for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
            if (i == j) {
                if (!(s > 0.0)) return false;
                L[i][i] = std::sqrt(s);
            } else {
                L[i][j] = s / L[j][j];
            }
        }
    }
    double y[kMaxN];
    for (int i = 0; i < n; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= L[i][k] * y[k];
        y[i] = s / L[i][i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = y[i];
        for (int k = i + 1; k < n; ++k) s -= L[k][i] * x[k];
        x[i] = s / L[i][i];
    }
    return true;
}

// Nodal-DG lift (Sec. 2.3): the strong form's L = M^-1 M^A reduces on a
// tensor-product element to M^-1 l(+-1) along each line; with the outward
// normal -1 on the left face the CPR form has dgl = -M^-1 l(-1).
bool ndg_lift(int n, bool lumped, HostTab* t)
{
    double M[kMaxN][kMaxN] = {};
    if (lumped) {
        for (int i = 0; i < n; ++i) M[i][i] = t->w[i];
    } else {
        double gx[kMaxN + 1], gw[kMaxN + 1];
        gauss(n + 1, gx, gw);
        for (int q = 0; q < n + 1; ++q) {
            double lq[kMaxN];
            for (int i = 0; i < n; ++i) lq[i] = lagrange_at(n, t->xi, i, gx[q]);
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j) M[i][j] += gw[q] * lq[i] * lq[j];
        }
    }
    double x[kMaxN];
    if (!spd_solve(n, M, t->lp, x)) return false;
    for (int a = 0; a < n; ++a) t->dgr[a] = x[a];
    if (!spd_solve(n, M, t->lm, x)) return false;
    for (int a = 0; a < n; ++a) t->dgl[a] = -x[a];
    return true;
}

}  // namespace

int build_tables(int p, int pts, int corr, HostTab* t)
{
    if (p == 0 && t) {
        // the one-point element of the FV scheme: the average itself at the
        // centre (weight 2 on [-1, 1]); no derivative, no correction
        *t = HostTab{};
        t->n = 1;
        t->w[0] = 2.0;
        t->lm[0] = t->lp[0] = 1.0;
        return 0;
    }
    if (p < 1 || p > kMaxN - 1 || !t) return -1;
    const int n = p + 1;
    *t = HostTab{};
    t->n = n;
    if (pts == 0) gauss(n, t->xi, t->w);
    else if (pts == 1) lobatto(n, t->xi, t->w);
    else return -1;

    double lam[kMaxN];
    for (int l = 0; l < n; ++l) {
        double prod = 1.0;
        for (int m = 0; m < n; ++m)
            if (m != l) prod *= t->xi[l] - t->xi[m];
        lam[l] = 1.0 / prod;
    }
    for (int a = 0; a < n; ++a) {
        double diag = 0.0;
        for (int l = 0; l < n; ++l) {
            if (l == a) continue;
            const double d = (lam[l] / lam[a]) / (t->xi[a] - t->xi[l]);
            t->D[a][l] = d;
            diag -= d;
        }
        t->D[a][a] = diag;
    }
    for (int side = 0; side < 2; ++side) {
        const double xe = side ? 1.0 : -1.0;
        double* out = side ? t->lp : t->lm;
        int hit = -1;
        for (int l = 0; l < n; ++l)
            if (t->xi[l] == xe) hit = l;
        if (hit >= 0) {
            for (int l = 0; l < n; ++l) out[l] = l == hit ? 1.0 : 0.0;
        } else {
            double den = 0.0;
            for (int l = 0; l < n; ++l) den += lam[l] / (xe - t->xi[l]);
            for (int l = 0; l < n; ++l) out[l] = (lam[l] / (xe - t->xi[l])) / den;
        }
    }
    const double s = (p % 2) ? 1.0 : -1.0;  // (-1)^(p+1)
    for (int a = 0; a < n; ++a) {
        const double d1 = legendre_deriv(p + 1, t->xi[a]);
        const double d0 = legendre_deriv(p, t->xi[a]);
        t->dgl[a] = 0.5 * s * (d1 - d0);
        t->dgr[a] = 0.5 * (d1 + d0);
    }
    if (corr == 1 || corr == 2) return ndg_lift(n, corr == 2, t) ? 0 : -1;
    return corr == 0 ? 0 : -1;
}

}  // namespace cpr
