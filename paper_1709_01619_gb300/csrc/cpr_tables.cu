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
//             Sec. 2.2): g_L = (-1)^(p+1)/2 (P_{p+1} - P_p), g_R = (P_{p+1} + P_p)/2.
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

}  // namespace

int build_tables(int p, int pts, HostTab* t)
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
    return 0;
}

}  // namespace cpr
