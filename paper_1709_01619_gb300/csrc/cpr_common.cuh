// cpr_common.cuh -- device-side types and physics shared by the CPR kernels.
//
// Euler flux and equation of state: Sec. 2, Eqs. 3-5.  Rusanov common flux:
// Sec. 2.2 (Eq. 12 replaces the normal flux by a Riemann flux) and Sec. 4.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cpr {

constexpr int kMaxN = 5;      // p <= 4
constexpr int kAuxElems = 64; // elements per CTA in the element-wise passes

enum { EQ_ADV = 0, EQ_EULER = 1 };
enum { DIV_LP = 0, DIV_CHAIN = 1 };
enum { FLUX_RUSANOV = 0, FLUX_UPWIND = 1 };

template <int EQ>
struct NVars;
template <>
struct NVars<EQ_ADV> {
    static constexpr int value = 1;
};
template <>
struct NVars<EQ_EULER> {
    static constexpr int value = 4;
};

// 1D operator tables in the arithmetic type, passed by value as kernel
// parameters (constant bank): D[a][l] = l_l'(xi_a), edge interpolation
// lm[l] = l_l(-1), lp[l] = l_l(+1), correction derivatives g_L'(xi_a),
// g_R'(xi_a), quadrature weights and nodes, and the weights of the element
// average.
template <class T>
struct Tab {
    T D[kMaxN][kMaxN];
    T lm[kMaxN], lp[kMaxN];
    T dgl[kMaxN], dgr[kMaxN];
    T w[kMaxN], xi[kMaxN];
    T cavg[kMaxN][kMaxN];  // cavg[b][a] = w_a w_b / 4, average weights (Algorithm 9)
};

// Per-context device control block: simulated time and the step size of the
// step in flight.  Written only by the last CTA of the stage-3 (or wave)
// kernel, after every other CTA of that kernel has finished reading it.
struct Ctrl {
    double t;          // simulated time
    double dt;         // step size of the current step
    double t_end;      // <= 0: no end time
    double dt_fixed;   // > 0: fixed step size
    double cfl_h;      // cfl * min(hx, hy)
    double max_wave;   // last reduced max speed
    long long steps;   // steps taken
    long long marked;  // elements marked by the last limiter pass
    unsigned int counter;  // CTA completion ticket for the last-CTA reduction
    int done;          // 1: t reached t_end, stage kernels do no work
    int last;          // 1: the step in flight was shortened to land on t_end
    int pad;
};

// Physics in the arithmetic type T.
template <class T>
struct Phys {
    T gamma;  // Euler
    T ax, ay; // advection
};

__device__ __forceinline__ float dsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double dsqrt(double x) { return sqrt(x); }

// Pressure, Eq. 5: p = (gamma - 1)(e - (rho u u + rho v v)/2) with u = rho u / rho.
template <class T>
__device__ __forceinline__ T pressure(const T* q, T gamma, T& u, T& v)
{
    T r = T(1) / q[0];
    u = q[1] * r;
    v = q[2] * r;
    return (gamma - T(1)) * (q[3] - T(0.5) * (q[1] * u + q[2] * v));
}

// x-flux f(q) and y-flux g(q) of Eq. 4.
template <int EQ, class T>
__device__ __forceinline__ void flux_x(const T* q, const Phys<T>& ph, T* f)
{
    if constexpr (EQ == EQ_ADV) {
        f[0] = ph.ax * q[0];
    } else {
        T u, v;
        T p = pressure(q, ph.gamma, u, v);
        f[0] = q[1];
        f[1] = q[1] * u + p;
        f[2] = q[2] * u;
        f[3] = (q[3] + p) * u;
    }
}

template <int EQ, class T>
__device__ __forceinline__ void flux_y(const T* q, const Phys<T>& ph, T* g)
{
    if constexpr (EQ == EQ_ADV) {
        g[0] = ph.ay * q[0];
    } else {
        T u, v;
        T p = pressure(q, ph.gamma, u, v);
        g[0] = q[2];
        g[1] = q[1] * v;
        g[2] = q[2] * v + p;
        g[3] = (q[3] + p) * v;
    }
}

// Directional derivative of the x- or y-flux, A(q) dq (the chain-rule
// divergence of Sec. 2.2).  DIR 0: x, 1: y.
template <int EQ, int DIR, class T>
__device__ __forceinline__ void flux_jvp(const T* q, const T* dq, const Phys<T>& ph, T* df)
{
    if constexpr (EQ == EQ_ADV) {
        df[0] = (DIR == 0 ? ph.ax : ph.ay) * dq[0];
    } else {
        T u, v;
        T p = pressure(q, ph.gamma, u, v);
        T r = T(1) / q[0];
        T vn = DIR == 0 ? u : v;
        T dvn = ((DIR == 0 ? dq[1] : dq[2]) - vn * dq[0]) * r;
        T dp = (ph.gamma - T(1)) * (dq[3] - (u * dq[1] + v * dq[2]) + T(0.5) * (u * u + v * v) * dq[0]);
        df[0] = DIR == 0 ? dq[1] : dq[2];
        df[1] = dq[1] * vn + q[1] * dvn + (DIR == 0 ? dp : T(0));
        df[2] = dq[2] * vn + q[2] * dvn + (DIR == 1 ? dp : T(0));
        df[3] = (dq[3] + dp) * vn + (q[3] + p) * dvn;
    }
}

// Common flux through an x-face (DIR 0, normal +x) or y-face (DIR 1, normal
// +y) between qm (left/bottom) and qp (right/top).
// Rusanov: F = (F(qm) + F(qp))/2 - lambda (qp - qm)/2 with lambda the larger
// one-sided speed |Vn| + c.  Upwind (advection): F = a_n q_upwind.
template <int EQ, int FLUX, int DIR, class T>
__device__ __forceinline__ void common_flux(const T* qm, const T* qp, const Phys<T>& ph, T* F)
{
    if constexpr (EQ == EQ_ADV) {
        T an = DIR == 0 ? ph.ax : ph.ay;
        if constexpr (FLUX == FLUX_UPWIND) {
            F[0] = an >= T(0) ? an * qm[0] : an * qp[0];
        } else {
            T lam = an >= T(0) ? an : -an;
            F[0] = T(0.5) * (an * qm[0] + an * qp[0]) - T(0.5) * lam * (qp[0] - qm[0]);
        }
    } else {
        T um, vm, up, vp;
        T pm = pressure(qm, ph.gamma, um, vm);
        T pp = pressure(qp, ph.gamma, up, vp);
        T vnm = DIR == 0 ? um : vm;
        T vnp = DIR == 0 ? up : vp;
        T sm = (vnm >= T(0) ? vnm : -vnm) + dsqrt(ph.gamma * pm / qm[0]);
        T sp = (vnp >= T(0) ? vnp : -vnp) + dsqrt(ph.gamma * pp / qp[0]);
        T lam = sm >= sp ? sm : sp;
        T Fm[4], Fp[4];
        Fm[0] = qm[0] * vnm;
        Fp[0] = qp[0] * vnp;
        Fm[1] = qm[1] * vnm + (DIR == 0 ? pm : T(0));
        Fp[1] = qp[1] * vnp + (DIR == 0 ? pp : T(0));
        Fm[2] = qm[2] * vnm + (DIR == 1 ? pm : T(0));
        Fp[2] = qp[2] * vnp + (DIR == 1 ? pp : T(0));
        Fm[3] = (qm[3] + pm) * vnm;
        Fp[3] = (qp[3] + pp) * vnp;
#pragma unroll
        for (int k = 0; k < 4; ++k) F[k] = T(0.5) * (Fm[k] + Fp[k]) - T(0.5) * lam * (qp[k] - qm[k]);
    }
}

// Largest signal speed sqrt(u^2 + v^2) + c at one point (Eq. 36).
template <int EQ, class T>
__device__ __forceinline__ T point_speed(const T* q, const Phys<T>& ph)
{
    if constexpr (EQ == EQ_ADV) {
        return dsqrt(ph.ax * ph.ax + ph.ay * ph.ay);
    } else {
        T u, v;
        T p = pressure(q, ph.gamma, u, v);
        return dsqrt(u * u + v * v) + dsqrt(ph.gamma * p / q[0]);
    }
}

// Point is physical: finite values, rho > 0, p > 0 (Euler).
template <int EQ, class T>
__device__ __forceinline__ bool point_ok(const T* q, const Phys<T>& ph)
{
    constexpr int V = NVars<EQ>::value;
    bool ok = true;
#pragma unroll
    for (int v = 0; v < V; ++v) ok = ok && isfinite(q[v]);
    if constexpr (EQ == EQ_EULER) {
        if (ok) {
            T u, vv;
            ok = q[0] > T(0) && pressure(q, ph.gamma, u, vv) > T(0);
        }
    }
    return ok;
}

// Minmod functions of the limiter (Sec. 2.6).
template <class T>
__device__ __forceinline__ T minmod2(T a, T b)
{
    if (a > T(0) && b > T(0)) return a < b ? a : b;
    if (a < T(0) && b < T(0)) return a > b ? a : b;
    return T(0);
}

template <class T>
__device__ __forceinline__ T minmod3(T a, T b, T c)
{
    if (a > T(0) && b > T(0) && c > T(0)) return ::fmin(a, ::fmin(b, c));
    if (a < T(0) && b < T(0) && c < T(0)) return ::fmax(a, ::fmax(b, c));
    return T(0);
}

}  // namespace cpr
