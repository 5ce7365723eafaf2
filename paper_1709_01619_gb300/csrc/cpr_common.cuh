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
enum { FLUX_RUSANOV = 0, FLUX_UPWIND = 1, FLUX_ROE = 2 };

// What a stage-kernel launch computes (see cpr_stage.cuh).
enum {
    MODE_RESIDUAL = 0,
    MODE_SO1 = 1, MODE_SO2 = 2, MODE_SO3 = 3,        // Shu-Osher stages
    MODE_INC1 = 4, MODE_INC2 = 5, MODE_INC3 = 6      // increment stages
};

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
    int parity;        // steps completed in the current cpr_step call, mod 2
    unsigned long long wmax;  // running maximum speed of the kernel in flight (bits of a
                              // non-negative double); 0 between kernels
};

// Physics in the arithmetic type T.
template <class T>
struct Phys {
    T gamma;  // Euler
    T ax, ay; // advection
};

// Reciprocal and square root in the FP32 physics (1/rho, sound speed): the
// hardware approximations (a few ulp), at the level of the rounding of the
// flux itself.  FP64 keeps IEEE operations.
__device__ __forceinline__ float frcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double frcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float fsqrt(float x)
{
    // 0 -> 0, negative -> NaN, otherwise x / sqrt(x) from the approximate rsqrt
    return x >= 0.0f ? x * rsqrtf(fmaxf(x, 1.17549435e-38f)) : __int_as_float(0x7fffffff);
}
__device__ __forceinline__ double fsqrt(double x) { return sqrt(x); }

// Pressure, Eq. 5: p = (gamma - 1)(e - (rho u u + rho v v)/2) with u = rho u / rho.
// Also returns r = 1 / rho.
template <class T>
__device__ __forceinline__ T pressure(const T* q, T gamma, T& u, T& v, T& r)
{
    r = frcp(q[0]);
    u = q[1] * r;
    v = q[2] * r;
    return (gamma - T(1)) * (q[3] - T(0.5) * (q[1] * u + q[2] * v));
}
template <class T>
__device__ __forceinline__ T pressure(const T* q, T gamma, T& u, T& v)
{
    T r;
    return pressure(q, gamma, u, v, r);
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
        T u, v, r;
        T p = pressure(q, ph.gamma, u, v, r);
        T vn = DIR == 0 ? u : v;
        T dvn = ((DIR == 0 ? dq[1] : dq[2]) - vn * dq[0]) * r;
        T dp = (ph.gamma - T(1)) * (dq[3] - (u * dq[1] + v * dq[2]) + T(0.5) * (u * u + v * v) * dq[0]);
        df[0] = DIR == 0 ? dq[1] : dq[2];
        df[1] = dq[1] * vn + q[1] * dvn + (DIR == 0 ? dp : T(0));
        df[2] = dq[2] * vn + q[2] * dvn + (DIR == 1 ? dp : T(0));
        df[3] = (dq[3] + dp) * vn + (q[3] + p) * dvn;
    }
}

// |lambda| of an acoustic field with the Harten-Hyman entropy fix: lam_m,
// lam_p are the field's speeds at the two states; only across a transonic
// rarefaction (delta > 0) is |lambda| < delta smoothed.
template <class T>
__device__ __forceinline__ T roe_abs(T lam, T lam_m, T lam_p)
{
    T d = T(0);
    d = lam - lam_m > d ? lam - lam_m : d;
    d = lam_p - lam > d ? lam_p - lam : d;
    const T a = lam >= T(0) ? lam : -lam;
    return a < d ? (lam * lam + d * d) * frcp(T(2) * d) : a;
}

// Roe's flux for the Euler equations through an x-face (DIR 0) or y-face
// (DIR 1): (f(qm) + f(qp))/2 - (1/2) sum_k |lambda_k| alpha_k r_k over the
// acoustic, entropy and shear fields of the Roe-averaged state (density
// sqrt(rho_m rho_p); velocity and total enthalpy averaged with weights
// sqrt(rho)), with the Harten-Hyman fix on the acoustic fields.
template <int DIR, class T>
__device__ __forceinline__ void roe_flux(const T* qm, const T* qp, const Phys<T>& ph, T* F)
{
    const T g = ph.gamma;
    T um, vm, rm, up, vp, rp;
    const T pm = pressure(qm, g, um, vm, rm), pp = pressure(qp, g, up, vp, rp);
    const T vnm = DIR == 0 ? um : vm, vnp = DIR == 0 ? up : vp;
    T Fm[4], Fp[4];
    Fm[0] = qm[0] * vnm;
    Fp[0] = qp[0] * vnp;
    Fm[1] = qm[1] * vnm + (DIR == 0 ? pm : T(0));
    Fp[1] = qp[1] * vnp + (DIR == 0 ? pp : T(0));
    Fm[2] = qm[2] * vnm + (DIR == 1 ? pm : T(0));
    Fp[2] = qp[2] * vnp + (DIR == 1 ? pp : T(0));
    Fm[3] = (qm[3] + pm) * vnm;
    Fp[3] = (qp[3] + pp) * vnp;
    const T Hm = (qm[3] + pm) * rm, Hp = (qp[3] + pp) * rp;
    const T wm = fsqrt(qm[0]), wp = fsqrt(qp[0]), iw = frcp(wm + wp);
    const T rho = wm * wp;
    const T u = (wm * um + wp * up) * iw, v = (wm * vm + wp * vp) * iw, H = (wm * Hm + wp * Hp) * iw;
    const T c2 = (g - T(1)) * (H - T(0.5) * (u * u + v * v));
    const T cs = fsqrt(c2), ic2 = frcp(c2);
    const T vn = DIR == 0 ? u : v;
    const T vt = DIR == 0 ? v : -u;  // along t = (-n_y, n_x)
    const T dvn = vnp - vnm;
    const T dvt = DIR == 0 ? vp - vm : um - up;
    const T dp = pp - pm;
    const T a1 = (dp - rho * cs * dvn) * T(0.5) * ic2;
    const T a2 = (qp[0] - qm[0]) - dp * ic2;
    const T a3 = rho * dvt;
    const T a4 = (dp + rho * cs * dvn) * T(0.5) * ic2;
    const T cm = fsqrt(g * pm * rm), cp = fsqrt(g * pp * rp);
    const T l1 = roe_abs(vn - cs, vnm - cm, vnp - cp);
    const T l2 = vn >= T(0) ? vn : -vn;
    const T l4 = roe_abs(vn + cs, vnm + cm, vnp + cp);
    const T nx = DIR == 0 ? T(1) : T(0), ny = DIR == 0 ? T(0) : T(1);
    const T r1[4] = {T(1), u - cs * nx, v - cs * ny, H - vn * cs};
    const T r2[4] = {T(1), u, v, T(0.5) * (u * u + v * v)};
    const T r3[4] = {T(0), -ny, nx, vt};
    const T r4[4] = {T(1), u + cs * nx, v + cs * ny, H + vn * cs};
#pragma unroll
    for (int k = 0; k < 4; ++k)
        F[k] = T(0.5) * (Fm[k] + Fp[k]) -
               T(0.5) * (l1 * a1 * r1[k] + l2 * a2 * r2[k] + l2 * a3 * r3[k] + l4 * a4 * r4[k]);
}

// Common flux through an x-face (DIR 0, normal +x) or y-face (DIR 1, normal
// +y) between qm (left/bottom) and qp (right/top).
// Rusanov: F = (F(qm) + F(qp))/2 - lambda (qp - qm)/2 with lambda the larger
// one-sided speed |Vn| + c.  Upwind (advection; also Roe's flux there):
// F = a_n q_upwind.  Roe (Euler): roe_flux.
template <int EQ, int FLUX, int DIR, class T>
__device__ __forceinline__ void common_flux(const T* qm, const T* qp, const Phys<T>& ph, T* F)
{
    if constexpr (EQ == EQ_EULER && FLUX == FLUX_ROE) {
        roe_flux<DIR>(qm, qp, ph, F);
        return;
    }
    if constexpr (EQ == EQ_ADV) {
        T an = DIR == 0 ? ph.ax : ph.ay;
        if constexpr (FLUX == FLUX_UPWIND || FLUX == FLUX_ROE) {
            F[0] = an >= T(0) ? an * qm[0] : an * qp[0];
        } else {
            T lam = an >= T(0) ? an : -an;
            F[0] = T(0.5) * (an * qm[0] + an * qp[0]) - T(0.5) * lam * (qp[0] - qm[0]);
        }
    } else {
        T um, vm, up, vp, rm, rp;
        T pm = pressure(qm, ph.gamma, um, vm, rm);
        T pp = pressure(qp, ph.gamma, up, vp, rp);
        T vnm = DIR == 0 ? um : vm;
        T vnp = DIR == 0 ? up : vp;
        T sm = (vnm >= T(0) ? vnm : -vnm) + fsqrt(ph.gamma * pm * rm);
        T sp = (vnp >= T(0) ? vnp : -vnp) + fsqrt(ph.gamma * pp * rp);
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
        return fsqrt(ph.ax * ph.ax + ph.ay * ph.ay);
    } else {
        T u, v, r;
        T p = pressure(q, ph.gamma, u, v, r);
        return fsqrt(u * u + v * v) + fsqrt(ph.gamma * p * r);
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

// Reference state of an element for the delta form: the conserved values
// and the derived velocity, pressure and total enthalpy e + p.
template <class T>
struct Ref {
    T q[4];
    T u, v, p, H;
};

template <int EQ, class T>
__device__ __forceinline__ Ref<T> make_ref(const T* q, const Phys<T>& ph)
{
    Ref<T> r;
    constexpr int V = NVars<EQ>::value;
#pragma unroll
    for (int k = 0; k < 4; ++k) r.q[k] = k < V ? q[k] : T(0);
    if constexpr (EQ == EQ_EULER) {
        r.p = pressure(q, ph.gamma, r.u, r.v);
        r.H = q[3] + r.p;
    } else {
        r.u = r.v = r.p = r.H = T(0);
    }
    return r;
}

// Flux difference f_DIR(ref + d) - f_DIR(ref) written with differences only
// (exact algebra; every term is O(d)):
//   du = (dm - u0 drho) / rho1,  d(m u) = dm u0 + m1 du,
//   dp = (gamma - 1)(de - (d(m u) + d(n v)) / 2),
//   d((e + p) u) = (de + dp) u0 + (H0 + de + dp) du,  and likewise in y.
// Also returns the signal speed |Vn| + c of the state ref + d (speed).
template <int EQ, int DIR, class T>
__device__ __forceinline__ void dflux_speed(const Ref<T>& r, const T* d, const Phys<T>& ph, T* out, T& speed)
{
    if constexpr (EQ == EQ_ADV) {
        const T an = DIR == 0 ? ph.ax : ph.ay;
        out[0] = an * d[0];
        speed = an >= T(0) ? an : -an;
    } else {
        const T inv = frcp(r.q[0] + d[0]);
        const T du = (d[1] - r.u * d[0]) * inv;
        const T dv = (d[2] - r.v * d[0]) * inv;
        const T m1 = r.q[1] + d[1], n1 = r.q[2] + d[2];
        const T dmu = d[1] * r.u + m1 * du;
        const T dnv = d[2] * r.v + n1 * dv;
        const T dp = (ph.gamma - T(1)) * (d[3] - T(0.5) * (dmu + dnv));
        const T dH = d[3] + dp;
        const T dvn = DIR == 0 ? du : dv;
        const T vn0 = DIR == 0 ? r.u : r.v;
        if (DIR == 0) {
            out[0] = d[1];
            out[1] = dmu + dp;
            out[2] = d[2] * r.u + n1 * du;
        } else {
            out[0] = d[2];
            out[1] = d[1] * r.v + m1 * dv;
            out[2] = dnv + dp;
        }
        out[3] = dH * vn0 + (r.H + dH) * dvn;
        const T vn1 = vn0 + dvn;
        speed = (vn1 >= T(0) ? vn1 : -vn1) + fsqrt(ph.gamma * (r.p + dp) * inv);
    }
}

template <int EQ, int DIR, class T>
__device__ __forceinline__ void dflux(const Ref<T>& r, const T* d, const Phys<T>& ph, T* out)
{
    T s;
    dflux_speed<EQ, DIR>(r, d, ph, out, s);
}

// Common flux relative to the reference: G = F*(ref + dm, ref + dp) - f(ref),
// Rusanov (lambda = larger one-sided speed) or upwind (advection).
template <int EQ, int FLUX, int DIR, class T>
__device__ __forceinline__ void common_flux_delta(const Ref<T>& r, const T* dm, const T* dp, const Phys<T>& ph,
                                                  T* G)
{
    if constexpr (EQ == EQ_EULER && FLUX == FLUX_ROE) {
        // no difference form of Roe's flux: the flux of the full states,
        // shifted to the reference
        T qm[4], qp[4], F[4], f0[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            qm[k] = r.q[k] + dm[k];
            qp[k] = r.q[k] + dp[k];
        }
        roe_flux<DIR>(qm, qp, ph, F);
        if constexpr (DIR == 0) flux_x<EQ>(r.q, ph, f0);
        else flux_y<EQ>(r.q, ph, f0);
#pragma unroll
        for (int k = 0; k < 4; ++k) G[k] = F[k] - f0[k];
        return;
    }
    if constexpr (EQ == EQ_ADV) {
        const T an = DIR == 0 ? ph.ax : ph.ay;
        if constexpr (FLUX == FLUX_UPWIND || FLUX == FLUX_ROE) {
            G[0] = an >= T(0) ? an * dm[0] : an * dp[0];
        } else {
            const T lam = an >= T(0) ? an : -an;
            G[0] = T(0.5) * (an * dm[0] + an * dp[0]) - T(0.5) * lam * (dp[0] - dm[0]);
        }
    } else {
        T Fm[4], Fp[4], sm, sp;
        dflux_speed<EQ, DIR>(r, dm, ph, Fm, sm);
        dflux_speed<EQ, DIR>(r, dp, ph, Fp, sp);
        const T lam = sm >= sp ? sm : sp;
#pragma unroll
        for (int k = 0; k < 4; ++k) G[k] = T(0.5) * (Fm[k] + Fp[k]) - T(0.5) * lam * (dp[k] - dm[k]);
    }
}

// ---- transposed linearisations (discrete adjoint) --------------------------

// qbar += (dF_DIR/dq)^T w at state q (F_DIR the x- or y-flux of Eq. 4).
template <int EQ, int DIR, class T>
__device__ __forceinline__ void flux_vjp(const T* q, const T* w, const Phys<T>& ph, T* qbar)
{
    if constexpr (EQ == EQ_ADV) {
        qbar[0] += (DIR == 0 ? ph.ax : ph.ay) * w[0];
    } else {
        const T g1 = ph.gamma - T(1);
        const T r = q[0], ir = frcp(r);
        const T u = q[1] * ir, v = q[2] * ir;
        const T p = g1 * (q[3] - T(0.5) * (q[1] * u + q[2] * v));
        const T vn = DIR == 0 ? u : v;
        const T nx = DIR == 0 ? T(1) : T(0), ny = DIR == 0 ? T(0) : T(1);
        const T dvn[4] = {-vn * ir, nx * ir, ny * ir, T(0)};
        const T dpq[4] = {g1 * T(0.5) * (u * u + v * v), -g1 * u, -g1 * v, g1};
        const T C = w[1] * q[1] + w[2] * q[2] + w[3] * (q[3] + p);
        const T Pc = w[1] * nx + w[2] * ny + w[3] * vn;
        qbar[0] += C * dvn[0] + Pc * dpq[0];
        qbar[1] += w[0] * nx + vn * w[1] + C * dvn[1] + Pc * dpq[1];
        qbar[2] += w[0] * ny + vn * w[2] + C * dvn[2] + Pc * dpq[2];
        qbar[3] += vn * w[3] + Pc * dpq[3];
    }
}

// Gradient of the signal speed |Vn| + c (Euler).
template <int DIR, class T>
__device__ __forceinline__ void speed_grad(const T* q, const Phys<T>& ph, T* gs)
{
    const T g1 = ph.gamma - T(1);
    const T r = q[0], ir = frcp(r);
    const T u = q[1] * ir, v = q[2] * ir;
    const T p = g1 * (q[3] - T(0.5) * (q[1] * u + q[2] * v));
    const T cs = fsqrt(ph.gamma * p * ir);
    const T vn = DIR == 0 ? u : v;
    const T sg = vn >= T(0) ? T(1) : T(-1);
    const T nx = DIR == 0 ? T(1) : T(0), ny = DIR == 0 ? T(0) : T(1);
    const T dvn[4] = {-vn * ir, nx * ir, ny * ir, T(0)};
    const T dpq[4] = {g1 * T(0.5) * (u * u + v * v), -g1 * u, -g1 * v, g1};
    const T k = ph.gamma * frcp(T(2) * cs * r);
#pragma unroll
    for (int m = 0; m < 4; ++m) gs[m] = sg * dvn[m] + k * (dpq[m] - (m == 0 ? p * ir : T(0)));
}

// Transpose of the common flux (Rusanov with lambda the larger one-sided
// speed, differentiated on the branch the forward takes; or upwind):
// qbm, qbp = cotangents of the lower and upper states for cotangent w.
template <int EQ, int FLUX, int DIR, class T>
__device__ __forceinline__ void common_flux_vjp(const T* qm, const T* qp, const T* w, const Phys<T>& ph, T* qbm,
                                                T* qbp)
{
    if constexpr (EQ == EQ_ADV) {
        const T an = DIR == 0 ? ph.ax : ph.ay;
        if constexpr (FLUX == FLUX_UPWIND) {
            qbm[0] = an >= T(0) ? an * w[0] : T(0);
            qbp[0] = an >= T(0) ? T(0) : an * w[0];
        } else {
            const T lam = an >= T(0) ? an : -an;
            qbm[0] = T(0.5) * an * w[0] + T(0.5) * lam * w[0];
            qbp[0] = T(0.5) * an * w[0] - T(0.5) * lam * w[0];
        }
    } else {
        T hw[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            hw[k] = T(0.5) * w[k];
            qbm[k] = T(0);
            qbp[k] = T(0);
        }
        flux_vjp<EQ, DIR>(qm, hw, ph, qbm);
        flux_vjp<EQ, DIR>(qp, hw, ph, qbp);
        T um, vm, up, vp, rm, rp;
        const T pm = pressure(qm, ph.gamma, um, vm, rm);
        const T pp = pressure(qp, ph.gamma, up, vp, rp);
        const T vnm = DIR == 0 ? um : vm, vnp = DIR == 0 ? up : vp;
        const T sm = (vnm >= T(0) ? vnm : -vnm) + fsqrt(ph.gamma * pm * rm);
        const T sp = (vnp >= T(0) ? vnp : -vnp) + fsqrt(ph.gamma * pp * rp);
        const T lam = sm >= sp ? sm : sp;
        T jump = T(0);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            qbm[k] += T(0.5) * lam * w[k];
            qbp[k] -= T(0.5) * lam * w[k];
            jump += w[k] * (qp[k] - qm[k]);
        }
        T gs[4];
        if (sm >= sp) {
            speed_grad<DIR>(qm, ph, gs);
#pragma unroll
            for (int k = 0; k < 4; ++k) qbm[k] -= T(0.5) * jump * gs[k];
        } else {
            speed_grad<DIR>(qp, ph, gs);
#pragma unroll
            for (int k = 0; k < 4; ++k) qbp[k] -= T(0.5) * jump * gs[k];
        }
    }
}

// Two-argument minmod of the limiter and of the MUSCL slopes (Sec. 2.6).
template <class T>
__device__ __forceinline__ T minmod2(T a, T b)
{
    if (a > T(0) && b > T(0)) return a < b ? a : b;
    if (a < T(0) && b < T(0)) return a > b ? a : b;
    return T(0);
}

// ---- two-lane arithmetic ----------------------------------------------------
// Pr<T> holds one value of two solution points of a line.  In FP32 the
// operations map onto Blackwell's packed FFMA2 / FMUL2 / FADD2 instructions
// (two IEEE single-precision operations, each rounded as its scalar
// counterpart, in one issue slot); in FP64 they are two scalar operations.
template <class T>
struct Pr;
template <>
struct alignas(8) Pr<float> {
    float2 v;
};
template <>
struct alignas(16) Pr<double> {
    double2 v;
};

__device__ __forceinline__ Pr<float> pmk(float a, float b) { return {make_float2(a, b)}; }
__device__ __forceinline__ Pr<double> pmk(double a, double b) { return {make_double2(a, b)}; }
template <class T>
__device__ __forceinline__ Pr<T> pbc(T a) { return pmk(a, a); }

__device__ __forceinline__ Pr<float> pfma(Pr<float> a, Pr<float> b, Pr<float> c) { return {__ffma2_rn(a.v, b.v, c.v)}; }
__device__ __forceinline__ Pr<float> pmul(Pr<float> a, Pr<float> b) { return {__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ Pr<float> padd(Pr<float> a, Pr<float> b) { return {__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ Pr<double> pfma(Pr<double> a, Pr<double> b, Pr<double> c)
{
    return {make_double2(fma(a.v.x, b.v.x, c.v.x), fma(a.v.y, b.v.y, c.v.y))};
}
__device__ __forceinline__ Pr<double> pmul(Pr<double> a, Pr<double> b)
{
    return {make_double2(a.v.x * b.v.x, a.v.y * b.v.y)};
}
__device__ __forceinline__ Pr<double> padd(Pr<double> a, Pr<double> b)
{
    return {make_double2(a.v.x + b.v.x, a.v.y + b.v.y)};
}
// a - b, exact as b * (-1) + a
template <class T>
__device__ __forceinline__ Pr<T> psub(Pr<T> a, Pr<T> b) { return pfma(b, pbc(T(-1)), a); }
template <class T>
__device__ __forceinline__ Pr<T> prcp(Pr<T> a) { return pmk(frcp(a.v.x), frcp(a.v.y)); }

// Euler flux f (DIR 0) or g (DIR 1) of Eq. 4 at two points; q, f: V pairs.
template <int EQ, int DIR, class T>
__device__ __forceinline__ void flux_pair(const Pr<T>* q, const Phys<T>& ph, Pr<T>* f)
{
    if constexpr (EQ == EQ_ADV) {
        f[0] = pmul(pbc(DIR == 0 ? ph.ax : ph.ay), q[0]);
    } else {
        const Pr<T> r = prcp(q[0]);
        const Pr<T> u = pmul(q[1], r), v = pmul(q[2], r);
        Pr<T> t = pmul(q[1], u);
        t = pfma(q[2], v, t);
        const Pr<T> p = pmul(pbc(ph.gamma - T(1)), pfma(pbc(T(-0.5)), t, q[3]));
        if constexpr (DIR == 0) {
            f[0] = q[1];
            f[1] = pfma(q[1], u, p);
            f[2] = pmul(q[2], u);
            f[3] = pmul(padd(q[3], p), u);
        } else {
            f[0] = q[2];
            f[1] = pmul(q[1], v);
            f[2] = pfma(q[2], v, p);
            f[3] = pmul(padd(q[3], p), v);
        }
    }
}

// sum_l c_l x_l over a line of 2 NP values held as NP pairs: products
// accumulated per lane, then the two lanes added.  Every edge state of the
// stage kernel (own or neighbour's) goes through this one sequence, so the
// two CTAs that share a face see the same bits.
template <int NP, class T>
__device__ __forceinline__ T pdot(const Pr<T>* c, const Pr<T>* x)
{
    Pr<T> s = pmul(c[0], x[0]);
#pragma unroll
    for (int j = 1; j < NP; ++j) s = pfma(c[j], x[j], s);
    return s.v.x + s.v.y;
}

// Operator tables in pairs over points (even N): D2[i][l] = (D[2i][l],
// D[2i+1][l]); lm2[j] = (lm[2j], lm[2j+1]) and likewise lp2, dgl2, dgr2.
template <class T>
struct TabPr {
    Pr<T> D2[(kMaxN + 1) / 2][kMaxN];
    Pr<T> lm2[(kMaxN + 1) / 2], lp2[(kMaxN + 1) / 2];
    Pr<T> dgl2[(kMaxN + 1) / 2], dgr2[(kMaxN + 1) / 2];
};

}  // namespace cpr
