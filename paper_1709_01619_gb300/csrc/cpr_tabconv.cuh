// cpr_tabconv.cuh -- FP64 host tables to the kernels' Tab<T>.
#pragma once

#include "cpr_launch.h"

namespace cpr {

template <class T>
inline Tab<T> host_tab(const HostTab& h)
{
    Tab<T> t;
    for (int a = 0; a < kMaxN; ++a) {
        for (int l = 0; l < kMaxN; ++l) {
            const bool in = a < h.n && l < h.n;
            t.D[a][l] = in ? T(h.D[a][l]) : T(0);
            t.cavg[a][l] = in ? T(h.w[a] * h.w[l] * 0.25) : T(0);
        }
        const bool in = a < h.n;
        t.lm[a] = in ? T(h.lm[a]) : T(0);
        t.lp[a] = in ? T(h.lp[a]) : T(0);
        t.dgl[a] = in ? T(h.dgl[a]) : T(0);
        t.dgr[a] = in ? T(h.dgr[a]) : T(0);
        t.w[a] = in ? T(h.w[a]) : T(0);
        t.xi[a] = in ? T(h.xi[a]) : T(0);
    }
    return t;
}


inline void set_pr(Pr<float>& p, double a, double b) { p.v = make_float2(float(a), float(b)); }
inline void set_pr(Pr<double>& p, double a, double b) { p.v = make_double2(a, b); }

// The tables in pairs over points (TabPr); entries past n are zero.
template <class T>
inline TabPr<T> host_tabpr(const HostTab& h)
{
    TabPr<T> t;
    auto at = [&](const double* a, int i) { return i < h.n ? a[i] : 0.0; };
    for (int i = 0; i < (kMaxN + 1) / 2; ++i) {
        for (int l = 0; l < kMaxN; ++l) {
            const double d0 = (2 * i < h.n && l < h.n) ? h.D[2 * i][l] : 0.0;
            const double d1 = (2 * i + 1 < h.n && l < h.n) ? h.D[2 * i + 1][l] : 0.0;
            set_pr(t.D2[i][l], d0, d1);
        }
        set_pr(t.lm2[i], at(h.lm, 2 * i), at(h.lm, 2 * i + 1));
        set_pr(t.lp2[i], at(h.lp, 2 * i), at(h.lp, 2 * i + 1));
        set_pr(t.dgl2[i], at(h.dgl, 2 * i), at(h.dgl, 2 * i + 1));
        set_pr(t.dgr2[i], at(h.dgr, 2 * i), at(h.dgr, 2 * i + 1));
    }
    return t;
}

}  // namespace cpr
