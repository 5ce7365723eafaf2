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

}  // namespace cpr
