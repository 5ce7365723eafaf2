// cpr_aux_inst.cuh -- per-dtype launchers: order dispatch of the stage
// kernel and the element-wise passes.  Included by one translation unit per
// dtype.
#pragma once

#include "cpr_aux.cuh"
#include "cpr_launch.h"
#include "cpr_tabconv.cuh"

namespace cpr {


template <class T>
static AuxArgs<T> make_aux(const LaunchCfg& c)
{
    AuxArgs<T> A;
    A.q = nullptr;
    A.ref = nullptr;
    A.avg_in = nullptr;
    A.avg_out = nullptr;
    A.marks = c.marks;
    A.ctrl = c.ctrl;
    A.partials = c.partials;
    A.ne = c.ne;
    A.npts = c.npts;
    A.nx = c.nx;
    A.ny = c.ny;
    div_magic((unsigned int)c.nx, &A.nx_magic, &A.nx_shift);
    A.bcx = c.bcx;
    A.bcy = c.bcy;
    A.do_wave = 0;
    A.check_done = 0;
    A.hx = T(c.hx);
    A.hy = T(c.hy);
    A.tvb_M = T(c.tvb_M);
    A.lim_eps = T(c.lim_eps);
    A.ph.gamma = T(c.gamma);
    A.ph.ax = T(c.ax);
    A.ph.ay = T(c.ay);
    A.tab = host_tab<T>(c.tab);
    A.tab64 = host_tab<double>(c.tab);
    A.gamma64 = c.gamma;
    A.ax64 = c.ax;
    A.ay64 = c.ay;
    return A;
}

// Dispatch an element-wise kernel template over (order, equation).
#define CPR_AUX_DISPATCH(KERNEL, GRID, BLOCK, STREAM, ARGS)                                      \
    do {                                                                                         \
        const bool euler = c.eqn == EQ_EULER;                                                    \
        switch (c.p) {                                                                           \
        case 0: if (euler) KERNEL<T, 0, EQ_EULER><<<GRID, BLOCK, 0, STREAM>>>(ARGS);             \
                else KERNEL<T, 0, EQ_ADV><<<GRID, BLOCK, 0, STREAM>>>(ARGS); break;              \
        case 1: if (euler) KERNEL<T, 1, EQ_EULER><<<GRID, BLOCK, 0, STREAM>>>(ARGS);             \
                else KERNEL<T, 1, EQ_ADV><<<GRID, BLOCK, 0, STREAM>>>(ARGS); break;              \
        case 2: if (euler) KERNEL<T, 2, EQ_EULER><<<GRID, BLOCK, 0, STREAM>>>(ARGS);             \
                else KERNEL<T, 2, EQ_ADV><<<GRID, BLOCK, 0, STREAM>>>(ARGS); break;              \
        case 3: if (euler) KERNEL<T, 3, EQ_EULER><<<GRID, BLOCK, 0, STREAM>>>(ARGS);             \
                else KERNEL<T, 3, EQ_ADV><<<GRID, BLOCK, 0, STREAM>>>(ARGS); break;              \
        case 4: if (euler) KERNEL<T, 4, EQ_EULER><<<GRID, BLOCK, 0, STREAM>>>(ARGS);             \
                else KERNEL<T, 4, EQ_ADV><<<GRID, BLOCK, 0, STREAM>>>(ARGS); break;              \
        default: return cudaErrorInvalidValue;                                                   \
        }                                                                                        \
    } while (0)

template <class T>
cudaError_t launch_stage(const LaunchCfg& c, int mode, const StagePtrs& b, bool do_wave, cudaStream_t s)
{
    switch (c.p) {
    case 0: return launch_fv<T>(c, mode, b, do_wave, s);
    case 1: return launch_stage_p<T, 1>(c, mode, b, do_wave, s);
    case 2: return launch_stage_p<T, 2>(c, mode, b, do_wave, s);
    case 3: return launch_stage_p<T, 3>(c, mode, b, do_wave, s);
    case 4: return launch_stage_p<T, 4>(c, mode, b, do_wave, s);
    default: return cudaErrorInvalidValue;
    }
}

template <class T>
cudaError_t launch_stage(const LaunchCfg& c, int mode, const void* qs, const void* qn, void* out, void* avg,
                         bool do_wave, cudaStream_t s)
{
    StagePtrs b{qs, nullptr, qn, out, nullptr, avg};
    return launch_stage<T>(c, mode, b, do_wave, s);
}

template <class T>
cudaError_t launch_vjp(const LaunchCfg& c, const VjpPtrs& b, cudaStream_t s, bool prep)
{
    switch (c.p) {
    case 1: return launch_vjp_p<T, 1>(c, b, s, prep);
    case 2: return launch_vjp_p<T, 2>(c, b, s, prep);
    case 3: return launch_vjp_p<T, 3>(c, b, s, prep);
    case 4: return launch_vjp_p<T, 4>(c, b, s, prep);
    default: return cudaErrorInvalidValue;
    }
}

template <class T>
cudaError_t prepare_stage(const LaunchCfg& c)
{
    switch (c.p) {
    case 0: return cudaSuccess;  // the FV kernel uses static shared memory only
    case 1: return prepare_stage_p<T, 1>(c);
    case 2: return prepare_stage_p<T, 2>(c);
    case 3: return prepare_stage_p<T, 3>(c);
    case 4: return prepare_stage_p<T, 4>(c);
    default: return cudaErrorInvalidValue;
    }
}

// Element-wise kernels: grid of ceil(ne / EB) CTAs of EB threads.
template <class T, int P, int EQ>
static void elem_launch(bool lim, const AuxArgs<T>& A, cudaStream_t s)
{
    constexpr int EB = AuxShape<T, P, EQ>::EB;
    const int grid = (int)((A.ne + EB - 1) / EB);
    if (lim) cpr_limit_kernel<T, P, EQ><<<grid, LimShape<T, P, EQ>::NT, 0, s>>>(A);
    else cpr_averages_kernel<T, P, EQ><<<grid, EB, 0, s>>>(A);
}

template <class T>
static cudaError_t elem_dispatch(const LaunchCfg& c, bool lim, const AuxArgs<T>& A, cudaStream_t s)
{
    const bool eu = c.eqn == EQ_EULER;
    switch (c.p) {
    case 1: eu ? elem_launch<T, 1, EQ_EULER>(lim, A, s) : elem_launch<T, 1, EQ_ADV>(lim, A, s); break;
    case 2: eu ? elem_launch<T, 2, EQ_EULER>(lim, A, s) : elem_launch<T, 2, EQ_ADV>(lim, A, s); break;
    case 3: eu ? elem_launch<T, 3, EQ_EULER>(lim, A, s) : elem_launch<T, 3, EQ_ADV>(lim, A, s); break;
    case 4: eu ? elem_launch<T, 4, EQ_EULER>(lim, A, s) : elem_launch<T, 4, EQ_ADV>(lim, A, s); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_averages(const LaunchCfg& c, const void* q, void* avg, cudaStream_t s)
{
    AuxArgs<T> A = make_aux<T>(c);
    A.q = const_cast<T*>(static_cast<const T*>(q));
    A.avg_out = static_cast<T*>(avg);
    return elem_dispatch<T>(c, false, A, s);
}

template <class T>
cudaError_t launch_limit(const LaunchCfg& c, void* q, const void* avg, int role, cudaStream_t s)
{
    AuxArgs<T> A = make_aux<T>(c);
    A.q = static_cast<T*>(q);
    A.avg_in = static_cast<const T*>(avg);
    A.do_wave = role == 2;
    A.check_done = role >= 1;
    return elem_dispatch<T>(c, true, A, s);
}

template <class T>
cudaError_t launch_wave(const LaunchCfg& c, const void* q, cudaStream_t s)
{
    AuxArgs<T> A = make_aux<T>(c);
    A.q = const_cast<T*>(static_cast<const T*>(q));
    const long long want = (c.npts + 255) / 256;
    const int grid = (int)(want < 1024 ? want : 1024);
    CPR_AUX_DISPATCH(cpr_wave_kernel, grid, 256, s, A);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_norms(const LaunchCfg& c, const void* q, const void* ref, int nblocks, cudaStream_t s)
{
    AuxArgs<T> A = make_aux<T>(c);
    A.q = const_cast<T*>(static_cast<const T*>(q));
    A.ref = static_cast<const T*>(ref);
    CPR_AUX_DISPATCH(cpr_norms_kernel, nblocks, kNormThreads, s, A);
    return cudaGetLastError();
}

}  // namespace cpr

#define CPR_INSTANTIATE_AUX(T)                                                                              \
    template cudaError_t cpr::launch_stage<T>(const LaunchCfg&, int, const void*, const void*, void*, void*, \
                                              bool, cudaStream_t);                                          \
    template cudaError_t cpr::launch_stage<T>(const LaunchCfg&, int, const StagePtrs&, bool, cudaStream_t);  \
    template cudaError_t cpr::prepare_stage<T>(const LaunchCfg&);                                            \
    template cudaError_t cpr::launch_vjp<T>(const LaunchCfg&, const VjpPtrs&, cudaStream_t, bool);          \
    template cudaError_t cpr::launch_averages<T>(const LaunchCfg&, const void*, void*, cudaStream_t);        \
    template cudaError_t cpr::launch_limit<T>(const LaunchCfg&, void*, const void*, int, cudaStream_t);      \
    template cudaError_t cpr::launch_wave<T>(const LaunchCfg&, const void*, cudaStream_t);                   \
    template cudaError_t cpr::launch_norms<T>(const LaunchCfg&, const void*, const void*, int, cudaStream_t);
