// cpr_stage_inst.cuh -- launcher of the stage kernel for one (dtype, order);
// included by one translation unit per (dtype, order) so that they compile
// in parallel.
#pragma once

#include "cpr_launch.h"
#include "cpr_tabconv.cuh"
#include "cpr_stage.cuh"
#include "cpr_adjoint.cuh"

// Small-tile FP64 stage kernel for grids of at most one tile per two SMs
// (0: off).
#ifndef CPR_STAGE_SMALL
#define CPR_STAGE_SMALL 1
#endif

namespace cpr {


template <class T, int P, int EQ, int DIV, int FLUX>
static cudaError_t stage_one(const LaunchCfg& c, const StageArgs<T>& A, int ctas, cudaStream_t s, bool prep)
{
    constexpr int N = P + 1, V = NVars<EQ>::value;
    constexpr int TX = stage_tile_x(P), TY = stage_tile_y(P);
    constexpr int NT = TX * TY * N;
    const size_t smem = sizeof(T) * StageLayout<N, V, TX, TY, stage_delta<T>()>::TOTAL;
    auto kern = cpr_stage_kernel<T, P, EQ, DIV, FLUX, TX, TY, stage_delta<T>()>;
    // the prefetching instantiation only where the compensated FP32 stages
    // run on large states: Euler, LP divergence, Rusanov flux
    constexpr bool HAS_PF = sizeof(T) == 4 && EQ == EQ_EULER && DIV == DIV_LP && FLUX == FLUX_RUSANOV;
    auto kern_pf = cpr_stage_kernel<T, P, EQ, DIV, FLUX, TX, TY, stage_delta<T>(), HAS_PF>;
    // and the one for grids of at most two CTAs per SM: FP32 Euler, every
    // divergence and flux
    constexpr bool HAS_WIDE = sizeof(T) == 4 && EQ == EQ_EULER;
    auto kern_w = cpr_stage_kernel<T, P, EQ, DIV, FLUX, TX, TY, stage_delta<T>(), false, HAS_WIDE>;
    // CTAs per SM the wide instantiation is compiled for: the grid fits the
    // device at once up to that many per SM
    constexpr int WIDE_PER_SM = stage_min_blocks<T, N, true, TX * TY>();
    // and, in FP64, tiles of 4 x 4 elements for grids of at most one tile per
    // two SMs: four times the CTAs, so that more SMs share the FP64 work of a
    // grid that would leave most of them idle (Euler, LP divergence, Rusanov
    // flux; 24^2 p = 3 192.6 -> 109.9 ms for 1003 steps, 64^2 514 -> 317 ms;
    // at 96^2, 144 tiles, slower: 773 -> 807 ms; in FP32 slower at every size,
    // 24^2 17.1 -> 17.5 ms, 96^2 70.5 -> 78.9 ms)
    // (whole warps only: p = 1 and 3, 32 and 64 threads)
    constexpr int SX = 4, SY = 4;
    constexpr bool HAS_SMALL = sizeof(T) == 8 && EQ == EQ_EULER && DIV == DIV_LP && FLUX == FLUX_RUSANOV &&
                               (SX * SY * N) % 32 == 0 && CPR_STAGE_SMALL != 0;
    [[maybe_unused]] const size_t smem_s = sizeof(T) * StageLayout<N, V, SX, SY, stage_delta<T>()>::TOTAL;
    if (prep) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess && HAS_PF)
            e = cudaFuncSetAttribute(kern_pf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess && HAS_WIDE)
            e = cudaFuncSetAttribute(kern_w, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if constexpr (HAS_SMALL)
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(cpr_stage_kernel<T, P, EQ, DIV, FLUX, SX, SY, stage_delta<T>(), false, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_s);
        return e;
    }
    if constexpr (HAS_SMALL) {
        if (c.sms > 0 && 2 * ctas <= c.sms) {
            StageArgs<T> As = A;
            As.tiles_x = (c.nx + SX - 1) / SX;
            const int grid = As.tiles_x * ((c.ny + SY - 1) / SY);
            cpr_stage_kernel<T, P, EQ, DIV, FLUX, SX, SY, stage_delta<T>(), false, true>
                <<<grid, SX * SY * N, smem_s, s>>>(As);
            return cudaGetLastError();
        }
    }
    if (HAS_PF && A.pf_lo) kern_pf<<<ctas, NT, smem, s>>>(A);
    else if (HAS_WIDE && c.sms > 0 && ctas <= WIDE_PER_SM * c.sms) kern_w<<<ctas, NT, smem, s>>>(A);
    else kern<<<ctas, NT, smem, s>>>(A);
    return cudaGetLastError();
}

template <class T, int P>
static cudaError_t stage_dispatch(const LaunchCfg& c, const StageArgs<T>& A, int ctas, cudaStream_t s, bool prep)
{
    if (c.eqn == EQ_ADV) {
        if (c.flux == FLUX_UPWIND)
            return c.div == DIV_LP ? stage_one<T, P, EQ_ADV, DIV_LP, FLUX_UPWIND>(c, A, ctas, s, prep)
                                   : stage_one<T, P, EQ_ADV, DIV_CHAIN, FLUX_UPWIND>(c, A, ctas, s, prep);
        return c.div == DIV_LP ? stage_one<T, P, EQ_ADV, DIV_LP, FLUX_RUSANOV>(c, A, ctas, s, prep)
                               : stage_one<T, P, EQ_ADV, DIV_CHAIN, FLUX_RUSANOV>(c, A, ctas, s, prep);
    }
    if (c.flux == FLUX_ROE)
        return c.div == DIV_LP ? stage_one<T, P, EQ_EULER, DIV_LP, FLUX_ROE>(c, A, ctas, s, prep)
                               : stage_one<T, P, EQ_EULER, DIV_CHAIN, FLUX_ROE>(c, A, ctas, s, prep);
    return c.div == DIV_LP ? stage_one<T, P, EQ_EULER, DIV_LP, FLUX_RUSANOV>(c, A, ctas, s, prep)
                           : stage_one<T, P, EQ_EULER, DIV_CHAIN, FLUX_RUSANOV>(c, A, ctas, s, prep);
}

template <class T>
static StageArgs<T> make_stage_args(const LaunchCfg& c, int mode, const StagePtrs& b, bool do_wave)
{
    StageArgs<T> A;
    A.qs = static_cast<const T*>(b.qs);
    A.qb = static_cast<const T*>(b.qb);
    A.qn = static_cast<const T*>(b.qn);
    A.out = static_cast<T*>(b.out);
    A.lo = static_cast<T*>(b.lo);
    A.avg = static_cast<T*>(b.avg);
    A.ctrl = c.ctrl;
    A.npts = c.npts;
    A.nx = c.nx;
    A.ny = c.ny;
    A.bcx = c.bcx;
    A.bcy = c.bcy;
    A.tiles_x = (c.nx + stage_tile_x(c.p) - 1) / stage_tile_x(c.p);
    A.mode = mode;
    A.do_avg = b.avg != nullptr;
    A.do_wave = do_wave;
    // the five state arrays of the compensated stage exceed L2
    A.pf_lo = mode == MODE_INC3 && b.lo != nullptr &&
              (double)c.npts * (c.eqn == EQ_EULER ? 4 : 1) * sizeof(T) * 5.0 > (double)c.l2_bytes;
    A.rhx2 = T(2.0 / c.hx);
    A.rhy2 = T(2.0 / c.hy);
    A.ph.gamma = T(c.gamma);
    A.ph.ax = T(c.ax);
    A.ph.ay = T(c.ay);
    A.tab = host_tab<T>(c.tab);
    A.tp = host_tabpr<T>(c.tab);
    return A;
}

template <class T, int P>
cudaError_t launch_stage_p(const LaunchCfg& c, int mode, const StagePtrs& b, bool do_wave, cudaStream_t s)
{
    StageArgs<T> A = make_stage_args<T>(c, mode, b, do_wave);
    return stage_dispatch<T, P>(c, A, stage_ctas(c), s, false);
}

template <class T, int P>
cudaError_t prepare_stage_p(const LaunchCfg& c)
{
    StagePtrs b{};
    StageArgs<T> A = make_stage_args<T>(c, 0, b, false);
    return stage_dispatch<T, P>(c, A, 0, 0, true);
}

// Tile of the adjoint kernel: FP32 8 x 4 elements (twice as many CTAs per
// SM as 8 x 8 ones in the same shared memory: 1024^2 p = 3 0.441 -> 0.411 ms
// per launch; the height is overridable for tuning sweeps); FP64 8 x 8, or
// 8 x 4 where 8 x 8 would exceed the shared memory of one CTA.
#ifndef CPR_VJP_TILE_Y
#define CPR_VJP_TILE_Y 4
#endif
template <class T, int P>
struct VjpTile {
    static constexpr int X = 8;
    static constexpr int Y = sizeof(T) == 8 ? (P == 4 ? 4 : 8) : CPR_VJP_TILE_Y;
};

template <class T, int P, int EQ, int FLUX>
static cudaError_t vjp_one(const LaunchCfg& c, const VjpPtrs& b, cudaStream_t s, bool prep)
{
    constexpr int N = P + 1, V = NVars<EQ>::value;
    constexpr int TX = VjpTile<T, P>::X, TY = VjpTile<T, P>::Y;
    auto kern = cpr_residual_vjp_kernel<T, P, EQ, FLUX, TX, TY>;
    const size_t smem = sizeof(T) * VjpLayout<N, V, TX, TY>::TOTAL;
    if (prep) return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    VjpArgs<T> A;
    A.q = static_cast<const T*>(b.q);
    A.rbar = static_cast<const T*>(b.rbar);
    A.out = static_cast<T*>(b.out);
    A.X0 = static_cast<const T*>(b.X0);
    A.X1 = static_cast<const T*>(b.X1);
    A.X2 = static_cast<const T*>(b.X2);
    A.c0 = T(b.c0);
    A.c1 = T(b.c1);
    A.c2 = T(b.c2);
    A.cv = T(b.cv);
    A.npts = c.npts;
    A.nx = c.nx;
    A.ny = c.ny;
    A.bcx = c.bcx;
    A.bcy = c.bcy;
    A.tiles_x = (c.nx + TX - 1) / TX;
    A.rhx2 = T(2.0 / c.hx);
    A.rhy2 = T(2.0 / c.hy);
    A.ph.gamma = T(c.gamma);
    A.ph.ax = T(c.ax);
    A.ph.ay = T(c.ay);
    A.tab = host_tab<T>(c.tab);
    for (int a = 0; a < kMaxN; ++a)
        for (int l = 0; l < kMaxN; ++l)
            A.M[a][l] = (a < N && l < N)
                            ? T(c.tab.D[a][l] - c.tab.lm[l] * c.tab.dgl[a] - c.tab.lp[l] * c.tab.dgr[a])
                            : T(0);
    const int ctas = A.tiles_x * ((c.ny + TY - 1) / TY);
    kern<<<ctas, TX * TY * N, smem, s>>>(A);
    return cudaGetLastError();
}

template <class T, int P>
cudaError_t launch_vjp_p(const LaunchCfg& c, const VjpPtrs& b, cudaStream_t s, bool prep)
{
    if (c.eqn == EQ_EULER) return vjp_one<T, P, EQ_EULER, FLUX_RUSANOV>(c, b, s, prep);
    if (c.flux == FLUX_UPWIND) return vjp_one<T, P, EQ_ADV, FLUX_UPWIND>(c, b, s, prep);
    return vjp_one<T, P, EQ_ADV, FLUX_RUSANOV>(c, b, s, prep);
}

}  // namespace cpr

#define CPR_INSTANTIATE_STAGE(T, P)                                                                     \
    template cudaError_t cpr::launch_stage_p<T, P>(const LaunchCfg&, int, const StagePtrs&, bool, cudaStream_t); \
    template cudaError_t cpr::prepare_stage_p<T, P>(const LaunchCfg&);                                  \
    template cudaError_t cpr::launch_vjp_p<T, P>(const LaunchCfg&, const VjpPtrs&, cudaStream_t, bool);
