// cpr_fv_inst.cuh -- launcher of the FV stage kernel for one dtype; included
// by one translation unit per dtype.
#pragma once

#include "cpr_fv.cuh"
#include "cpr_stage_inst.cuh"

namespace cpr {

template <class T>
cudaError_t launch_fv(const LaunchCfg& c, int mode, const StagePtrs& b, bool do_wave, cudaStream_t s)
{
    StageArgs<T> A = make_stage_args<T>(c, mode, b, do_wave);
    A.tiles_x = (c.nx + kFvTX - 1) / kFvTX;
    A.do_avg = 0;  // FV runs have no troubled-cell limiter, hence no averages pass
    if (c.eqn == EQ_EULER)
        return c.flux == FLUX_ROE ? fv_one<T, EQ_EULER, FLUX_ROE>(c, A, s) : fv_one<T, EQ_EULER, FLUX_RUSANOV>(c, A, s);
    if (c.flux == FLUX_UPWIND) return fv_one<T, EQ_ADV, FLUX_UPWIND>(c, A, s);
    return fv_one<T, EQ_ADV, FLUX_RUSANOV>(c, A, s);
}

}  // namespace cpr

#define CPR_INSTANTIATE_FV(T)                                                                      \
    template cudaError_t cpr::launch_fv<T>(const LaunchCfg&, int, const StagePtrs&, bool, cudaStream_t);
