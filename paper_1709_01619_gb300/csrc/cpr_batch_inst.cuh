// cpr_batch_inst.cuh -- host launchers of the batched stage kernels for one
// (dtype, tile family); included by one translation unit each.
#pragma once

#include "cpr_batch.cuh"
#include "cpr_tabconv.cuh"

namespace cpr {

template <class T, int P, int EQ, int FLUX, int FAM>
static cudaError_t batch_one(const BatchArgs<T>& B, int grid, cudaStream_t s, int what, int* occ)
{
    constexpr int N = P + 1, V = NVars<EQ>::value;
    constexpr int TX = BatchTile<FAM>::X, TY = BatchTile<FAM>::Y;
    constexpr int NT = TX * TY * N;
    auto loop = cpr_batch_stage_kernel<T, P, EQ, DIV_LP, FLUX, TX, TY, stage_delta<T>(), true>;
    auto flat = cpr_batch_stage_kernel<T, P, EQ, DIV_LP, FLUX, TX, TY, stage_delta<T>(), false>;
    const size_t smem = sizeof(T) * StageLayout<N, V, TX, TY, stage_delta<T>()>::TOTAL;
    if (what == 1) {
        cudaError_t e = cudaFuncSetAttribute(loop, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        return cudaFuncSetAttribute(flat, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    if (what == 2) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, loop, NT, smem);
    // a grid as large as the work list takes the one-tile-per-CTA form
    if (grid >= B.total) flat<<<B.total, NT, smem, s>>>(B);
    else loop<<<grid, NT, smem, s>>>(B);
    return cudaGetLastError();
}

template <class T, int P, int FAM>
static cudaError_t batch_p(int eqn, int flux, const BatchArgs<T>& B, int grid, cudaStream_t s, int what, int* occ)
{
    if (eqn == EQ_EULER) return batch_one<T, P, EQ_EULER, FLUX_RUSANOV, FAM>(B, grid, s, what, occ);
    if (flux == FLUX_UPWIND) return batch_one<T, P, EQ_ADV, FLUX_UPWIND, FAM>(B, grid, s, what, occ);
    return batch_one<T, P, EQ_ADV, FLUX_RUSANOV, FAM>(B, grid, s, what, occ);
}

template <class T, int FAM>
cudaError_t batch_fam(int p, int eqn, int flux, const BatchArgs<T>& B, int grid, cudaStream_t s, int what,
                      int* occ)
{
    switch (p) {
    case 1: return batch_p<T, 1, FAM>(eqn, flux, B, grid, s, what, occ);
    case 2: return batch_p<T, 2, FAM>(eqn, flux, B, grid, s, what, occ);
    case 3: return batch_p<T, 3, FAM>(eqn, flux, B, grid, s, what, occ);
    case 4: return batch_p<T, 4, FAM>(eqn, flux, B, grid, s, what, occ);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace cpr

#define CPR_INSTANTIATE_BATCH(T, FAM)                                                                        \
    template cudaError_t cpr::batch_fam<T, FAM>(int, int, int, const BatchArgs<T>&, int, cudaStream_t, int, \
                                                int*);
