// cpr_batch.cuh -- many independent CPR problems of uneven size and order,
// advanced together.
//
// The instances are grouped by polynomial order p.  For each RK stage there
// is one persistent launch per order present: its CTAs walk the work list of
// all tiles of all instances of that order (instance-major, each instance's
// tiles row-major) with a grid stride, and run the same tile body as the
// single-problem kernel.  Each instance keeps its own time-control block
// (step size, running maximum speed); the last tile of an instance to
// finish closes that instance's step.  Tile shape (family) and the number of
// resident CTAs per SM are chosen by the autotuner (cpr_batch_tune).
#pragma once

#include "cpr_launch.h"
#include "cpr_stage.cuh"

namespace cpr {

// Tile families: 0 = 8 x 8 elements, 1 = 16 x 4 elements.
template <int FAM>
struct BatchTile {
    static constexpr int X = FAM == 0 ? 8 : 16;
    static constexpr int Y = FAM == 0 ? 8 : 4;
};

// Per-instance data of a batch (device memory, one entry per instance of the
// order group).
template <class T>
struct BatchInst {
    T* X;          // caller's state
    T* Y;          // stage buffer / alternate high part
    T* Z;          // stage buffer
    T* lo;         // low part (FP32 increment form)
    Ctrl* ctrl;
    long long npts;
    int nx, ny, bcx, bcy;
    int tiles_x, ntiles, tile0;  // tiles of this instance, its first work item
    T rhx2, rhy2;
    Phys<T> ph;
};

template <class T>
struct BatchArgs {
    const BatchInst<T>* inst;
    const int* tile_inst;  // work item -> instance of the group
    int ninst, total;  // instances of the group, work items
    int mode;          // stage mode (cpr_common.cuh)
    int swap;          // increment form: the high part of q^n is in Y (else X)
    Tab<T> tab;        // operator tables of the group's order
    TabPr<T> tp;       // the same in pairs over points
};

// Register budget: as the single-problem kernel.
template <class T, int N>
constexpr int batch_min_blocks()
{
    return stage_min_blocks<T, N>();
}

// One work item (tile w of the group's list): thread 0 looks up its
// instance (one load from the work-item map, instead of a binary search of
// dependent loads that the whole CTA would wait out) and fills the stage
// arguments in shared memory, then the CTA runs the tile.
template <class T, int P, int EQ, int DIV, int FLUX, int TX, int TY, bool DELTA>
__device__ __forceinline__ void batch_item(const BatchArgs<T>& B, int w, StageArgs<T>& sA, int& s_t, int& s_n,
                                           unsigned char* smem_raw)
{
    if (threadIdx.x == 0) {
        const BatchInst<T>& I = B.inst[B.tile_inst[w]];
        StageArgs<T>& A = sA;
        A.npts = I.npts;
        A.nx = I.nx;
        A.ny = I.ny;
        A.bcx = I.bcx;
        A.bcy = I.bcy;
        A.tiles_x = I.tiles_x;
        A.mode = B.mode;
        A.do_avg = 0;
        A.avg = nullptr;
        A.do_wave = B.mode == MODE_SO3 || B.mode == MODE_INC3;
        A.pf_lo = 0;
        A.ctrl = I.ctrl;
        A.rhx2 = I.rhx2;
        A.rhy2 = I.rhy2;
        A.ph = I.ph;
        A.qb = nullptr;
        A.qn = nullptr;
        A.lo = I.lo;
        T* hiq = B.swap ? I.Y : I.X;
        T* other = B.swap ? I.X : I.Y;
        switch (B.mode) {
        case MODE_SO1: A.qs = I.X; A.out = I.Y; break;
        case MODE_SO2: A.qs = I.Y; A.qn = I.X; A.out = I.Z; break;
        case MODE_SO3: A.qs = I.Z; A.qn = I.X; A.out = I.X; break;
        case MODE_INC1: A.qs = hiq; A.out = other; break;
        case MODE_INC2: A.qs = hiq; A.qb = other; A.out = I.Z; break;
        default: A.qs = hiq; A.qb = I.Z; A.out = other; break;
        }
        s_t = w - I.tile0;
        s_n = I.ntiles;
    }
    __syncthreads();
    stage_tile<T, P, EQ, DIV, FLUX, TX, TY, DELTA>(sA, B.tab, B.tp, s_t, threadIdx.x, smem_raw, s_n);
}

// PERSIST: CTAs walk the work list with a grid stride; otherwise the grid
// has one CTA per work item.  The loop costs registers (the tile body spills
// more inside it), so the autotuner weighs both forms.
template <class T, int P, int EQ, int DIV, int FLUX, int TX, int TY, bool DELTA, bool PERSIST>
__global__ void __launch_bounds__(TX * TY * (P + 1), (batch_min_blocks<T, P + 1>()))
cpr_batch_stage_kernel(const BatchArgs<T> B)
{
    static_assert((TX * TY * (P + 1)) % 32 == 0, "whole warps: the warp-level reductions use every lane");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // The work item's arguments live in shared memory, read at their points
    // of use instead of occupying registers through the whole tile.
    __shared__ StageArgs<T> sA;
    __shared__ int s_t, s_n;
    if constexpr (PERSIST) {
        for (int w = blockIdx.x; w < B.total; w += gridDim.x) {
            batch_item<T, P, EQ, DIV, FLUX, TX, TY, DELTA>(B, w, sA, s_t, s_n, smem_raw);
            __syncthreads();
        }
    } else {
        batch_item<T, P, EQ, DIV, FLUX, TX, TY, DELTA>(B, blockIdx.x, sA, s_t, s_n, smem_raw);
    }
}

}  // namespace cpr
