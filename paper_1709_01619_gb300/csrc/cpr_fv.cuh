// cpr_fv.cuh -- the finite-volume comparison scheme of the paper, fused into
// one SSP-RK3 stage kernel.
//
// One average per element (Sec. 2.1):
//   dq_ij/dt = -(f_{i+1/2,j} - f_{i-1/2,j}) / dx - (g_{i,j+1/2} - g_{i,j-1/2}) / dy,
// the face states reconstructed by second-order MUSCL with minmod-limited
// slopes (Sec. 2.6), q_face = q_i +- (1/2) minmod(q_{i+1} - q_i, q_i - q_{i-1}),
// and the face flux from the same common flux as the CPR kernel
// (reconstruct, then Riemann flux: Algorithm 1).  ORDER 3 takes the
// third-order MUSCL face values of Sec. 2.6 (van Leer's kappa = 1/3, each
// one-sided difference D-, D+ limited by minmod against four times the other):
//   q_{i+1/2}^- = q_i + mm(D-, 4 D+)/6 + mm(D+, 4 D-)/3,
//   q_{i-1/2}^+ = q_i - mm(D+, 4 D-)/6 - mm(D-, 4 D+)/3,
// on the same five-element stencil.  Ghost elements: periodic directions
// wrap, transmissive ones repeat the boundary element.
//
// CTA: a tile of 32 x 8 elements, one thread per element.  Phase 1 stages
// the tile with a ring of two elements in shared memory; phase 2 evaluates
// every face of the tile once (the faces on the tile boundary are also
// evaluated by the neighbouring CTA, from the same values and in the same
// order, so the flux leaving one element is the flux entering the next);
// phase 3 forms the residual, applies the RK stage (the modes of the CPR
// stage kernel) and stores, with the fused maximum signal speed on the last
// stage.
#pragma once

#include "cpr_common.cuh"
#include "cpr_launch.h"
#include "cpr_reduce.cuh"
#include "cpr_stage.cuh"

namespace cpr {

constexpr int kFvTX = 32, kFvTY = 8;

// Wrapped (periodic) or clamped (transmissive) element index, for indices
// at most two outside [0, n) (no integer division: n may be 1).
__device__ __forceinline__ int fv_ghost(int i, int n, int transmissive)
{
    if (transmissive) return min(max(i, 0), n - 1);
    while (i < 0) i += n;
    while (i >= n) i -= n;
    return i;
}

// Face states of element b (neighbours a below, c above along the line):
// its value on the upper face (up) and on the lower face (down).
template <int ORDER, class T>
__device__ __forceinline__ T fv_up(T a, T b, T c)
{
    if constexpr (ORDER == 2) {
        return b + T(0.5) * minmod2(c - b, b - a);
    } else {
        const T dm = b - a, dp = c - b;
        return b + (minmod2(dm, T(4) * dp) * T(1.0 / 6.0) + minmod2(dp, T(4) * dm) * T(1.0 / 3.0));
    }
}
template <int ORDER, class T>
__device__ __forceinline__ T fv_down(T a, T b, T c)
{
    if constexpr (ORDER == 2) {
        return b - T(0.5) * minmod2(c - b, b - a);
    } else {
        const T dm = b - a, dp = c - b;
        return b - (minmod2(dp, T(4) * dm) * T(1.0 / 6.0) + minmod2(dm, T(4) * dp) * T(1.0 / 3.0));
    }
}

template <class T, int EQ, int FLUX, int ORDER>
__global__ void __launch_bounds__(kFvTX * kFvTY) cpr_fv_stage_kernel(const StageArgs<T> A)
{
    constexpr int TX = kFvTX, TY = kFvTY, NT = TX * TY, HX = TX + 4, HY = TY + 4;
    constexpr int V = NVars<EQ>::value;
    __shared__ T s[V][HY][HX];           // tile and two-element ring; s[v][ly][lx] = element (lx-2, ly-2)
    __shared__ T fx[V][TY][TX + 1];      // x-face fluxes; face fi between elements fi-1 and fi
    __shared__ T gy[V][TY + 1][TX];      // y-face fluxes; face fj between elements fj-1 and fj

    if (A.mode > 0 && A.ctrl->done) return;  // t_end reached: uniform exit
    const int tid = threadIdx.x;
    const int i0 = (blockIdx.x % A.tiles_x) * TX, j0 = (blockIdx.x / A.tiles_x) * TY;
    const int TXe = min(TX, A.nx - i0), TYe = min(TY, A.ny - j0);
    const bool addb = A.mode == MODE_INC2 || A.mode == MODE_INC3;

    // ---- phase 1: stage input of the tile and its ring --------------------
    for (int t = tid; t < HX * HY; t += NT) {
        const int lx = t % HX, ly = t / HX;
        const int gi = fv_ghost(i0 + lx - 2, A.nx, A.bcx), gj = fv_ghost(j0 + ly - 2, A.ny, A.bcy);
        const long long e = (long long)gj * A.nx + gi;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            T x = A.qs[v * A.npts + e];
            if (addb) x += A.qb[v * A.npts + e];
            s[v][ly][lx] = x;
        }
    }
    __syncthreads();

    // ---- phase 2: reconstruction and common flux on every face -------------
    for (int f = tid; f < (TX + 1) * TY; f += NT) {
        const int fi = f % (TX + 1), fj = f / (TX + 1);
        if (fi > TXe || fj >= TYe) continue;
        T qm[V], qp[V], F[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const T* r = &s[v][fj + 2][fi];  // elements fi-2 .. fi+1
            qm[v] = fv_up<ORDER>(r[0], r[1], r[2]);
            qp[v] = fv_down<ORDER>(r[1], r[2], r[3]);
        }
        common_flux<EQ, FLUX, 0>(qm, qp, A.ph, F);
#pragma unroll
        for (int v = 0; v < V; ++v) fx[v][fj][fi] = F[v];
    }
    for (int f = tid; f < TX * (TY + 1); f += NT) {
        const int fi = f % TX, fj = f / TX;
        if (fi >= TXe || fj > TYe) continue;
        T qm[V], qp[V], F[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const T a = s[v][fj][fi + 2], b = s[v][fj + 1][fi + 2], c = s[v][fj + 2][fi + 2],
                    d = s[v][fj + 3][fi + 2];  // elements fj-2 .. fj+1
            qm[v] = fv_up<ORDER>(a, b, c);
            qp[v] = fv_down<ORDER>(b, c, d);
        }
        common_flux<EQ, FLUX, 1>(qm, qp, A.ph, F);
#pragma unroll
        for (int v = 0; v < V; ++v) gy[v][fj][fi] = F[v];
    }
    __syncthreads();

    // ---- phase 3: residual, stage update, store -----------------------------
    const int tx = tid % TX, ty = tid / TX;
    const bool valid = tx < TXe && ty < TYe;
    T o[V];
    if (valid) {
        const T ihx = T(0.5) * A.rhx2, ihy = T(0.5) * A.rhy2;  // 1/dx, 1/dy
        const long long e = (long long)(j0 + ty) * A.nx + (i0 + tx);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const T r = -(fx[v][ty][tx + 1] - fx[v][ty][tx]) * ihx - (gy[v][ty + 1][tx] - gy[v][ty][tx]) * ihy;
            const long long k = v * A.npts + e;
            T y = r;
            if (A.mode == MODE_RESIDUAL) {
            } else if (A.mode <= MODE_SO3) {
                const T dt = T(A.ctrl->dt);
                const T qs = A.qs[k];
                if (A.mode == MODE_SO1) {
                    y = qs + dt * r;
                } else {
                    const T cA = A.mode == MODE_SO2 ? T(0.75) : T(1.0 / 3.0);
                    const T cB = A.mode == MODE_SO2 ? T(0.25) : T(2.0 / 3.0);
                    y = cA * A.qn[k] + cB * (qs + dt * r);
                }
            } else {
                const T dt = T(A.ctrl->dt);
                if (A.mode == MODE_INC1) {
                    y = dt * r;
                } else if (A.mode == MODE_INC2) {
                    y = T(0.25) * (A.qb[k] + dt * r);
                } else {
                    T hi = A.qs[k], lo = A.lo[k];
                    compensated_add(hi, lo, T(2.0 / 3.0) * (A.qb[k] + dt * r));
                    A.lo[k] = lo;
                    y = hi;
                }
            }
            A.out[k] = y;
            o[v] = y;
        }
    }
    if (A.do_wave) {
        T m = valid ? point_speed<EQ>(o, A.ph) : T(0);
        block_time_update<T>(m, A.ctrl, /*advance=*/true, gridDim.x);
    }
}

template <class T, int EQ, int FLUX>
static cudaError_t fv_one(const LaunchCfg& c, const StageArgs<T>& A, cudaStream_t s)
{
    const int ctas = ((c.nx + kFvTX - 1) / kFvTX) * ((c.ny + kFvTY - 1) / kFvTY);
    if (c.fv_order == 3) cpr_fv_stage_kernel<T, EQ, FLUX, 3><<<ctas, kFvTX * kFvTY, 0, s>>>(A);
    else cpr_fv_stage_kernel<T, EQ, FLUX, 2><<<ctas, kFvTX * kFvTY, 0, s>>>(A);
    return cudaGetLastError();
}

}  // namespace cpr
